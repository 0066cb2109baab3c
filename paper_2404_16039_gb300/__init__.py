"""Python binding of libvla (GB300 page-wise linear algebra and FE assembly).

Argument marshalling only: every computation happens in the CUDA kernels of
``libvla.so`` behind the C ABI declared in ``include/vla.h``.  PyTorch
supplies device memory and the current CUDA stream.  There is no CPU path:
if the shared library is missing or fails to load, every call raises.

Shapes (torch tensors on the current CUDA device, C-contiguous):
  page layout  (N, cols, rows)  -- page k is a column-major rows x cols matrix,
                                   exactly the paper's n x m x N array;
  SoA layout   (cols, rows, N)  -- entry (r, c) of page k at [c, r, k].
  mesh coords  (nn, dim) float64, elems (ne, nlb) int32, faces (nfb, dim) int32.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

__all__ = [
    "VlaError", "lib", "version", "amtam", "astam", "avtam", "amdet", "aminv", "amt", "avtav", "amsm", "amsv",
    "smamt", "svamt", "Mesh", "element_pages_static", "static_skipped", "partition_rows",
    "Batch", "batch_assemble", "autotune", "tune_get", "tune_set", "Server", "PENDING", "quad_rule", "gi",
    "avtamav", "F32", "F64", "LAYOUT_PAGE", "LAYOUT_SOA", "PREC_FP64", "PREC_MIXED", "COEFF_POLY", "COEFF_EXP",
    "COEFF_POLY_IP", "COEFF_EXP_IP",
]

F32, F64 = 0, 1
LAYOUT_PAGE, LAYOUT_SOA = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
COEFF_POLY, COEFF_EXP, COEFF_POLY_IP, COEFF_EXP_IP = 0, 1, 2, 3
VLA_ERR_INDEX_OOB = -2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvla.so")
_lock = threading.Lock()
_lib = None


class VlaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"vla status {status}: {message}")
        self.status = status


class _DeviceArray:
    """An int32 device array owned by the library, exposed through the CUDA
    array interface so that torch.as_tensor makes a view of it without a copy;
    the view keeps this object, and through it the owning handle, alive."""

    def __init__(self, ptr, n, owner):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i4", "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}
        self._owner = owner


class MeshInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("order", C.c_int32), ("nlb", C.c_int32),
                ("nn", C.c_int64), ("ne", C.c_int64), ("nfb", C.c_int64), ("nnz", C.c_int64),
                ("max_row_len", C.c_int32), ("n_tiles", C.c_int32), ("device_bytes", C.c_int64),
                ("tile_elems", C.c_int64), ("n_codes", C.c_int64), ("tile_budget", C.c_int32),
                ("reserved", C.c_int32), ("smem_bytes", C.c_int64)]


class BatchJob(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("coeff_kind", C.c_int32), ("reserved", C.c_int32),
                ("ca", C.c_double), ("cb", C.c_double), ("K_vals", C.c_void_p), ("M_vals", C.c_void_p),
                ("vol", C.c_void_p), ("K_pages", C.c_void_p), ("M_pages", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("count", C.c_int32), ("n_work", C.c_int32), ("grid", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("smem_bytes", C.c_int64), ("elements", C.c_int64), ("tile_elems", C.c_int64),
                ("graph", C.c_int32), ("split", C.c_int32)]


class Tune(C.Structure):
    _fields_ = [("tile_budget", C.c_int32), ("ctas_per_sm", C.c_int32), ("us", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("precision", C.c_int32), ("ingest_workers", C.c_int32),
                ("max_batch", C.c_int32), ("max_inflight", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("key", C.c_int64), ("dim", C.c_int32), ("order", C.c_int32), ("nn", C.c_int64),
                ("ne", C.c_int64), ("nfb", C.c_int64), ("coords", C.c_void_p), ("elems", C.c_void_p),
                ("faces", C.c_void_p), ("keep_resident", C.c_int32), ("coeff_kind", C.c_int32),
                ("ca", C.c_double), ("cb", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("new_mesh", C.c_int32), ("batch_size", C.c_int32),
                ("reserved", C.c_int32), ("batch_id", C.c_int64), ("nn", C.c_int64), ("ne", C.c_int64),
                ("nnz", C.c_int64), ("K_vals", C.c_void_p), ("M_vals", C.c_void_p), ("vol", C.c_void_p),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_ready", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("t_ingest", C.c_double), ("h2d_ms", C.c_double), ("build_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("budget_bytes", "used_bytes", "peak_bytes", "n_done", "n_failed",
                                         "n_batches", "n_ingested", "n_reused", "n_evicted", "n_resident",
                                         "n_queued", "max_batch")] + [("mean_batch", C.c_double),
                                                                      ("assembly_busy_s", C.c_double)]


BATCH_GRAPH, BATCH_FUSED, BATCH_SPLIT, BATCH_AUTOTUNE = 1, 2, 4, 8
PENDING = 2


def lib():
    """The loaded libvla.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(python paper_2404_16039_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.vla_version.restype = i32
        L.vla_last_error.argtypes = [C.c_char_p, C.c_size_t]
        L.vla_last_error.restype = C.c_size_t
        L.vla_amtam.argtypes = [i32, i32, i64, i32, i32, i32, vp, vp, vp, vp]
        L.vla_astam.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp, vp]
        L.vla_avtam.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp, vp]
        L.vla_amdet.argtypes = [i32, i32, i64, i32, vp, vp, vp]
        L.vla_aminv.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp, vp]
        L.vla_amt.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp]
        L.vla_avtav.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp]
        L.vla_amsm.argtypes = [i32, i32, i64, i32, i32, i32, vp, vp, vp, vp]
        L.vla_amsv.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp, vp]
        L.vla_smamt.argtypes = [i32, i32, i64, i32, i32, i32, vp, vp, vp, vp]
        L.vla_svamt.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp, vp]
        L.vla_mesh_create.argtypes = [i32, i32, i64, i64, vp, vp, i64, vp, vp, C.POINTER(vp)]
        L.vla_mesh_info.argtypes = [vp, C.POINTER(MeshInfo)]
        L.vla_mesh_csr.argtypes = [vp, vp, vp, vp]
        L.vla_mesh_csr_view.argtypes = [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]
        L.vla_assemble.argtypes = [vp, i32, dbl, dbl, i32, vp, vp, vp, vp, vp, vp, vp]
        L.vla_assemble_with_boundary.argtypes = [vp, i32, dbl, dbl, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.vla_boundary.argtypes = [vp, i32, vp, vp, vp]
        L.vla_simplex_normals.argtypes = [vp, vp, vp]
        L.vla_mesh_destroy.argtypes = [vp]
        L.vla_element_pages_static.argtypes = [i32, i32, i64, i64, vp, vp, i32, dbl, dbl, i32, vp, vp, vp, vp, vp]
        L.vla_element_pages_static_check.argtypes = [C.POINTER(i64), vp]
        L.vla_mesh_check.argtypes = [vp, vp]
        L.vla_partition_rows.argtypes = [i32, i64, vp, i32, i32, vp, C.POINTER(i64), vp]
        L.vla_mesh_create_rows.argtypes = [i32, i32, i64, i64, vp, vp, i64, vp, i32, i32, vp, C.POINTER(vp)]
        L.vla_batch_create.argtypes = [C.POINTER(BatchJob), i32, i32, vp, i32, vp, C.POINTER(vp)]
        L.vla_batch_set_job.argtypes = [vp, i32, C.POINTER(BatchJob), vp]
        L.vla_batch_run.argtypes = [vp, vp]
        L.vla_batch_info.argtypes = [vp, C.POINTER(BatchInfo)]
        L.vla_batch_check.argtypes = [vp, vp]
        L.vla_batch_destroy.argtypes = [vp]
        L.vla_batch_assemble.argtypes = [C.POINTER(BatchJob), i32, i32, vp, vp]
        L.vla_autotune.argtypes = [i32, i32, i32, i64, i64, vp, vp, i32, vp, C.POINTER(Tune)]
        L.vla_tune_get.argtypes = [i32, i32, i32, C.POINTER(Tune)]
        L.vla_tune_set.argtypes = [i32, i32, i32, C.POINTER(Tune)]
        L.vla_quad_rule.argtypes = [i32, i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl)]
        L.vla_mesh_facets.argtypes = [vp, vp, vp, vp, C.POINTER(i64), C.POINTER(i64), vp]
        L.vla_quad_points.argtypes = [vp, i32, i32, vp, vp]
        L.vla_gi.argtypes = [i64, i32, i32, vp, C.POINTER(dbl), vp, vp, vp, vp]
        L.vla_rhs.argtypes = [vp, i32, vp, vp, vp, vp]
        L.vla_energies.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.vla_avtamav.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp, vp]
        L.vla_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(vp)]
        L.vla_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(i64)]
        L.vla_server_poll.argtypes = [vp, i64, dbl, C.POINTER(Result)]
        L.vla_server_release.argtypes = [vp, i64]
        L.vla_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.vla_server_destroy.argtypes = [vp]
        for name in ("vla_amtam", "vla_astam", "vla_avtam", "vla_amdet", "vla_aminv", "vla_mesh_create",
                     "vla_mesh_info", "vla_mesh_csr", "vla_mesh_csr_view", "vla_assemble", "vla_assemble_with_boundary", "vla_boundary", "vla_simplex_normals",
                     "vla_mesh_destroy", "vla_element_pages_static", "vla_element_pages_static_check", "vla_mesh_check",
                     "vla_partition_rows", "vla_mesh_create_rows", "vla_batch_create",
                     "vla_batch_set_job", "vla_batch_run", "vla_batch_info", "vla_batch_check", "vla_batch_destroy",
                     "vla_batch_assemble", "vla_autotune", "vla_tune_get", "vla_tune_set", "vla_server_create",
                     "vla_server_submit", "vla_server_poll", "vla_server_release", "vla_server_stats",
                     "vla_server_destroy", "vla_quad_rule", "vla_quad_points", "vla_gi", "vla_rhs", "vla_energies",
                     "vla_avtamav", "vla_mesh_facets"):
            getattr(L, name).restype = i32
        _lib = L
        return L


def _check(st: int):
    if st < 0:
        buf = C.create_string_buffer(1024)
        lib().vla_last_error(buf, 1024)
        raise VlaError(st, buf.value.decode(errors="replace"))
    return st


def version() -> int:
    return lib().vla_version()


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError("page arrays must be float32 or float64")


def _req(t, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t


def _buf(t, numel, dtype, device, name):
    """A caller-supplied tensor of which the library reads or writes exactly
    ``numel`` entries: checked here, since the C entry points see only a
    pointer."""
    _req(t, dtype)
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got {t.device}")
    return t


def _same_device(first, *rest):
    for t in rest:
        if t is not None and t.device != first.device:
            raise ValueError(f"all tensors must be on {first.device}, got {t.device}")


def _nlb(dim, order):
    return dim + 1 if order == 1 else (dim + 1) * (dim + 2) // 2


def _mesh_arrays(coords, elems, faces, order):
    """Shapes of mesh arrays against the element order: the library reads
    ne x nlb element indices and nfb x dim facet indices."""
    if coords.dim() != 2 or coords.shape[1] not in (2, 3):
        raise ValueError("coords must be (nn, dim) with dim 2 or 3")
    dim = coords.shape[1]
    if order not in (1, 2):
        raise ValueError("order must be 1 or 2")
    if elems.dim() != 2 or elems.shape[1] != _nlb(dim, order):
        raise ValueError(f"elems must be (ne, {_nlb(dim, order)}) for dim {dim}, order {order}")
    if faces is not None and (faces.dim() != 2 or faces.shape[1] != dim):
        raise ValueError(f"faces must be (nfb, {dim})")
    return dim


def _page_dims(A, layout):
    # returns (N, rows, cols)
    if layout == LAYOUT_PAGE:
        N, cols, rows = A.shape
    else:
        cols, rows, N = A.shape
    return N, rows, cols


def _new_pages(N, rows, cols, layout, like):
    shape = (N, cols, rows) if layout == LAYOUT_PAGE else (cols, rows, N)
    return torch.empty(shape, dtype=like.dtype, device=like.device)


def _new_vec(N, n, layout, like):
    shape = (N, n) if layout == LAYOUT_PAGE else (n, N)
    return torch.empty(shape, dtype=like.dtype, device=like.device)


# ---------------------------------------------------------------------------
# page primitives
# ---------------------------------------------------------------------------

def amtam(A, B, out=None, layout=LAYOUT_PAGE, stream=None):
    """C_k = A_k^T B_k (amtam).  A: p x m pages, B: p x n pages -> m x n pages.  Section 2.4."""
    _req(A), _req(B)
    _same_device(A, B)
    N, p, m = _page_dims(A, layout)
    N2, p2, n = _page_dims(B, layout)
    if N2 != N or p2 != p or A.dtype != B.dtype:
        raise ValueError("amtam: page counts, row counts and dtypes must match")
    out = _new_pages(N, m, n, layout, A) if out is None else _buf(out, N * m * n, A.dtype, A.device, "out")
    _check(lib().vla_amtam(_dtype_code(A), layout, N, p, m, n, _p(A), _p(B), _p(out), _stream(stream)))
    return out


def astam(s, A, out=None, layout=LAYOUT_PAGE, stream=None):
    """C_k = s_k A_k (astam).  Sections 2.2, 2.4."""
    _req(s, A.dtype), _req(A)
    _same_device(A, s)
    N, m, n = _page_dims(A, layout)
    if s.numel() != N:
        raise ValueError("astam: one scalar per page")
    out = _new_pages(N, m, n, layout, A) if out is None else _buf(out, N * m * n, A.dtype, A.device, "out")
    _check(lib().vla_astam(_dtype_code(A), layout, N, m, n, _p(s), _p(A), _p(out), _stream(stream)))
    return out


def avtam(v, A, out=None, layout=LAYOUT_PAGE, stream=None):
    """y_k = v_k^T A_k (avtam).  v: (N, p) page layout or (p, N) SoA.  Section 2.4."""
    _req(v, A.dtype), _req(A)
    _same_device(A, v)
    N, p, n = _page_dims(A, layout)
    if v.numel() != N * p:
        raise ValueError("avtam: v must hold p values per page")
    out = _new_vec(N, n, layout, A) if out is None else _buf(out, N * n, A.dtype, A.device, "out")
    _check(lib().vla_avtam(_dtype_code(A), layout, N, p, n, _p(v), _p(A), _p(out), _stream(stream)))
    return out


def amdet(A, out=None, layout=LAYOUT_PAGE, stream=None):
    """Signed page determinants (amdet).  Sections 2.3, 3.2."""
    _req(A)
    N, n, n2 = _page_dims(A, layout)
    if n != n2:
        raise ValueError("amdet: square pages required")
    out = torch.empty(N, dtype=A.dtype, device=A.device) if out is None else _buf(out, N, A.dtype, A.device, "out")
    _check(lib().vla_amdet(_dtype_code(A), layout, N, n, _p(A), _p(out), _stream(stream)))
    return out


def aminv(A, out=None, det=None, want_det=True, count_singular=True, layout=LAYOUT_PAGE, stream=None):
    """Page inverses (aminv).  Returns (Ainv, det or None, n_singular device tensor or None).  Section 2.3."""
    _req(A)
    N, n, n2 = _page_dims(A, layout)
    if n != n2:
        raise ValueError("aminv: square pages required")
    out = torch.empty_like(A) if out is None else _buf(out, N * n * n, A.dtype, A.device, "out")
    if want_det and det is None:
        det = torch.empty(N, dtype=A.dtype, device=A.device)
    elif want_det:
        _buf(det, N, A.dtype, A.device, "det")
    ns = torch.zeros(1, dtype=torch.int64, device=A.device) if count_singular else None
    _check(lib().vla_aminv(_dtype_code(A), layout, N, n, _p(A), _p(out), _p(det) if want_det else None, _p(ns),
                           _stream(stream)))
    return out, (det if want_det else None), ns


def amt(A, out=None, layout=LAYOUT_PAGE, stream=None):
    """C_k = A_k^T (amt).  A: m x n pages -> n x m pages.  Section 2.4."""
    _req(A)
    N, m, n = _page_dims(A, layout)
    out = _new_pages(N, n, m, layout, A) if out is None else _buf(out, N * m * n, A.dtype, A.device, "out")
    _check(lib().vla_amt(_dtype_code(A), layout, N, m, n, _p(A), _p(out), _stream(stream)))
    return out


def avtav(a, b, out=None, layout=LAYOUT_PAGE, stream=None):
    """out_k = a_k^T b_k (avtav).  a, b: (N, n) page layout or (n, N) SoA.  Section 2.4."""
    _req(a), _req(b, a.dtype)
    _same_device(a, b)
    N, n = a.shape if layout == LAYOUT_PAGE else a.shape[::-1]
    if b.shape != a.shape:
        raise ValueError("avtav: a and b must have the same shape")
    out = torch.empty(N, dtype=a.dtype, device=a.device) if out is None else _buf(out, N, a.dtype, a.device, "out")
    _check(lib().vla_avtav(_dtype_code(a), layout, N, n, _p(a), _p(b), _p(out), _stream(stream)))
    return out


def amsm(A, S, out=None, layout=LAYOUT_PAGE, stream=None):
    """C_k = A_k S (amsm).  A: m x p pages; S: one p x n matrix as a (n, p)
    tensor (its columns, column-major like a page) -> m x n pages.  Section 2.4."""
    _req(A), _req(S, A.dtype)
    _same_device(A, S)
    N, m, p = _page_dims(A, layout)
    n, p2 = S.shape
    if p2 != p:
        raise ValueError("amsm: S must have p rows")
    out = _new_pages(N, m, n, layout, A) if out is None else _buf(out, N * m * n, A.dtype, A.device, "out")
    _check(lib().vla_amsm(_dtype_code(A), layout, N, m, p, n, _p(A), _p(S), _p(out), _stream(stream)))
    return out


def amsv(A, s, out=None, layout=LAYOUT_PAGE, stream=None):
    """y_k = A_k s (amsv).  A: m x n pages; s: (n,) -> (N, m) page layout or (m, N) SoA.  Section 2.4."""
    _req(A), _req(s, A.dtype)
    _same_device(A, s)
    N, m, n = _page_dims(A, layout)
    if s.numel() != n:
        raise ValueError("amsv: s must hold n values")
    out = _new_vec(N, m, layout, A) if out is None else _buf(out, N * m, A.dtype, A.device, "out")
    _check(lib().vla_amsv(_dtype_code(A), layout, N, m, n, _p(A), _p(s), _p(out), _stream(stream)))
    return out


def smamt(S, A, out=None, layout=LAYOUT_PAGE, stream=None):
    """C_k = S A_k^T (smamt).  S: one m x p matrix as a (p, m) tensor; A: n x p
    pages -> m x n pages.  Section 2.4."""
    _req(A), _req(S, A.dtype)
    _same_device(A, S)
    N, n, p = _page_dims(A, layout)
    p2, m = S.shape
    if p2 != p:
        raise ValueError("smamt: S must have p columns")
    out = _new_pages(N, m, n, layout, A) if out is None else _buf(out, N * m * n, A.dtype, A.device, "out")
    _check(lib().vla_smamt(_dtype_code(A), layout, N, m, p, n, _p(S), _p(A), _p(out), _stream(stream)))
    return out


def svamt(s, A, out=None, layout=LAYOUT_PAGE, stream=None):
    """y_k = s^T A_k^T (svamt), a 1 x m page per k.  s: (n,); A: m x n pages ->
    (N, m) page layout or (m, N) SoA.  Section 2.4."""
    _req(A), _req(s, A.dtype)
    _same_device(A, s)
    N, m, n = _page_dims(A, layout)
    if s.numel() != n:
        raise ValueError("svamt: s must hold n values")
    out = _new_vec(N, m, layout, A) if out is None else _buf(out, N * m, A.dtype, A.device, "out")
    _check(lib().vla_svamt(_dtype_code(A), layout, N, m, n, _p(s), _p(A), _p(out), _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

class Mesh:
    """A mesh resident on the device with its CSR pattern and assembly tiles
    (vla_mesh_create).  ``coords`` (nn, dim) float64 and ``elems`` (ne, nlb)
    int32 are CUDA tensors; ``faces`` (nfb, dim) int32 or None."""

    def __init__(self, coords, elems, faces=None, order=1, stream=None, rows=None):
        """``rows=(r0, r1)`` builds the sub-mesh of one row block instead
        (vla_mesh_create_rows): the elements with a node in [r0, r1) and the
        facets whose smallest node lies there, global node numbering; rows
        [r0, r1) of its CSR and values are those of the whole mesh (see
        ``block``).  Section 3.5 assembly split by rows."""
        _req(coords, torch.float64), _req(elems, torch.int32)
        if faces is not None:
            _req(faces, torch.int32)
        _same_device(coords, elems, faces)
        _mesh_arrays(coords, elems, faces, order)
        nn, dim = coords.shape
        ne = elems.shape[0]
        nfb = 0 if faces is None else faces.shape[0]
        h = C.c_void_p()
        if rows is None:
            _check(lib().vla_mesh_create(dim, order, nn, ne, _p(coords), _p(elems), nfb, _p(faces), _stream(stream),
                                         C.byref(h)))
            self.rows = (0, nn)
        else:
            r0, r1 = int(rows[0]), int(rows[1])
            _check(lib().vla_mesh_create_rows(dim, order, nn, ne, _p(coords), _p(elems), nfb, _p(faces), r0, r1,
                                              _stream(stream), C.byref(h)))
            self.rows = (r0, r1)
        self._h = h
        info = MeshInfo()
        _check(lib().vla_mesh_info(h, C.byref(info)))
        self.dim, self.order, self.nlb = info.dim, info.order, info.nlb
        self.nn, self.ne, self.nfb, self.nnz = info.nn, info.ne, info.nfb, info.nnz
        self.max_row_len, self.n_tiles, self.device_bytes = info.max_row_len, info.n_tiles, info.device_bytes
        self.tile_elems, self.n_codes = info.tile_elems, info.n_codes
        self.tile_budget, self.smem_bytes = info.tile_budget, info.smem_bytes
        self.device = coords.device

    def close(self):
        if getattr(self, "_h", None):
            lib().vla_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def csr(self, stream=None):
        rp = torch.empty(self.nn + 1, dtype=torch.int32, device=self.device)
        ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=self.device)
        _check(lib().vla_mesh_csr(self._h, _p(rp), _p(ci), _stream(stream)))
        return rp, ci[: self.nnz]

    def csr_view(self):
        """row_ptr (nn+1) and col_idx (nnz) of the mesh's own CSR pattern as
        int32 device tensors without a copy (vla_mesh_csr_view).  Read-only,
        valid until ``close()``."""
        rp, ci = C.c_void_p(), C.c_void_p()
        _check(lib().vla_mesh_csr_view(self._h, C.byref(rp), C.byref(ci)))
        return (torch.as_tensor(_DeviceArray(rp.value, self.nn + 1, self), device=self.device),
                torch.as_tensor(_DeviceArray(ci.value, self.nnz, self), device=self.device))

    def block(self, values=(), stream=None):
        """The CSR rows [r0, r1) this mesh owns (all rows for a whole mesh):
        (row_ptr (r1 - r0 + 1, starting at 0), col_idx, and the same slice of
        each tensor in ``values``, e.g. the K and M values of ``assemble``).
        col_idx and the values are views without a copy (col_idx of the
        mesh's own pattern, valid until ``close()``)."""
        r0, r1 = self.rows
        rp, ci = self.csr_view()
        if r0 == 0 and r1 == self.nn:   # the whole pattern: its bounds are known on the host
            a, b = 0, self.nnz
        else:
            a, b = int(rp[r0].item()), int(rp[r1].item())
        for v in values:
            _buf(v, self.nnz, torch.float64, self.device, "values")
        return (rp[r0:r1 + 1] - a if a else rp[r0:r1 + 1], ci[a:b]) + tuple(v[a:b] for v in values)

    def assemble(self, ca=1.0, cb=0.0, kind=COEFF_POLY, precision=PREC_MIXED, K=None, M=None, vol=None,
                 want_K=True, want_M=True, want_vol=True, pages=False, count_singular=False, stream=None,
                 boundary=False, normals=None, areas=None):
        """K and M values in CSR order (FP64), element volumes and optionally the
        element pages (ne, nlb, nlb).  Returns a dict of tensors.  Section 3.5.
        ``boundary=True`` also computes the boundary facets' normals and areas
        in the same launch (vla_assemble_with_boundary; "normals", "areas" in
        the dict, as from ``boundary``).  Sections 3.2, 3.4."""
        dev = self.device
        f64 = torch.float64
        if want_K:
            K = torch.empty(self.nnz, dtype=f64, device=dev) if K is None else _buf(K, self.nnz, f64, dev, "K")
        if want_M:
            M = torch.empty(self.nnz, dtype=f64, device=dev) if M is None else _buf(M, self.nnz, f64, dev, "M")
        if want_vol:
            vol = torch.empty(self.ne, dtype=f64, device=dev) if vol is None else _buf(vol, self.ne, f64, dev, "vol")
        Kp = torch.empty((self.ne, self.nlb, self.nlb), dtype=f64, device=dev) if pages else None
        Mp = torch.empty((self.ne, self.nlb, self.nlb), dtype=f64, device=dev) if pages else None
        ns = torch.zeros(1, dtype=torch.int64, device=dev) if count_singular else None
        if boundary:
            if normals is None:
                normals = torch.empty((max(self.nfb, 1), self.dim), dtype=f64, device=dev)[: self.nfb]
            else:
                _buf(normals, self.nfb * self.dim, f64, dev, "normals")
            if areas is None:
                areas = torch.empty(max(self.nfb, 1), dtype=f64, device=dev)[: self.nfb]
            else:
                _buf(areas, self.nfb, f64, dev, "areas")
            _check(lib().vla_assemble_with_boundary(self._h, kind, float(ca), float(cb), precision,
                                                    _p(K) if want_K else None, _p(M) if want_M else None,
                                                    _p(vol) if want_vol else None, _p(Kp), _p(Mp), _p(ns),
                                                    _p(normals), _p(areas), _stream(stream)))
        else:
            _check(lib().vla_assemble(self._h, kind, float(ca), float(cb), precision,
                                      _p(K) if want_K else None, _p(M) if want_M else None,
                                      _p(vol) if want_vol else None, _p(Kp), _p(Mp), _p(ns), _stream(stream)))
        out = {"K": K if want_K else None, "M": M if want_M else None, "vol": vol if want_vol else None}
        if boundary:
            out["normals"], out["areas"] = normals, areas
        if pages:
            out["K3D"], out["M3D"] = Kp, Mp
        if count_singular:
            out["n_singular"] = ns
        return out

    def boundary(self, precision=PREC_MIXED, normals=None, areas=None, stream=None):
        """Outward unit normals (nfb, dim) and facet measures (nfb,).  Sections 3.2, 3.4."""
        dev = self.device
        if normals is None:
            normals = torch.empty((max(self.nfb, 1), self.dim), dtype=torch.float64, device=dev)[: self.nfb]
        else:
            _buf(normals, self.nfb * self.dim, torch.float64, dev, "normals")
        if areas is None:
            areas = torch.empty(max(self.nfb, 1), dtype=torch.float64, device=dev)[: self.nfb]
        else:
            _buf(areas, self.nfb, torch.float64, dev, "areas")
        _check(lib().vla_boundary(self._h, precision, _p(normals), _p(areas), _stream(stream)))
        return normals, areas

    def facets(self, stream=None):
        """(faces (nf, dim), owner (nf, 2), neighbor (nf,), n_boundary): every
        facet once, ordered by owning element and local facet (vla_mesh_facets).  Section 3.2."""
        nf, nb = C.c_int64(), C.c_int64()
        _check(lib().vla_mesh_facets(self._h, None, None, None, C.byref(nf), C.byref(nb), _stream(stream)))
        n = nf.value
        dev = self.device
        faces = torch.empty((max(n, 1), self.dim), dtype=torch.int32, device=dev)
        owner = torch.empty((max(n, 1), 2), dtype=torch.int32, device=dev)
        nbr = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        _check(lib().vla_mesh_facets(self._h, _p(faces), _p(owner), _p(nbr), C.byref(nf), C.byref(nb),
                                     _stream(stream)))
        return faces[:n], owner[:n], nbr[:n], nb.value

    def quad_points(self, gqo, facets=False, stream=None):
        """Quadrature points (n, nip, dim) of the elements (or boundary facets)
        for the degree-gqo rule (vla_quad_points).  Section 3.4."""
        nip = quad_rule(self.dim - 1 if facets else self.dim, gqo)[1].shape[0]
        n = self.nfb if facets else self.ne
        X = torch.empty((max(n, 1), nip, self.dim), dtype=torch.float64, device=self.device)[:n]
        _check(lib().vla_quad_points(self._h, gqo, 1 if facets else 0, _p(X), _stream(stream)))
        return X

    def rhs(self, gqo, fip, b=None, b2D=None, want_b2D=True, stream=None):
        """Load vector b (nn,) and element loads b2D (ne, nlb) for f at the
        degree-gqo points (fip (ne, nip)) (vla_rhs).  Section 3.5."""
        dev, f64 = self.device, torch.float64
        nip = quad_rule(self.dim, gqo)[1].shape[0]
        _buf(fip, self.ne * nip, f64, dev, "fip")
        b = torch.empty(self.nn, dtype=f64, device=dev) if b is None else _buf(b, self.nn, f64, dev, "b")
        if want_b2D:
            b2D = (torch.empty((self.ne, self.nlb), dtype=f64, device=dev) if b2D is None
                   else _buf(b2D, self.ne * self.nlb, f64, dev, "b2D"))
        _check(lib().vla_rhs(self._h, gqo, _p(fip), _p(b), _p(b2D) if want_b2D else None, _stream(stream)))
        return b, (b2D if want_b2D else None)

    def energies(self, u, K3D=None, M3D=None, b2D=None, local=True, stream=None):
        """Local energies (ne, 3) and their sums (3,) (vla_energies).  Section 3.5."""
        dev, f64 = self.device, torch.float64
        _buf(u, self.nn, f64, dev, "u")
        for name, t, n in (("K3D", K3D, self.ne * self.nlb * self.nlb), ("M3D", M3D, self.ne * self.nlb * self.nlb),
                           ("b2D", b2D, self.ne * self.nlb)):
            if t is not None:
                _buf(t, n, f64, dev, name)
        J = torch.empty((self.ne, 3), dtype=torch.float64, device=dev) if local else None
        tot = torch.empty(3, dtype=torch.float64, device=dev)
        _check(lib().vla_energies(self._h, _p(u), _p(K3D), _p(M3D), _p(b2D), _p(J), _p(tot), _stream(stream)))
        return J, tot

    def check(self, stream=None):
        """Raises VlaError (VLA_ERR_TIMEOUT) if a bounded wait of a kernel on
        this mesh expired since the last check (vla_mesh_check)."""
        _check(lib().vla_mesh_check(self._h, _stream(stream)))

    def outputs(self, want_K=True, want_M=True, want_vol=True, pages=False):
        """Fresh output tensors for one assembly of this mesh."""
        dev, f64 = self.device, torch.float64
        return {"K": torch.empty(self.nnz, dtype=f64, device=dev) if want_K else None,
                "M": torch.empty(self.nnz, dtype=f64, device=dev) if want_M else None,
                "vol": torch.empty(self.ne, dtype=f64, device=dev) if want_vol else None,
                "K3D": torch.empty((self.ne, self.nlb, self.nlb), dtype=f64, device=dev) if pages else None,
                "M3D": torch.empty((self.ne, self.nlb, self.nlb), dtype=f64, device=dev) if pages else None}

    def simplex_normals(self, stream=None):
        """Unnormalised facet normals of every element: (ne, dim+1, dim), [k, j] = column j.  Section 3.2."""
        out = torch.empty((self.ne, self.dim + 1, self.dim), dtype=torch.float64, device=self.device)
        _check(lib().vla_simplex_normals(self._h, _p(out), _stream(stream)))
        return out


def partition_rows(elems, row_begin, row_end, stream=None):
    """Ascending ids (int32 tensor) of the elements with a node in rows
    [row_begin, row_end): the elements a GPU owning those rows assembles,
    halo included (vla_partition_rows; synchronises).  Section 3.5 assembly
    split by rows."""
    _req(elems, torch.int32)
    ne, nlb = elems.shape
    ids = torch.empty(max(ne, 1), dtype=torch.int32, device=elems.device)
    n = C.c_int64(0)
    _check(lib().vla_partition_rows(nlb, ne, _p(elems), int(row_begin), int(row_end), _p(ids), C.byref(n),
                                     _stream(stream)))
    return ids[: n.value]


def element_pages_static(coords, elems, order=1, ca=1.0, cb=0.0, kind=COEFF_POLY, precision=PREC_MIXED,
                         count_singular=False, stream=None):
    """Element pages (ne, nlb, nlb), volumes (ne,) and optionally the singular
    count from raw mesh arrays, without a mesh handle and without any device
    allocation inside the library (vla_element_pages_static; at most 262,144
    nodes; the centroid coefficient kinds).  The output tensors are allocated
    here by PyTorch; callers that cannot allocate pass the C entry point their
    own buffers.  The element indices are checked here against [0, nn) before
    the call (the library also skips and counts out-of-range elements on the
    device, see static_skipped).  Section 3.5."""
    _req(coords, torch.float64), _req(elems, torch.int32)
    _same_device(coords, elems)
    _mesh_arrays(coords, elems, None, order)
    nn, dim = coords.shape
    ne, nlb = elems.shape
    if ne > 0:
        lo, hi = int(elems.min().item()), int(elems.max().item())
        if lo < 0 or hi >= nn:
            raise VlaError(VLA_ERR_INDEX_OOB, f"element node index outside [0, {nn}) (min {lo}, max {hi})")
    dev = coords.device
    Kp = torch.empty((ne, nlb, nlb), dtype=torch.float64, device=dev)
    Mp = torch.empty((ne, nlb, nlb), dtype=torch.float64, device=dev)
    vol = torch.empty(ne, dtype=torch.float64, device=dev)
    ns = torch.zeros(1, dtype=torch.int64, device=dev) if count_singular else None
    _check(lib().vla_element_pages_static(dim, order, nn, ne, _p(coords), _p(elems), kind, float(ca), float(cb),
                                          precision, _p(Kp), _p(Mp), _p(vol), _p(ns), _stream(stream)))
    out = {"K3D": Kp, "M3D": Mp, "vol": vol}
    if count_singular:
        out["n_singular"] = ns
    return out


def static_skipped(stream=None) -> int:
    """Number of elements the last element_pages_static call on the current
    device skipped for an index outside [0, nn) (synchronises the stream;
    vla_element_pages_static_check).  No counterpart in the paper."""
    n = C.c_int64(0)
    st = lib().vla_element_pages_static_check(C.byref(n), _stream(stream))
    if st < 0 and st != VLA_ERR_INDEX_OOB:
        _check(st)
    return int(n.value)


# ---------------------------------------------------------------------------
# batches and tuning
# ---------------------------------------------------------------------------

def _job(mesh, out, kind, ca, cb):
    sizes = {"K": mesh.nnz, "M": mesh.nnz, "vol": mesh.ne, "K3D": mesh.ne * mesh.nlb * mesh.nlb,
             "M3D": mesh.ne * mesh.nlb * mesh.nlb}
    for name, n in sizes.items():
        if out.get(name) is not None:
            _buf(out[name], n, torch.float64, mesh.device, name)
    return BatchJob(mesh._h, kind, 0, float(ca), float(cb), _p(out.get("K")), _p(out.get("M")),
                    _p(out.get("vol")), _p(out.get("K3D")), _p(out.get("M3D")))


class Batch:
    """Many meshes assembled by one persistent launch (vla_batch_create).

    ``jobs`` is a list of (mesh, outputs, kind, ca, cb) where outputs is a
    dict with optional keys K, M, vol, K3D, M3D (tensors, e.g. from
    Mesh.outputs()).  With ``graph`` the launch is captured into a CUDA graph.
    ``n_singular`` (int64 tensor, one entry per job) is filled by each run."""

    def __init__(self, jobs, precision=PREC_MIXED, graph=False, count_singular=False, form=None, tune=False,
                 stream=None):
        if not jobs:
            raise ValueError("a batch needs at least one job")
        self.meshes = [j[0] for j in jobs]
        self.outs = [j[1] for j in jobs]
        arr = (BatchJob * len(jobs))(*[_job(m, o, k, a, b) for (m, o, k, a, b) in jobs])
        dev = self.meshes[0].device
        self.n_singular = torch.zeros(len(jobs), dtype=torch.int64, device=dev) if count_singular else None
        h = C.c_void_p()
        flags = (BATCH_GRAPH if graph else 0) | {None: 0, "fused": BATCH_FUSED, "split": BATCH_SPLIT}[form]
        flags |= BATCH_AUTOTUNE if tune else 0
        _check(lib().vla_batch_create(arr, len(jobs), precision, _p(self.n_singular), flags, _stream(stream),
                                      C.byref(h)))
        self._h = h
        info = BatchInfo()
        _check(lib().vla_batch_info(h, C.byref(info)))
        self.count, self.n_work, self.grid = info.count, info.n_work, info.grid
        self.ctas_per_sm, self.smem_bytes = info.ctas_per_sm, info.smem_bytes
        self.elements, self.tile_elems, self.graph = info.elements, info.tile_elems, bool(info.graph)
        self.split = bool(info.split)

    def set_job(self, index, out, kind=COEFF_POLY, ca=1.0, cb=0.0, stream=None):
        job = _job(self.meshes[index], out, kind, ca, cb)
        _check(lib().vla_batch_set_job(self._h, index, C.byref(job), _stream(stream)))
        self.outs[index] = out

    def run(self, stream=None):
        _check(lib().vla_batch_run(self._h, _stream(stream)))
        return self.outs

    def check(self, stream=None):
        _check(lib().vla_batch_check(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().vla_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_assemble(jobs, precision=PREC_MIXED, n_singular=None, stream=None):
    """One-shot batch (vla_batch_assemble): jobs as for Batch; stream-ordered."""
    arr = (BatchJob * len(jobs))(*[_job(m, o, k, a, b) for (m, o, k, a, b) in jobs])
    if n_singular is not None:
        _buf(n_singular, len(jobs), torch.int64, jobs[0][0].device, "n_singular")
    _check(lib().vla_batch_assemble(arr, len(jobs), precision, _p(n_singular), _stream(stream)))
    return [j[1] for j in jobs]


def autotune(coords, elems, order=1, precision=PREC_MIXED, reps=5, stream=None):
    """Times candidate tile budgets and CTA residencies on this sample mesh,
    stores the fastest for its element type and precision, and returns
    (tile_budget, ctas_per_sm, microseconds)."""
    _req(coords, torch.float64), _req(elems, torch.int32)
    _same_device(coords, elems)
    _mesh_arrays(coords, elems, None, order)
    nn, dim = coords.shape
    t = Tune()
    _check(lib().vla_autotune(dim, order, precision, nn, elems.shape[0], _p(coords), _p(elems), reps,
                              _stream(stream), C.byref(t)))
    return t.tile_budget, t.ctas_per_sm, t.us


def tune_get(dim, order, precision=PREC_MIXED):
    t = Tune()
    _check(lib().vla_tune_get(dim, order, precision, C.byref(t)))
    return t.tile_budget, t.ctas_per_sm


def tune_set(dim, order, precision=PREC_MIXED, tile_budget=0, ctas_per_sm=0):
    t = Tune(tile_budget, ctas_per_sm, 0.0)
    _check(lib().vla_tune_set(dim, order, precision, C.byref(t)))


# ---------------------------------------------------------------------------
# assembly server
# ---------------------------------------------------------------------------

class _DevView:
    """A device array given by pointer, seen by torch through the CUDA array interface."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2}


def _view(ptr, n, typestr, device):
    if n == 0:
        return torch.empty(0, dtype=torch.float64 if typestr == "<f8" else torch.int32, device=device)
    return torch.as_tensor(_DevView(ptr, n, typestr), device=device)


class Server:
    """Continuous-batching assembly server (vla_server_*).

    submit() takes host (numpy) or device (torch) mesh arrays, coords (nn, dim)
    float64 and elems (ne, nlb) int32, and returns a ticket; poll() returns
    None while the request runs, else its result record; result() copies K,
    M, vol (and the CSR pattern) into fresh tensors; release() frees the
    server's copies."""

    def __init__(self, budget_bytes, precision=PREC_MIXED, ingest_workers=4, max_batch=0, max_inflight=0):
        cfg = ServerConfig(int(budget_bytes), precision, ingest_workers, max_batch, max_inflight)
        h = C.c_void_p()
        _check(lib().vla_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = {}
        self.device = torch.device("cuda", torch.cuda.current_device())

    @staticmethod
    def _ptr(a, dtype):
        if isinstance(a, torch.Tensor):   # device tensor, or host tensor (pinned for full copy speed)
            if a.is_cuda:
                _req(a, dtype)
            elif not a.is_contiguous() or a.dtype != dtype:
                raise TypeError(f"expected a contiguous {dtype} tensor")
            return a, a.data_ptr()
        import numpy as np
        a = np.ascontiguousarray(a, dtype={torch.float64: np.float64, torch.int32: np.int32}[dtype])
        return a, a.ctypes.data

    def submit(self, coords, elems, order=1, key=-1, keep_resident=True, kind=COEFF_POLY, ca=1.0, cb=0.0,
               faces=None):
        c, cp = self._ptr(coords, torch.float64)
        e, ep = self._ptr(elems, torch.int32)
        f, fp = (None, None) if faces is None else self._ptr(faces, torch.int32)
        if len(c.shape) != 2 or c.shape[1] not in (2, 3):
            raise ValueError("coords must be (nn, dim) with dim 2 or 3")
        nn, dim = c.shape
        if order not in (1, 2) or len(e.shape) != 2 or e.shape[1] != _nlb(dim, order):
            nlb = _nlb(dim, order) if order in (1, 2) else "nlb"
            raise ValueError(f"elems must be (ne, {nlb}) for order {order}")
        if f is not None and (len(f.shape) != 2 or f.shape[1] != dim):
            raise ValueError(f"faces must be (nfb, {dim})")
        ne = e.shape[0]
        nfb = 0 if f is None else f.shape[0]
        r = Request(int(key), dim, order, nn, ne, nfb, cp, ep, fp, 1 if keep_resident else 0, kind,
                    float(ca), float(cb))
        t = C.c_int64()
        _check(lib().vla_server_submit(self._h, C.byref(r), C.byref(t)))
        self._keep[t.value] = (c, e, f)
        return t.value

    def poll(self, ticket, timeout=0.0):
        res = Result()
        st = lib().vla_server_poll(self._h, int(ticket), float(timeout), C.byref(res))
        if st == PENDING:
            return None
        self._keep.pop(ticket, None)
        if st < 0 and res.status == 0:
            _check(st)
        return res

    def result(self, ticket, res=None, pattern=False):
        """K, M, vol (and row_ptr, col_idx) of a finished request as new tensors."""
        if res is None:
            res = self.poll(ticket)
            if res is None:
                raise RuntimeError("request not finished")
        if res.status < 0:
            raise VlaError(res.status, f"request {ticket} failed")
        dev = self.device
        out = {"K": _view(res.K_vals, res.nnz, "<f8", dev).clone(),
               "M": _view(res.M_vals, res.nnz, "<f8", dev).clone(),
               "vol": _view(res.vol, res.ne, "<f8", dev).clone()}
        if pattern:
            out["row_ptr"] = _view(res.row_ptr, res.nn + 1, "<i4", dev).clone()
            out["col_idx"] = _view(res.col_idx, res.nnz, "<i4", dev).clone()
        return out

    def release(self, ticket):
        _check(lib().vla_server_release(self._h, int(ticket)))
        self._keep.pop(ticket, None)

    def stats(self):
        st = ServerStats()
        _check(lib().vla_server_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().vla_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# quadrature and integrals
# ---------------------------------------------------------------------------

def quad_rule(sdim, gqo):
    """(ip (nip, sdim+1), w (nip,)) of the degree-gqo rule on an sdim-simplex.  Section 3.4."""
    import numpy as np
    n = C.c_int32()
    ip = (C.c_double * 32)()
    w = (C.c_double * 8)()
    _check(lib().vla_quad_rule(sdim, gqo, C.byref(n), ip, w))
    k = n.value
    return (np.array(ip[: k * (sdim + 1)]).reshape(k, sdim + 1), np.array(w[:k]))


def gi(fip, w, sizes, normals=None, stream=None):
    """GI of Section 3.4 on the device: fip (n, nip, d), w (nip,) host weights,
    sizes (n,), normals (n, d) or None.  Returns a (d,) tensor, or a (1,)
    tensor holding the flux when normals are given."""
    _req(fip, torch.float64)
    n, nip, d = fip.shape
    _buf(sizes, n, torch.float64, fip.device, "sizes")
    if normals is not None:
        _buf(normals, n * d, torch.float64, fip.device, "normals")
    if len(w) != nip:
        raise ValueError(f"gi: {nip} points in fip but {len(w)} weights")
    out = torch.empty(d if normals is None else 1, dtype=torch.float64, device=fip.device)
    wa = (C.c_double * nip)(*[float(x) for x in w])
    _check(lib().vla_gi(n, nip, d, _p(fip), wa, _p(sizes), _p(normals), _p(out), _stream(stream)))
    return out


def avtamav(v, A, w, out=None, layout=LAYOUT_PAGE, stream=None):
    """out_k = v_k^T A_k w_k.  Page layout: v, w (N, n); A (N, n, n) (N, cols, rows).  Section 2.4."""
    _req(v), _req(A, v.dtype), _req(w, v.dtype)
    _same_device(v, A, w)
    if layout == LAYOUT_PAGE:
        N, n = v.shape
    else:
        n, N = v.shape
    if w.shape != v.shape or A.numel() != N * n * n:
        raise ValueError("avtamav: v and w must have the same shape and A n x n pages, one per vector")
    out = torch.empty(N, dtype=v.dtype, device=v.device) if out is None else _buf(out, N, v.dtype, v.device, "out")
    _check(lib().vla_avtamav(_dtype_code(v), layout, N, n, _p(v), _p(A), _p(w), _p(out), _stream(stream)))
    return out
