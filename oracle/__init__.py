"""CPU FP64 oracle for the page-wise linear algebra and FE assembly path.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The library package
never imports this module, and this module never imports the library.

The arithmetic lives in ``vla_oracle.c`` (plain C, explicit loops, FP64);
this file only compiles it with gcc (once, next to the source) and marshals
numpy arrays through ctypes.  Each wrapper names the paper passage its C
function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vla_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = C.c_int64


def build(force: bool = False) -> str:
    """Compile ``vla_oracle.c`` into ``liboracle.so`` (gcc, -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-pthread", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.orc_amtam.argtypes = [_i64, C.c_int, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_astam.argtypes = [_i64, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_avtam.argtypes = [_i64, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_amdet.argtypes = [_i64, C.c_int, _d, _d]
        lib.orc_amt.argtypes = [_i64, C.c_int, C.c_int, _d, _d]
        lib.orc_avtav.argtypes = [_i64, C.c_int, _d, _d, _d]
        lib.orc_amsm.argtypes = [_i64, C.c_int, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_amsv.argtypes = [_i64, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_smamt.argtypes = [_i64, C.c_int, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_svamt.argtypes = [_i64, C.c_int, C.c_int, _d, _d, _d]
        lib.orc_aminv.argtypes = [_i64, C.c_int, _d, _d, vp]
        lib.orc_aminv.restype = _i64
        lib.orc_vectors.argtypes = [C.c_int, _i64, C.c_int, _i, _d, _d]
        lib.orc_volumes.argtypes = [C.c_int, _i64, C.c_int, _i, _d, _d, vp]
        lib.orc_simplex_normals.argtypes = [C.c_int, _i64, C.c_int, _i, _d, _d]
        lib.orc_element_pages.argtypes = [C.c_int, C.c_int, _i64, C.c_int, _i, _d, C.c_int, C.c_double, C.c_double,
                                          _d, _d, _d, _d]
        lib.orc_csr_pattern.argtypes = [_i64, _i64, C.c_int, _i, vp, vp]
        lib.orc_csr_pattern.restype = _i64
        lib.orc_csr_scatter.argtypes = [_i64, C.c_int, _i, _d, _i, _i, _d]
        lib.orc_csr_scatter.restype = C.c_int
        lib.orc_assemble.argtypes = [C.c_int, C.c_int, _i64, _i64, C.c_int, _i, _d, C.c_int, C.c_double, C.c_double,
                                     _i, _i, _d, _d, _d, vp, vp]
        lib.orc_assemble.restype = C.c_int
        lib.orc_assemble_threads.argtypes = [C.c_int, C.c_int, _i64, _i64, C.c_int, _i, _d, C.c_int, C.c_double,
                                             C.c_double, _i, _i, _d, _d, _d, C.c_int]
        lib.orc_assemble_threads.restype = C.c_int
        lib.orc_boundary.argtypes = [C.c_int, _i64, _i64, C.c_int, _i, _d, _i64, _i, _d, _d]
        lib.orc_boundary.restype = _i64
        lib.orc_count_facets.argtypes = [C.c_int, _i64, C.c_int, _i, C.POINTER(_i64), C.POINTER(_i64)]
        lib.orc_count_facets.restype = C.c_int
        lib.orc_quad_rule.argtypes = [C.c_int, C.c_int, _d, _d]
        lib.orc_quad_rule.restype = C.c_int
        lib.orc_quad_points.argtypes = [C.c_int, C.c_int, _i64, C.c_int, _i, _d, C.c_int, _d, _d]
        lib.orc_gi.argtypes = [_i64, C.c_int, C.c_int, _d, _d, _d, vp, _d]
        lib.orc_rhs.argtypes = [C.c_int, C.c_int, _i64, _i64, C.c_int, _i, _d, C.c_int, _d, _d, _d, _d, _d]
        lib.orc_energies.argtypes = [_i64, C.c_int, _i, _d, _d, _d, _d, _d]
        lib.orc_avtamav.argtypes = [_i64, C.c_int, _d, _d, _d, _d]
        lib.orc_facets.argtypes = [C.c_int, _i64, C.c_int, _i, vp, vp, vp, C.POINTER(_i64)]
        lib.orc_facets.restype = _i64
        _lib = lib
        return lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


# --------------------------------------------------------------------------
# page primitives (Section 2.4).  Page arrays are numpy (N, cols, rows) C
# arrays, i.e. column-major pages with the page index slowest.
# --------------------------------------------------------------------------

def amtam(A, B):
    """C_k = A_k^T B_k.  A: (N, m, p) = N pages p x m; B: (N, n, p); C: (N, n, m).  Follows amtam of Section
    2.4, read as A^T B."""
    A, B = _f64(A), _f64(B)
    N, m, p = A.shape
    n = B.shape[1]
    Cm = np.empty((N, n, m))
    _load().orc_amtam(N, p, m, n, A, B, Cm)
    return Cm


def astam(s, A):
    """C_k = s_k A_k.  Follows astam of Sections 2.2 and 2.4."""
    s, A = _f64(s), _f64(A)
    N, n, m = A.shape
    out = np.empty_like(A)
    _load().orc_astam(N, m, n, s, A, out)
    return out


def avtam(v, A):
    """y_k = v_k^T A_k.  v: (N, p); A: (N, n, p) = pages p x n; y: (N, n).  Follows avtam of Section 2.4."""
    v, A = _f64(v), _f64(A)
    N, n, p = A.shape
    y = np.empty((N, n))
    _load().orc_avtam(N, p, n, v, A, y)
    return y


def amt(A):
    """C_k = A_k^T (Section 2.4 amt).  A: (N, n, m) = N pages m x n; C: (N, m, n)."""
    A = _f64(A)
    N, n, m = A.shape
    out = np.empty((N, m, n))
    _load().orc_amt(N, m, n, A, out)
    return out


def avtav(a, b):
    """out_k = a_k^T b_k (Section 2.4 avtav).  a, b: (N, n)."""
    a, b = _f64(a), _f64(b)
    N, n = a.shape
    out = np.empty(max(N, 1))
    _load().orc_avtav(N, n, a, b, out)
    return out[:N]


def amsm(A, S):
    """C_k = A_k S (Section 2.4 amsm).  A: (N, p, m) = pages m x p; S: (n, p) =
    the p x n matrix; C: (N, n, m)."""
    A, S = _f64(A), _f64(S)
    N, p, m = A.shape
    n = S.shape[0]
    out = np.empty((N, n, m))
    _load().orc_amsm(N, m, p, n, A, S, out)
    return out


def amsv(A, s):
    """y_k = A_k s (Section 2.4 amsv).  A: (N, n, m) = pages m x n; s: (n,); y: (N, m)."""
    A, s = _f64(A), _f64(s)
    N, n, m = A.shape
    out = np.empty((N, m))
    _load().orc_amsv(N, m, n, A, s, out)
    return out


def smamt(S, A):
    """C_k = S A_k^T (Section 2.4 smamt).  S: (p, m) = the m x p matrix; A: (N, p, n)
    = pages n x p; C: (N, n, m)."""
    S, A = _f64(S), _f64(A)
    p, m = S.shape
    N, _, n = A.shape
    out = np.empty((N, n, m))
    _load().orc_smamt(N, m, p, n, S, A, out)
    return out


def svamt(s, A):
    """y_k = s^T A_k^T (Section 2.4 svamt), a 1 x m page.  s: (n,); A: (N, n, m) =
    pages m x n; y: (N, m)."""
    s, A = _f64(s), _f64(A)
    N, n, m = A.shape
    out = np.empty((N, m))
    _load().orc_svamt(N, m, n, s, A, out)
    return out


def amdet(A):
    """Signed page determinants (N,) of (N, n, n) pages.  Follows amdet of Sections 2.3 and 3.2."""
    A = _f64(A)
    N, n, _ = A.shape
    out = np.empty(N)
    _load().orc_amdet(N, n, A, out)
    return out


def aminv(A):
    """Returns (Ainv, det, n_singular).  Follows aminv of Section 2.3."""
    A = _f64(A)
    N, n, _ = A.shape
    inv = np.empty_like(A)
    det = np.empty(N)
    ns = _load().orc_aminv(N, n, A, inv, det.ctypes.data_as(C.c_void_p))
    return inv, det, int(ns)


# --------------------------------------------------------------------------
# geometry and FE assembly (Sections 3.1, 3.2, 3.5)
# --------------------------------------------------------------------------

def vectors(dim, elems, coords):
    """vectors3D pages: (ne, dim, dim) with [k, j, :] = x_{e_k[j]} - x_{e_k[dim]}.  Follows vectors3D of
    Sections 3.1 and 3.2."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    V = np.empty((ne, dim, dim))
    _load().orc_vectors(dim, ne, nlb, elems, coords, V)
    return V


def volumes(dim, elems, coords):
    """Returns (vol = |det|/dim!, signed det).  Follows the volume script of Section 3.2."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    vol, det = np.empty(ne), np.empty(ne)
    _load().orc_volumes(dim, ne, nlb, elems, coords, vol, det.ctypes.data_as(C.c_void_p))
    return vol, det


def simplex_normals(dim, elems, coords):
    """Unnormalised facet normals (V^{-T} normalsRef): (ne, dim+1, dim); [k, j] is column j.  Follows
    normals3D of Section 3.2, with the normal transform of Section 2.3."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    out = np.empty((ne, dim + 1, dim))
    _load().orc_simplex_normals(dim, ne, nlb, elems, coords, out)
    return out


def element_pages(dim, order, elems, coords, ca=1.0, cb=0.0, ckind=0):
    """Returns (K3D, M3D, vol, coef); pages as (ne, nlb, nlb) with [k, q, p] = P_k(p, q).
    Coefficient at the element's vertex centroid: ckind 0: a + b|x|^2; 1: a exp(b sum x).
    Follows the stiffness and mass listings of Section 3.5."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    K = np.empty((ne, nlb, nlb))
    M = np.empty((ne, nlb, nlb))
    vol, coef = np.empty(ne), np.empty(ne)
    _load().orc_element_pages(dim, order, ne, nlb, elems, coords, ckind, ca, cb, K, M, vol, coef)
    return K, M, vol, coef


def csr_pattern(nn, elems):
    """Sorted-unique (row, col) pattern of all element pairs: (row_ptr, col_idx).  Follows the sparse assembly
    of Section 3.5."""
    elems = _i32(elems)
    ne, nlb = elems.shape
    lib = _load()
    nnz = lib.orc_csr_pattern(nn, ne, nlb, elems, None, None)
    if nnz < 0:
        raise MemoryError("oracle pattern")
    rp = np.zeros(nn + 1, dtype=np.int32)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.orc_csr_pattern(nn, ne, nlb, elems, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p))
    return rp, ci[:nnz]


def csr_scatter(elems, pages, row_ptr, col_idx):
    """CSR values of element pages (ne, nlb, nlb) summed into the pattern (row_ptr,
    col_idx).  Follows the sparse assembly of Section 3.5."""
    elems = _i32(elems)
    ne, nlb = elems.shape
    vals = np.zeros(len(col_idx))
    rc = _load().orc_csr_scatter(ne, nlb, elems, _f64(pages), _i32(row_ptr), _i32(col_idx) if len(col_idx) else
                                 np.zeros(1, np.int32), vals if len(vals) else np.zeros(1))
    if rc != 0:
        raise ValueError("pair missing from pattern")
    return vals


def assemble(dim, order, nn, elems, coords, ca=1.0, cb=0.0, pattern=None, want_pages=False, ckind=0):
    """K and M in CSR (values FP64) plus volumes.  Returns a dict with
    row_ptr, col_idx, K, M, vol and (optionally) K3D, M3D.  Follows Section 3.5."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    rp, ci = pattern if pattern is not None else csr_pattern(nn, elems)
    nnz = len(ci)
    Kv, Mv, vol = np.zeros(max(nnz, 1)), np.zeros(max(nnz, 1)), np.zeros(max(ne, 1))
    K3D = M3D = None
    vp = None
    if want_pages:
        K3D = np.empty((ne, nlb, nlb))
        M3D = np.empty((ne, nlb, nlb))
    lib = _load()
    rc = lib.orc_assemble(dim, order, nn, ne, nlb, elems, coords, ckind, ca, cb, _i32(rp),
                          _i32(ci) if nnz else np.zeros(1, np.int32), Kv, Mv, vol,
                          K3D.ctypes.data_as(C.c_void_p) if want_pages else vp,
                          M3D.ctypes.data_as(C.c_void_p) if want_pages else vp)
    if rc != 0:
        raise ValueError("oracle assembly failed")
    out = {"row_ptr": rp, "col_idx": ci, "K": Kv[:nnz], "M": Mv[:nnz], "vol": vol[:ne]}
    if want_pages:
        out["K3D"], out["M3D"] = K3D, M3D
    return out


def assemble_threads(dim, order, nn, elems, coords, ca=1.0, cb=0.0, pattern=None, ckind=0, nthreads=1):
    """The same K, M and volumes as ``assemble`` (bit for bit) on ``nthreads``
    host threads: a timing entry for the CPU baseline, which runs the pinned
    element-page and scatter steps over element ranges and row blocks."""
    elems, coords = _i32(elems), _f64(coords)
    ne, nlb = elems.shape
    rp, ci = pattern if pattern is not None else csr_pattern(nn, elems)
    nnz = len(ci)
    Kv, Mv, vol = np.zeros(max(nnz, 1)), np.zeros(max(nnz, 1)), np.zeros(max(ne, 1))
    rc = _load().orc_assemble_threads(dim, order, nn, ne, nlb, elems, coords, ckind, ca, cb, _i32(rp),
                                      _i32(ci) if nnz else np.zeros(1, np.int32), Kv, Mv, vol, int(nthreads))
    if rc != 0:
        raise ValueError("oracle assembly failed")
    return {"row_ptr": rp, "col_idx": ci, "K": Kv[:nnz], "M": Mv[:nnz], "vol": vol[:ne]}


def boundary(dim, nn, elems, coords, faces):
    """Outward unit normals (nfb, dim) and facet measures (nfb,).  Returns
    (normals, areas, n_missing_owner).  Follows the boundary normals and areas of Sections 3.2 and 3.4."""
    elems, coords, faces = _i32(elems), _f64(coords), _i32(faces)
    ne, nlb = elems.shape
    nfb = faces.shape[0]
    nrm = np.empty((max(nfb, 1), dim))
    ar = np.empty(max(nfb, 1))
    miss = _load().orc_boundary(dim, nn, ne, nlb, elems, coords, nfb, faces if nfb else np.zeros((1, dim), np.int32),
                                nrm, ar)
    return nrm[:nfb], ar[:nfb], int(miss)


def count_facets(dim, elems):
    """(number of distinct facets, number of boundary facets).  Follows the face counts of Section 3.2."""
    elems = _i32(elems)
    ne, nlb = elems.shape
    a, b = _i64(0), _i64(0)
    if _load().orc_count_facets(dim, ne, nlb, elems, C.byref(a), C.byref(b)) != 0:
        raise MemoryError("oracle facets")
    return int(a.value), int(b.value)


def to_dense(nn, row_ptr, col_idx, vals):
    """Dense nn x nn matrix of a CSR triple (test helper)."""
    D = np.zeros((nn, nn))
    for r in range(nn):
        for q in range(row_ptr[r], row_ptr[r + 1]):
            D[r, col_idx[q]] += vals[q]
    return D


# --------------------------------------------------------------------------
# quadrature, integrals, load vector, energies (Sections 3.4, 3.5)
# --------------------------------------------------------------------------

def quad_rule(sdim, gqo):
    """(ip (nip, sdim+1) barycentric points, w (nip,) weights summing to 1).  Follows Gauss_points of Section 3.4."""
    ip = np.zeros((8, sdim + 1))
    w = np.zeros(8)
    nip = _load().orc_quad_rule(sdim, gqo, ip, w)
    if nip < 0:
        raise ValueError(f"no rule for simplex dimension {sdim}, order {gqo}")
    return ip[:nip].copy(), w[:nip].copy()


def quad_points(dim, cells, coords, ip):
    """X (n, nip, dim): quadrature points of the simplices cells (n, >= nvert).  Follows X_ip of Section 3.4."""
    cells, coords, ip = _i32(cells), _f64(coords), _f64(ip)
    n, stride = cells.shape
    nip, nvert = ip.shape
    X = np.empty((max(n, 1), nip, dim))
    _load().orc_quad_points(dim, nvert, n, stride, cells, coords, nip, ip, X)
    return X[:n]


def gi(fip, w, sizes, normals=None):
    """GI of Section 3.4: fip (n, nip, d).  Returns the d component integrals, or
    the flux through the simplices (a scalar) when normals (n, d) are given."""
    fip, w, sizes = _f64(fip), _f64(w), _f64(sizes)
    n, nip, d = fip.shape
    out = np.zeros(max(d, 1))
    nr = None if normals is None else _f64(normals)
    _load().orc_gi(n, nip, d, fip, w, sizes, None if nr is None else nr.ctypes.data_as(C.c_void_p), out)
    return out[0] if normals is not None else out


def rhs(dim, order, nn, elems, coords, ip, w, fip):
    """Load vector b (nn,) and element contributions b2D (ne, nlb) for f given at
    the rule's points (fip (ne, nip)).  Follows rhs_vectorP1 of Section 3.5."""
    elems, coords, ip, w, fip = _i32(elems), _f64(coords), _f64(ip), _f64(w), _f64(fip)
    ne, nlb = elems.shape
    b = np.empty(nn)
    b2D = np.empty((max(ne, 1), nlb))
    _load().orc_rhs(dim, order, nn, ne, nlb, elems, coords, ip.shape[0], ip, w, fip, b, b2D)
    return b, b2D[:ne]


def energies(elems, u, K3D, M3D, b2D):
    """Local energies (ne, 3): u_k^T K_k u_k / 2, u_k^T M_k u_k / 2, -b2D_k^T u_k.  Follows the local energies
    of Section 3.5."""
    elems, u, K3D, M3D, b2D = _i32(elems), _f64(u), _f64(K3D), _f64(M3D), _f64(b2D)
    ne, nlb = elems.shape
    J = np.empty((max(ne, 1), 3))
    _load().orc_energies(ne, nlb, elems, u, K3D, M3D, b2D, J)
    return J[:ne]


def avtamav(v, A, w):
    """out_k = v_k^T A_k w_k; v, w (N, n); A (N, n, n) pages (N, cols, rows).  Follows avtamav of Section 2.4."""
    v, A, w = _f64(v), _f64(A), _f64(w)
    N, n = v.shape
    out = np.empty(max(N, 1))
    _load().orc_avtamav(N, n, v, A, w, out)
    return out[:N]


def facets(dim, elems):
    """(faces (nf, dim), owner (nf, 2) = (element, local facet), neighbor (nf,),
    n_boundary): every distinct facet once, ordered by first element and local
    facet index.  Follows the normals of all faces, Section 3.2."""
    elems = _i32(elems)
    ne, nlb = elems.shape
    L = _load()
    nb = _i64(0)
    nf = L.orc_facets(dim, ne, nlb, elems, None, None, None, C.byref(nb))
    if nf < 0:
        raise MemoryError("oracle facets")
    faces = np.empty((max(nf, 1), dim), np.int32)
    owner = np.empty((max(nf, 1), 2), np.int32)
    nbr = np.empty(max(nf, 1), np.int32)
    L.orc_facets(dim, ne, nlb, elems, faces.ctypes.data_as(C.c_void_p), owner.ctypes.data_as(C.c_void_p),
                 nbr.ctypes.data_as(C.c_void_p), C.byref(nb))
    return faces[:nf], owner[:nf], nbr[:nf], int(nb.value)
