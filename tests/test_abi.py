"""CPU checks of the C ABI boundary: the shared library builds for sm_103a,
loads, and exports every entry point include/vla.h declares.  No kernel runs."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "vla.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vla_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2404_16039_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    syms = _declared_symbols()
    for s in ("vla_amtam", "vla_astam", "vla_avtam", "vla_amdet", "vla_aminv", "vla_mesh_create",
              "vla_assemble", "vla_boundary", "vla_simplex_normals", "vla_mesh_destroy", "vla_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in _declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    lib.vla_version.restype = ctypes.c_int32
    assert lib.vla_version() >= 100


def test_argument_validation_without_gpu(libpath):
    # argument checks run before any CUDA call and report through vla_last_error
    lib = ctypes.CDLL(libpath)
    lib.vla_amdet.restype = ctypes.c_int32
    lib.vla_amdet.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.vla_amdet(7, 0, 10, 3, None, None, None) == -1          # bad dtype
    assert lib.vla_amdet(1, 0, 10, 4, None, None, None) == -1          # n = 4 unsupported
    assert lib.vla_amdet(1, 0, 10, 3, None, None, None) == -1          # null arrays
    assert lib.vla_amdet(1, 0, 0, 3, None, None, None) == 0            # N = 0 is a no-op
    buf = ctypes.create_string_buffer(256)
    lib.vla_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.vla_last_error.restype = ctypes.c_size_t
    lib.vla_amdet(1, 0, 10, 4, None, None, None)
    lib.vla_last_error(buf, 256)
    assert b"n must be 2 or 3" in buf.value
    lib.vla_mesh_create.restype = ctypes.c_int32
    h = ctypes.c_void_p()
    lib.vla_mesh_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]
    assert lib.vla_mesh_create(4, 1, 10, 10, None, None, 0, None, None, ctypes.byref(h)) == -1
    assert lib.vla_mesh_create(3, 3, 10, 10, None, None, 0, None, None, ctypes.byref(h)) == -1
    assert lib.vla_mesh_create(3, 1, 10, 1 << 27, None, None, 0, None, None, ctypes.byref(h)) == -8


def test_page_function_argument_validation_without_gpu(libpath):
    # the Section 2.4 page functions beyond the core: shape, dtype and pointer
    # checks run before any CUDA call; zero pages are a no-op
    lib = ctypes.CDLL(libpath)
    i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.vla_amt.argtypes = [i32, i32, i64, i32, i32, vp, vp, vp]
    lib.vla_avtav.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp]
    for name in ("vla_amsm", "vla_smamt"):
        getattr(lib, name).argtypes = [i32, i32, i64, i32, i32, i32, vp, vp, vp, vp]
    for name in ("vla_amsv", "vla_svamt"):
        getattr(lib, name).argtypes = [i32, i32, i64, i32, i32, vp, vp, vp, vp]
    fake = 16   # never dereferenced: every call below fails its checks or has N = 0
    assert lib.vla_amt(1, 0, 10, 4, 3, fake, fake, None) == -1           # m = 4 unsupported
    assert lib.vla_amt(1, 2, 10, 3, 3, fake, fake, None) == -1           # unknown layout
    assert lib.vla_avtav(3, 0, 10, 3, fake, fake, fake, None) == -1      # unknown dtype
    assert lib.vla_avtav(1, 0, 10, 3, None, fake, fake, None) == -1      # null array
    assert lib.vla_amsm(1, 0, 10, 3, 17, 2, fake, fake, fake, None) == -1  # p > 16
    assert lib.vla_amsm(1, 0, 10, 0, 4, 2, fake, fake, fake, None) == -1   # m < 1
    assert lib.vla_smamt(0, 0, 10, 3, 4, 3, fake, None, fake, None) == -1  # null pages
    assert lib.vla_amsv(1, 0, -1, 3, 4, fake, fake, fake, None) == -1     # negative page count
    assert lib.vla_svamt(1, 1, 0, 3, 4, None, None, None, None) == 0      # N = 0: nothing to do
    assert lib.vla_amt(0, 0, 0, 2, 3, None, None, None) == 0


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_2404_16039_gb300 as vla
    monkeypatch.setattr(vla, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(vla, "_lib", None)
    with pytest.raises(ImportError):
        vla.lib()


def test_remaining_entry_points_validate_without_gpu(libpath):
    # every other entry point: arguments rejected before any CUDA call (null
    # handles, unknown shapes, kinds, precisions, flags, limits), destroy of
    # NULL is a no-op, and the quadrature rules are pure host code
    lib = ctypes.CDLL(libpath)
    i32, i64, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    fake = 16   # never dereferenced
    INVALID, BUDGET, UNSUPPORTED = -1, -6, -8

    lib.vla_quad_rule.argtypes = [i32, i32, ctypes.POINTER(i32), vp, vp]
    nip = i32()
    ip = (f64 * 32)()
    w = (f64 * 8)()
    assert lib.vla_quad_rule(3, 3, ctypes.byref(nip), ip, w) == 0
    assert nip.value == 5 and abs(sum(w[: nip.value]) - 1.0) < 1e-15
    assert lib.vla_quad_rule(2, 2, ctypes.byref(nip), ip, w) == 0 and nip.value == 3
    assert lib.vla_quad_rule(3, 4, ctypes.byref(nip), ip, w) == UNSUPPORTED
    assert lib.vla_quad_rule(0, 1, ctypes.byref(nip), ip, w) == UNSUPPORTED

    lib.vla_gi.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp]
    assert lib.vla_gi(10, 9, 1, fake, w, fake, None, fake, None) == INVALID      # more than 8 points
    assert lib.vla_gi(10, 4, 5, fake, w, fake, None, fake, None) == INVALID      # more than 4 components
    assert lib.vla_gi(-1, 4, 1, fake, w, fake, None, fake, None) == INVALID
    assert lib.vla_gi(10, 4, 1, fake, None, fake, None, fake, None) == INVALID   # no weights

    lib.vla_avtamav.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp, vp]
    assert lib.vla_avtamav(1, 0, 10, 17, fake, fake, fake, fake, None) == INVALID
    assert lib.vla_avtamav(3, 0, 10, 3, fake, fake, fake, fake, None) == INVALID
    assert lib.vla_avtamav(1, 0, 0, 3, None, None, None, None, None) == 0

    lib.vla_element_pages_static.argtypes = [i32, i32, i64, i64, vp, vp, i32, f64, f64, i32, vp, vp, vp, vp, vp]
    assert lib.vla_element_pages_static(4, 1, 10, 10, fake, fake, 0, 1.0, 0.0, 1, None, None, None, None, None) == INVALID
    assert lib.vla_element_pages_static(3, 3, 10, 10, fake, fake, 0, 1.0, 0.0, 1, None, None, None, None, None) == INVALID
    assert lib.vla_element_pages_static(3, 1, 1 << 20, 10, fake, fake, 0, 1.0, 0.0, 1,
                                        None, None, None, None, None) == BUDGET

    lib.vla_partition_rows.argtypes = [i32, i64, vp, i32, i32, vp, ctypes.POINTER(i64), vp]
    n = i64(-1)
    assert lib.vla_partition_rows(4, 10, fake, 0, 5, None, None, None) == INVALID          # no count output
    assert lib.vla_partition_rows(11, 10, fake, 0, 5, None, ctypes.byref(n), None) == INVALID
    assert lib.vla_partition_rows(4, 10, fake, 5, 2, None, ctypes.byref(n), None) == INVALID
    assert lib.vla_partition_rows(4, 10, fake, 3, 3, None, ctypes.byref(n), None) == 0 and n.value == 0
    lib.vla_mesh_create_rows.argtypes = [i32, i32, i64, i64, vp, vp, i64, vp, i32, i32, vp, ctypes.POINTER(vp)]
    hm = vp()
    for r0, r1 in ((-1, 3), (3, 3), (0, 11)):
        assert lib.vla_mesh_create_rows(3, 1, 10, 4, fake, fake, 0, None, r0, r1, None, ctypes.byref(hm)) == INVALID
    assert lib.vla_mesh_create_rows(4, 1, 10, 4, fake, fake, 0, None, 0, 5, None, ctypes.byref(hm)) == INVALID
    assert lib.vla_mesh_create_rows(3, 1, 10, 4, None, fake, 0, None, 0, 5, None, ctypes.byref(hm)) == INVALID
    lib.vla_element_pages_static_check.argtypes = [ctypes.POINTER(i64), vp]

    lib.vla_batch_create.argtypes = [vp, i32, i32, vp, i32, vp, ctypes.POINTER(vp)]
    lib.vla_batch_assemble.argtypes = [vp, i32, i32, vp, vp]
    h = vp()
    jobs = ctypes.create_string_buffer(1024)
    assert lib.vla_batch_create(None, 0, 1, None, 0, None, ctypes.byref(h)) == INVALID
    assert lib.vla_batch_create(jobs, 1, 7, None, 0, None, ctypes.byref(h)) == INVALID     # precision
    assert lib.vla_batch_create(jobs, 1, 1, None, 1 << 10, None, ctypes.byref(h)) == INVALID   # unknown flag
    assert lib.vla_batch_assemble(None, 0, 1, None, None) == INVALID

    class Tune(ctypes.Structure):
        _fields_ = [("tile_budget", i32), ("ctas_per_sm", i32), ("us", f64)]

    lib.vla_tune_get.argtypes = [i32, i32, i32, ctypes.POINTER(Tune)]
    lib.vla_tune_set.argtypes = [i32, i32, i32, ctypes.POINTER(Tune)]
    t = Tune(-1, 0, 0.0)
    assert lib.vla_tune_get(4, 1, 1, ctypes.byref(t)) == INVALID
    assert lib.vla_tune_set(3, 1, 1, ctypes.byref(t)) == INVALID                          # negative budget
    lib.vla_autotune.argtypes = [i32, i32, i32, i64, i64, vp, vp, i32, vp, ctypes.POINTER(Tune)]
    assert lib.vla_autotune(4, 1, 1, 10, 10, fake, fake, 3, None, ctypes.byref(t)) == INVALID

    class ServerConfig(ctypes.Structure):
        _fields_ = [("hbm_budget_bytes", i64), ("precision", i32), ("ingest_workers", i32),
                    ("max_batch", i32), ("max_inflight", i32)]

    lib.vla_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    for cfg in (ServerConfig(0, 1, 4, 0, 0), ServerConfig(1 << 30, 5, 4, 0, 0), ServerConfig(1 << 30, 1, 65, 0, 0)):
        assert lib.vla_server_create(ctypes.byref(cfg), ctypes.byref(h)) == INVALID
    lib.vla_server_poll.argtypes = [vp, i64, f64, vp]
    assert lib.vla_server_submit(None, None, None) == INVALID
    assert lib.vla_server_poll(None, 0, 0.0, None) == INVALID
    assert lib.vla_server_release(None, ctypes.c_int64(0)) == INVALID
    assert lib.vla_server_stats(None, None) == INVALID

    lib.vla_assemble.argtypes = [vp, i32, f64, f64, i32, vp, vp, vp, vp, vp, vp, vp]
    assert lib.vla_assemble(None, 0, 1.0, 0.0, 1, None, None, None, None, None, None, None) == INVALID
    lib.vla_mesh_csr_view.argtypes = [vp, vp, vp]
    assert lib.vla_mesh_csr_view(None, None, None) == INVALID
    lib.vla_assemble_with_boundary.argtypes = [vp, i32, f64, f64, i32] + [vp] * 9
    assert lib.vla_assemble_with_boundary(None, 0, 1.0, 0.0, 1, *([None] * 9)) == INVALID
    for name, nargs in (("vla_boundary", 5), ("vla_simplex_normals", 3), ("vla_mesh_csr", 4), ("vla_mesh_check", 2),
                        ("vla_mesh_info", 2), ("vla_quad_points", 5), ("vla_rhs", 6), ("vla_energies", 8),
                        ("vla_mesh_facets", 7)):
        args = [None] * nargs
        if name in ("vla_boundary", "vla_quad_points", "vla_rhs"):
            args[1] = 1
        assert getattr(lib, name)(*args) == INVALID, name
    for name in ("vla_mesh_destroy", "vla_batch_destroy", "vla_server_destroy"):
        assert getattr(lib, name)(None) == 0, name
