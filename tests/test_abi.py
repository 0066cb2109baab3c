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
