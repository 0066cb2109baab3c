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


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_2404_16039_gb300 as vla
    monkeypatch.setattr(vla, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(vla, "_lib", None)
    with pytest.raises(ImportError):
        vla.lib()
