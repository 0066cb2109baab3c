"""The allocation-free entry point vla_element_pages_static, called through the
C ABI, against the element pages and volumes of the handle-based path
(vla_mesh_create + vla_assemble).  It serves callers that cannot allocate
device memory where they need element matrices; its scratch is a fixed device
array inside the library, shared by every call, so two calls in a row on
different meshes must not see each other's data.  This file is collected last
so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _static_pages(vla, m, precision, ca, cb):
    """Direct ctypes call of the C entry point with caller-owned buffers."""
    L = vla.lib()
    coords = torch.from_numpy(m.coords).cuda()
    elems = torch.from_numpy(m.elems).cuda()
    Kp = torch.full((m.ne, m.nlb, m.nlb), np.nan, dtype=torch.float64, device="cuda")
    Mp = torch.full_like(Kp, np.nan)
    vol = torch.full((m.ne,), np.nan, dtype=torch.float64, device="cuda")
    ns = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = L.vla_element_pages_static(m.dim, m.order, m.nn, m.ne, ctypes.c_void_p(coords.data_ptr()),
                                    ctypes.c_void_p(elems.data_ptr()), 0, ca, cb, precision,
                                    ctypes.c_void_p(Kp.data_ptr()), ctypes.c_void_p(Mp.data_ptr()),
                                    ctypes.c_void_p(vol.data_ptr()), ctypes.c_void_p(ns.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return Kp.cpu().numpy(), Mp.cpu().numpy(), vol.cpu().numpy(), int(ns.item())


def _handle_pages(vla, m, precision, ca, cb):
    gm = vla.Mesh(torch.from_numpy(m.coords).cuda(), torch.from_numpy(m.elems).cuda(), order=m.order)
    out = gm.assemble(ca, cb, precision=precision, pages=True, count_singular=True)
    torch.cuda.synchronize()
    res = (out["K3D"].cpu().numpy(), out["M3D"].cpu().numpy(), out["vol"].cpu().numpy(), int(out["n_singular"].item()))
    gm.close()
    return res


@pytest.mark.parametrize("precision", [0, 1])
def test_static_pages_match_handle_path_twice(vla, precision):
    # two calls in a row on different meshes (the shared scratch keeps the last
    # call's contents), each against the handle-based assembly of the same mesh
    tol = 1e-12 if precision == 0 else 1e-5
    meshes = [(meshgen.kuhn_cube(7, jitter=0.1, seed=3), 1.0, 1.0),
              (meshgen.kuhn_cube(5, order=2, jitter=0.1, seed=8), 0.5, 2.0)]
    for m, ca, cb in meshes:
        got = _static_pages(vla, m, precision, ca, cb)
        ref = _handle_pages(vla, m, precision, ca, cb)
        for g, r in zip(got[:3], ref[:3]):
            assert np.all(np.isfinite(g))
            err = np.abs(g - r).max(axis=tuple(range(1, g.ndim))) if g.ndim > 1 else np.abs(g - r)
            scale = np.abs(r).max(axis=tuple(range(1, r.ndim))) if r.ndim > 1 else np.abs(r)
            assert np.all(err <= tol * scale), float((err / scale).max())
        assert got[3] == ref[3] == 0


def test_static_pages_rejects_oversized_mesh(vla):
    L = vla.lib()
    st = L.vla_element_pages_static(3, 1, (1 << 18) + 1, 10, ctypes.c_void_p(8), ctypes.c_void_p(8), 0, 1.0, 0.0, 1,
                                    None, None, None, None, None)
    assert st == -6
    buf = ctypes.create_string_buffer(512)
    L.vla_last_error(buf, 512)
    assert b"exceed" in buf.value
