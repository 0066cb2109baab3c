"""The allocation-free entry point vla_element_pages_static, called through the
C ABI.  It serves callers that cannot allocate device memory where they need
element matrices; its scratch is a fixed device array inside the library,
shared by every call, so two calls in a row on different meshes must not see
each other's data.  Each call is checked against the FP64 oracle (P1 and P2,
2-D and 3-D, both coefficient kinds) and against the handle-based path
(vla_mesh_create + vla_assemble), whose element arithmetic it shares bit for
bit.  An element with a node index outside [0, nn) is skipped on the device
before any coordinate is read and reported by vla_element_pages_static_check.
This file is collected last so that a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}   # FP64: relative to the page scale; mixed: relative Frobenius per element


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _static_pages(vla, m, precision, kind, ca, cb, elems=None):
    """Direct ctypes call of the C entry point with caller-owned buffers."""
    L = vla.lib()
    coords = torch.from_numpy(m.coords).cuda()
    elems = torch.from_numpy(m.elems if elems is None else elems).cuda()
    ne = elems.shape[0]
    Kp = torch.full((ne, m.nlb, m.nlb), 7.0, dtype=torch.float64, device="cuda")
    Mp = torch.full_like(Kp, 7.0)
    vol = torch.full((ne,), 7.0, dtype=torch.float64, device="cuda")
    ns = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = L.vla_element_pages_static(m.dim, m.order, m.nn, ne, ctypes.c_void_p(coords.data_ptr()),
                                    ctypes.c_void_p(elems.data_ptr()), kind, ca, cb, precision,
                                    ctypes.c_void_p(Kp.data_ptr()), ctypes.c_void_p(Mp.data_ptr()),
                                    ctypes.c_void_p(vol.data_ptr()), ctypes.c_void_p(ns.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return Kp.cpu().numpy(), Mp.cpu().numpy(), vol.cpu().numpy(), int(ns.item())


def _skipped(vla):
    n = ctypes.c_int64(-1)
    st = vla.lib().vla_element_pages_static_check(ctypes.byref(n),
                                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, int(n.value)


def _handle_pages(vla, m, precision, kind, ca, cb):
    gm = vla.Mesh(torch.from_numpy(m.coords).cuda(), torch.from_numpy(m.elems).cuda(), order=m.order)
    out = gm.assemble(ca, cb, kind=kind, precision=precision, pages=True, count_singular=True)
    torch.cuda.synchronize()
    res = (out["K3D"].cpu().numpy(), out["M3D"].cpu().numpy(), out["vol"].cpu().numpy(), int(out["n_singular"].item()))
    gm.close()
    return res


def _against_oracle(m, got, precision, kind, ca, cb):
    Kr, Mr, vr, _ = oracle.element_pages(m.dim, m.order, m.elems, m.coords, ca, cb, ckind=kind)
    tol = TOL[precision]
    for g, r in ((got[0], Kr), (got[1], Mr)):
        assert np.all(np.isfinite(g))
        if precision == 0:
            err = np.abs(g - r).max(axis=(1, 2)) / np.abs(r).max(axis=(1, 2))
        else:
            err = np.linalg.norm(g - r, axis=(1, 2)) / np.linalg.norm(r, axis=(1, 2))
        assert err.max() <= tol, float(err.max())
    assert np.all(np.abs(got[2] - vr) <= tol * vr)


MESHES = [  # (mesh, coefficient kind, ca, cb): every element type, both coefficient kinds
    (lambda: meshgen.kuhn_cube(7, jitter=0.1, seed=3), 0, 1.0, 1.0),
    (lambda: meshgen.kuhn_cube(5, order=2, jitter=0.1, seed=8), 0, 0.5, 2.0),
    (lambda: meshgen.unit_square(13, jitter=0.1, seed=5), 1, 1.5, 0.7),
    (lambda: meshgen.unit_square(9, order=2, jitter=0.1, seed=6), 0, 0.8, 1.3),
    (lambda: meshgen.kuhn_cube(4, jitter=0.1, seed=9), 1, 0.6, -0.4),
]


@pytest.mark.parametrize("precision", [0, 1])
def test_static_pages_match_oracle_and_handle_path(vla, precision):
    # several calls in a row on different meshes (the shared scratch keeps the
    # last call's contents): each against the oracle and, bit for bit, against
    # the handle-based assembly of the same mesh
    for make, kind, ca, cb in MESHES:
        m = make()
        got = _static_pages(vla, m, precision, kind, ca, cb)
        _against_oracle(m, got, precision, kind, ca, cb)
        ref = _handle_pages(vla, m, precision, kind, ca, cb)
        for g, r in zip(got[:3], ref[:3]):
            assert np.array_equal(g, r)
        assert got[3] == ref[3] == 0
        assert _skipped(vla) == (0, 0)


def test_static_pages_skip_out_of_range_indices(vla):
    # indices outside [0, nn) reach the C entry point unchecked (the binding
    # checks them; this calls the ABI directly): the kernel tests every index
    # before it reads a coordinate, skips the element and counts it
    m = meshgen.kuhn_cube(3, jitter=0.1, seed=2)
    el = m.elems.copy()
    el[5, 1] = m.nn
    el[17, 3] = -4
    got = _static_pages(vla, m, 1, 0, 1.0, 0.0, elems=el)
    assert _skipped(vla) == (-2, 2)   # VLA_ERR_INDEX_OOB, two elements
    for k in (5, 17):
        assert np.all(np.isnan(got[0][k])) and np.all(np.isnan(got[1][k])) and np.isnan(got[2][k])
    ok = np.ones(m.ne, bool)
    ok[[5, 17]] = False
    ref = _handle_pages(vla, m, 1, 0, 1.0, 0.0)
    assert np.array_equal(got[0][ok], ref[0][ok]) and np.array_equal(got[2][ok], ref[2][ok])
    # the next call starts from a cleared counter
    _static_pages(vla, m, 1, 0, 1.0, 0.0)
    assert _skipped(vla) == (0, 0)


def test_static_pages_rejects_oversized_mesh(vla):
    L = vla.lib()
    st = L.vla_element_pages_static(3, 1, (1 << 18) + 1, 10, ctypes.c_void_p(8), ctypes.c_void_p(8), 0, 1.0, 0.0, 1,
                                    None, None, None, None, None)
    assert st == -6
    buf = ctypes.create_string_buffer(512)
    L.vla_last_error(buf, 512)
    assert b"exceed" in buf.value
