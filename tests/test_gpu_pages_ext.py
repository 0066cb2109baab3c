"""GPU parity of amt, avtav, amsm, amsv, smamt and svamt (Section 2.4)
against the FP64 oracle on the same seeded pages, in page and SoA layouts,
FP32 and FP64, with a page count that leaves a ragged tail after the
128-page chunks of the staged kernel.  amt is exact (bit-equal); the
products within 1e-12 (FP64) or 2e-6 (FP32) of the sum of absolute terms."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

N_PAGES = 128 * 9 + 37


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x.astype(dt))).cuda()


def _to_layout(A, layout):        # numpy (N, cols, rows) -> (cols, rows, N) for SoA
    return A if layout == 0 else np.ascontiguousarray(np.transpose(A, (1, 2, 0)))


def _from_layout(A, layout):
    return A if layout == 0 else np.transpose(A, (2, 0, 1))


def _tol(dt):
    return 1e-12 if dt == np.float64 else 2e-6


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("m,n", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_amt(vla, layout, dt, m, n):
    rng = np.random.default_rng(m * 10 + n)
    A = rng.standard_normal((N_PAGES, n, m)).astype(dt)           # pages m x n
    got = vla.amt(_dev(_to_layout(A, layout), dt), layout=layout).cpu().numpy()
    ref = oracle.amt(A.astype(np.float64)).astype(dt)
    np.testing.assert_array_equal(_from_layout(got, layout), ref)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("n", [2, 3])
def test_avtav(vla, layout, dt, n):
    rng = np.random.default_rng(n)
    a, b = rng.standard_normal((N_PAGES, n)), rng.standard_normal((N_PAGES, n))
    ref = oracle.avtav(a, b)
    ta = _dev(a if layout == 0 else a.T, dt)
    tb = _dev(b if layout == 0 else b.T, dt)
    got = vla.avtav(ta, tb, layout=layout).cpu().numpy().astype(np.float64)
    scale = np.sum(np.abs(a * b), axis=1)
    assert np.all(np.abs(got - ref) <= _tol(dt) * scale + 1e-300)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("m,p,n", [(3, 4, 5), (2, 2, 2), (1, 10, 8), (3, 3, 16)])
def test_amsm_smamt(vla, layout, dt, m, p, n):
    rng = np.random.default_rng(m * 100 + p * 10 + n)
    A = rng.standard_normal((N_PAGES, p, m))                        # pages m x p
    S = rng.standard_normal((n, p))                                 # p x n
    ref = oracle.amsm(A, S)
    got = vla.amsm(_dev(_to_layout(A, layout), dt), _dev(S, dt), layout=layout).cpu().numpy()
    absref = oracle.amsm(np.abs(A), np.abs(S))
    assert np.all(np.abs(_from_layout(got, layout).astype(np.float64) - ref) <= _tol(dt) * absref + 1e-300)
    Sp = rng.standard_normal((p, m))                                # m x p
    B = rng.standard_normal((N_PAGES, p, n))                        # pages n x p
    ref2 = oracle.smamt(Sp, B)
    got2 = vla.smamt(_dev(Sp, dt), _dev(_to_layout(B, layout), dt), layout=layout).cpu().numpy()
    absref2 = oracle.smamt(np.abs(Sp), np.abs(B))
    assert np.all(np.abs(_from_layout(got2, layout).astype(np.float64) - ref2) <= _tol(dt) * absref2 + 1e-300)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("m,n", [(3, 4), (1, 5), (10, 1)])
def test_amsv_svamt(vla, layout, dt, m, n):
    rng = np.random.default_rng(m * 10 + n)
    A = rng.standard_normal((N_PAGES, n, m))                        # pages m x n
    s = rng.standard_normal(n)
    ref = oracle.amsv(A, s)
    absref = oracle.amsv(np.abs(A), np.abs(s))
    tA, ts = _dev(_to_layout(A, layout), dt), _dev(s, dt)
    for fn in (lambda: vla.amsv(tA, ts, layout=layout), lambda: vla.svamt(ts, tA, layout=layout)):
        got = fn().cpu().numpy().astype(np.float64)
        got = got if layout == 0 else got.T
        assert np.all(np.abs(got - ref) <= _tol(dt) * absref + 1e-300)


def test_single_object_argument_checks(vla):
    A = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        vla.amsm(A, torch.zeros((2, 2), dtype=torch.float64, device="cuda"))
    L = vla.lib()
    # dimensions above 16 are refused before any work
    assert L.vla_amsm(1, 0, 4, 17, 3, 3, A.data_ptr(), A.data_ptr(), A.data_ptr(), None) < 0
    # zero pages: nothing to do
    empty = torch.empty((0, 3, 3), dtype=torch.float64, device="cuda")
    assert vla.amt(empty).shape == (0, 3, 3)
