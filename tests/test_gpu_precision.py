"""Mixed precision on both sides of the fast path's guard, per element.

The mixed-precision element path computes the geometry in plain FP32 while
|det V| >= perm(|V|)/4 and switches to the float-pair (compensated) path below
that.  These simplices spread |det|/perm from about 1 down to 1/650 near
(37, -11, 5), so both paths run, and every element's K_k (entrywise), M_k and
volume must lie within the bound that tests/mixed_bounds.py derives for the
path it takes (the same bound an FP32 emulation of the fast path meets on the
CPU, tests/test_mixed_bounds.py).  Both mixed-precision entry points that form
element pages are checked: the tiled assembly (vla_assemble with pages) and
the allocation-free vla_element_pages_static.
"""
import numpy as np
import pytest
import torch

import mixed_bounds as mb
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _check(B, Kr, Mr, vol_r, K, M, vol):
    # K: entrywise against the bound (plus the oracle's own FP64 rounding, ~1e-14 of the page)
    slack = 1e-13 * np.abs(Kr).max(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(K - Kr) <= B["K_bound"] + slack), float(np.max(np.abs(K - Kr) / (B["K_bound"] + slack)))
    assert np.all(np.abs(vol - vol_r) / vol_r <= B["theta_vol"] + 1e-13)
    assert np.all(np.abs(M - Mr) / np.abs(Mr) <= B["theta_M"][:, None, None] + 1e-13)
    # below the guard the float-pair path holds vol within 10u although perm/|det| reaches 100 and more
    s = B["slow"]
    assert np.all(np.abs(vol - vol_r)[s] / vol_r[s] <= 10 * mb.U)


@pytest.mark.parametrize("dim", [3, 2])
def test_guard_band_per_element_bounds(vla, dim):
    co, el = mb.band_simplices(dim, 3000, seed=11)
    ca, cb = 0.5, 2.0
    B = mb.p1_bounds(dim, co, el, ca, cb)
    assert B["fast"].sum() > 500 and B["slow"].sum() > 500 and B["r"].max() > 100
    Kr, Mr, vol_r, _ = oracle.element_pages(dim, 1, el, co, ca, cb)
    c, e = torch.from_numpy(co).cuda(), torch.from_numpy(el).cuda()
    gm = vla.Mesh(c, e)
    out = gm.assemble(ca, cb, precision=vla.PREC_MIXED, pages=True)
    st = vla.element_pages_static(c, e, ca=ca, cb=cb, precision=vla.PREC_MIXED)
    torch.cuda.synchronize()
    for res in (out, st):
        _check(B, Kr, Mr, vol_r, res["K3D"].cpu().numpy(), res["M3D"].cpu().numpy(), res["vol"].cpu().numpy())
    # the two entry points run the same element arithmetic: identical pages
    for k in ("K3D", "M3D", "vol"):
        assert torch.equal(out[k], st[k]), k
    # the CSR values of disjoint elements are the page entries themselves, each a one-term compensated sum
    ref = oracle.assemble(dim, 1, len(co), el, co, ca, cb)
    for k in ("K", "M"):
        got = out[k].cpu().numpy()
        assert np.linalg.norm(got - ref[k]) / np.linalg.norm(ref[k]) <= 1e-5, k
    gm.close()
