"""CPU checks of the per-element error bounds of the mixed-precision P1 path
(tests/mixed_bounds.py): the exact element quantities the bounds start from
agree with the FP64 oracle, an operation-by-operation FP32 emulation of the
fast path stays inside them on simplices that straddle the perm/4 guard, and
the fast path's determinant bound stays below 11u perm (44u relative at the
guard).  The GPU test of the same elements is tests/test_gpu_precision.py."""
import numpy as np
import pytest

import mixed_bounds as mb
import oracle

U = mb.U


@pytest.mark.parametrize("dim", [3, 2])
def test_exact_quantities_match_oracle(dim):
    co, el = mb.band_simplices(dim, 500, seed=2)
    B = mb.p1_bounds(dim, co, el, 0.5, 2.0)
    Kr, Mr, vol, _ = oracle.element_pages(dim, 1, el, co, 0.5, 2.0)
    np.testing.assert_allclose(B["K"], Kr, rtol=0, atol=1e-12 * np.abs(Kr).max())
    np.testing.assert_allclose(B["vol"], vol, rtol=1e-12)


@pytest.mark.parametrize("dim", [3, 2])
def test_fp32_emulation_within_bounds(dim):
    co, el = mb.band_simplices(dim, 3000, seed=1)
    B = mb.p1_bounds(dim, co, el, 0.5, 2.0)
    E = mb.emulate_fast_p1(dim, co, el, 0.5, 2.0)
    Kr, Mr, vol, _ = oracle.element_pages(dim, 1, el, co, 0.5, 2.0)
    # the emulated guard sends exactly the elements with perm/|det| < 4 to the fast path
    assert np.array_equal(E["fast"][B["fast"] | B["slow"]], B["fast"][B["fast"] | B["slow"]])
    assert B["fast"].sum() > 500 and B["slow"].sum() > 500
    f = E["fast"]
    assert np.all(np.abs(E["K"] - Kr)[f] <= B["K_bound"][f])
    assert np.all((np.abs(E["vol"] - vol) / vol)[f] <= B["theta_vol"][f])
    moff = Mr[:, 0, 1]
    assert np.all((np.abs(E["mscale"] - moff) / moff)[f] <= B["theta_M"][f])


@pytest.mark.parametrize("dim", [3, 2])
def test_fast_path_det_bound_at_the_guard(dim):
    co, el = mb.band_simplices(dim, 2000, seed=3)
    B = mb.p1_bounds(dim, co, el, 1.0, 0.0)
    f = B["fast"]
    # 3-D: u (2Q + 5 perm) <= 11u perm, so <= 44u |det| while perm <= 4 |det|; 2-D: 4u perm2 + 2u |det| <= 18u |det|
    # (the 1e-3 covers the O(u^2 X) terms of coordinates far from the origin)
    cap = (44 if dim == 3 else 18) * U * mb.MARGIN * 1.001 + 2 * U
    assert np.all(B["theta_vol_fast"][f] <= cap)
    # below the guard the float-pair path keeps vol within 10u where perm/|det| reaches 100 and more
    # (the fast path's bound there would be 11u perm/|det|)
    s = B["slow"]
    assert B["r"][s].max() > 100
    assert np.all(B["theta_det_exact"][s] + 2 * U <= 10 * U)
