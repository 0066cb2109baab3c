"""GPU parity of quadrature points, the GI integrals, the load vector, the
local energies and avtamav against the FP64 oracle (same seeded inputs), and
the unit-cube closed forms at full size (64^3 x 6 tets)."""
import numpy as np
import pytest
import torch

import meshgen
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gm(vla, m):
    return vla.Mesh(_dev(m.coords), _dev(m.elems), _dev(m.faces) if m.nfb else None, order=m.order)


def _close(got, ref, tol=TOL64):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.abs(got - ref).max() <= tol * scale, float(np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("sdim", [1, 2, 3])
@pytest.mark.parametrize("gqo", [1, 2, 3])
def test_rules_match_oracle(vla, sdim, gqo):
    ip, w = vla.quad_rule(sdim, gqo)
    ipr, wr = oracle.quad_rule(sdim, gqo)
    np.testing.assert_allclose(ip, ipr, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-15)
    with pytest.raises(vla.VlaError):
        vla.quad_rule(sdim, 4)


CASES = [(2, 1, 7), (3, 1, 4), (2, 2, 5), (3, 2, 2)]


@pytest.mark.parametrize("dim,order,n", CASES)
@pytest.mark.parametrize("gqo", [1, 2, 3])
def test_points_gi_rhs_energies(vla, dim, order, n, gqo):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=10 * n + gqo)
    gm = _gm(vla, m)
    ip, w = oracle.quad_rule(dim, gqo)
    Xr = oracle.quad_points(dim, m.elems, m.coords, ip)
    X = gm.quad_points(gqo)
    _close(X, Xr, 1e-15)
    # facets
    ipb, wb = oracle.quad_rule(dim - 1, gqo)
    Yr = oracle.quad_points(dim, m.faces, m.coords, ipb)
    Y = gm.quad_points(gqo, facets=True)
    _close(Y, Yr, 1e-15)
    # GI: volume integral of rho = 1 + x1^2 + x2 x_last and its first moments; flux of F = x^2
    volr, _ = oracle.volumes(dim, m.elems, m.coords)
    rho = 1.0 + Xr[..., 0] ** 2 + Xr[..., 1] * Xr[..., dim - 1]
    fip = np.concatenate([rho[..., None], rho[..., None] * Xr], axis=2)
    ref = oracle.gi(fip, w, volr)
    out = gm.assemble(1.0, 0.0, precision=vla.PREC_FP64)
    got = vla.gi(_dev(fip), w, out["vol"])
    _close(got, ref)
    assert torch.equal(got, vla.gi(_dev(fip), w, out["vol"]))     # fixed reduction order
    nrm, ar = gm.boundary(precision=vla.PREC_FP64)
    nrm_r, ar_r, _ = oracle.boundary(dim, m.nn, m.elems, m.coords, m.faces)
    flux_r = oracle.gi(Yr ** 2, wb, ar_r, normals=nrm_r)
    flux = vla.gi(_dev(Yr ** 2), wb, ar, normals=nrm)
    assert abs(flux.item() - flux_r) <= TOL64 * max(1.0, abs(flux_r))
    # load vector for f = 1 + x1 - x2^2 at the points
    f = 1.0 + Xr[..., 0] - Xr[..., 1] ** 2
    br, b2Dr = oracle.rhs(dim, order, m.nn, m.elems, m.coords, ip, w, f)
    b, b2D = gm.rhs(gqo, _dev(f))
    _close(b2D, b2Dr)
    _close(b, br)
    # energies from FP64 pages and the element loads
    pg = gm.assemble(1.3, 0.4, precision=vla.PREC_FP64, pages=True)
    u = np.sin(3.0 * m.coords[:, 0]) + m.coords[:, 1]
    Jr = oracle.energies(m.elems, u, pg["K3D"].cpu().numpy(), pg["M3D"].cpu().numpy(), b2Dr)
    J, tot = gm.energies(_dev(u), pg["K3D"], pg["M3D"], b2D)
    _close(J[:, 0], Jr[:, 0])
    _close(J[:, 1], Jr[:, 1])
    _close(J[:, 2], Jr[:, 2])
    _close(tot, Jr.sum(axis=0))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("n", [2, 3, 4, 10])
def test_avtamav(vla, layout, dt, n):
    rng = np.random.default_rng(n)
    N = 1000 + 37 * n
    v, w = rng.standard_normal((N, n)), rng.standard_normal((N, n))
    A = rng.standard_normal((N, n, n))
    ref = oracle.avtamav(v, A, w)
    if layout == 0:
        tv, tA, tw = _dev(v.astype(dt)), _dev(A.astype(dt)), _dev(w.astype(dt))
    else:
        tv, tw = _dev(v.T.astype(dt)), _dev(w.T.astype(dt))
        tA = _dev(np.transpose(A, (1, 2, 0)).astype(dt))
    got = vla.avtamav(tv, tA, tw, layout=layout).cpu().numpy().astype(np.float64)
    tol = 1e-12 if dt == np.float64 else 2e-5
    scale = np.abs(v)[:, :, None] * np.abs(np.transpose(A, (0, 2, 1))) * np.abs(w)[:, None, :]
    assert np.all(np.abs(got - ref) <= tol * scale.sum(axis=(1, 2)))


def test_full_size_closed_forms(vla):
    # 64^3 x 6 jittered Kuhn tets: closed forms of the unit cube at full size
    m = meshgen.kuhn_cube(64, jitter=0.1, seed=0)
    gm = _gm(vla, m)
    out = gm.assemble(1.0, 0.0, precision=vla.PREC_FP64, pages=True)
    ip, w = vla.quad_rule(3, 3)
    X = gm.quad_points(3)
    rho = X[..., 0] ** 2 + X[..., 1] ** 2
    mass = vla.gi(rho[..., None].contiguous(), w, out["vol"]).item()
    assert mass == pytest.approx(2.0 / 3.0, abs=1e-13)
    b, b2D = gm.rhs(2, torch.ones((m.ne, 4), dtype=torch.float64, device="cuda"))
    assert b.sum().item() == pytest.approx(1.0, abs=1e-12)
    u = torch.from_numpy(m.coords[:, 0].copy()).cuda()
    _, tot = gm.energies(u, out["K3D"], out["M3D"], b2D)
    np.testing.assert_allclose(tot.cpu().numpy(), [0.5, 1.0 / 6.0, -0.5], rtol=0, atol=1e-12)
    # flux of x^2 through the 49,152 boundary triangles = 3
    nrm, ar = gm.boundary(precision=vla.PREC_FP64)
    ipb, wb = vla.quad_rule(2, 2)
    Y = gm.quad_points(2, facets=True)
    assert vla.gi((Y ** 2).contiguous(), wb, ar, normals=nrm).item() == pytest.approx(3.0, abs=1e-12)


@pytest.mark.parametrize("flux", [False, True])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_gi_every_component_count(vla, d, flux):
    # every compiled component count, volume integrals and fluxes, on random
    # signed data over more simplices than one pass of the reduction grid
    # (1024 blocks of 256) covers; bound: 1e-12 of the sum of absolute terms
    rng = np.random.default_rng(100 * d + flux)
    n, nip = 1024 * 256 + 12345, 5
    fip = rng.standard_normal((n, nip, d))
    w = rng.standard_normal(nip)
    sizes = rng.random(n)
    normals = rng.standard_normal((n, d)) if flux else None
    ref = oracle.gi(fip, w, sizes, normals)
    scale = oracle.gi(np.abs(fip), np.abs(w), sizes, None if normals is None else np.abs(normals))
    got = vla.gi(_dev(fip), w, _dev(sizes), None if normals is None else _dev(normals)).cpu().numpy()
    assert got.shape == ((1,) if flux else (d,))
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)
