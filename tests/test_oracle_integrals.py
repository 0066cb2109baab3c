"""Pins of the oracle's quadrature, GI integrals, load vector, local energies
and avtamav (Sections 2.4, 3.4, 3.5) against closed forms, exactness degrees
and invariants -- none of them re-types an oracle formula.

  * a rule of degree p integrates every barycentric monomial of degree <= p
    exactly: the mean of lambda^alpha over a simplex is alpha! d! / (|alpha| + d)!;
  * unit-cube integrals of polynomials have closed forms;
  * the divergence theorem ties the surface integral (facet normals and areas)
    to the volume integral (Section 3.4);
  * the load vector of f = 1 sums to the volume, and for a linear f it equals
    the consistent mass matrix times the nodal values of f (Section 3.5's
    remark b = M_0 f);
  * energies of a linear u have closed forms and the local energies sum to
    the global quadratic forms u^T K u / 2, u^T M u / 2, -b^T u.
"""
import itertools
import math

import numpy as np
import pytest

import meshgen
import oracle


def _monomials(nv, deg):
    for alpha in itertools.product(range(deg + 1), repeat=nv):
        if sum(alpha) <= deg:
            yield alpha


def _mean_bary_monomial(alpha, d):
    num = math.prod(math.factorial(a) for a in alpha)
    return num * math.factorial(d) / math.factorial(sum(alpha) + d)


@pytest.mark.parametrize("sdim", [1, 2, 3])
@pytest.mark.parametrize("gqo", [1, 2, 3])
def test_rule_exact_to_its_degree(sdim, gqo):
    ip, w = oracle.quad_rule(sdim, gqo)
    assert np.all(np.abs(ip.sum(axis=1) - 1.0) < 1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    exact_deg = 3 if (sdim == 1 and gqo == 2) else gqo   # the 2-point Gauss rule is exact to degree 3
    for alpha in _monomials(sdim + 1, exact_deg):
        q = np.sum(w * np.prod(ip ** np.array(alpha), axis=1))
        assert abs(q - _mean_bary_monomial(alpha, sdim)) < 1e-14, (alpha, q)
    # and not beyond: some monomial of the next degree is missed
    misses = [abs(np.sum(w * np.prod(ip ** np.array(a), axis=1)) - _mean_bary_monomial(a, sdim))
              for a in _monomials(sdim + 1, exact_deg + 1) if sum(a) == exact_deg + 1]
    assert max(misses) > 1e-6


def test_rule_unsupported():
    with pytest.raises(ValueError):
        oracle.quad_rule(3, 4)


def _cube(n, jitter=0.1, seed=0):
    return meshgen.kuhn_cube(n, jitter=jitter, seed=seed)


def test_quadrature_points_are_barycentric_combinations():
    m = _cube(2)
    ip, w = oracle.quad_rule(3, 3)
    X = oracle.quad_points(3, m.elems, m.coords, ip)
    assert X.shape == (m.ne, len(w), 3)
    # the centroid point (first point of the degree-3 rule) is the vertex mean
    cen = m.coords[m.elems].mean(axis=1)
    np.testing.assert_allclose(X[:, 0, :], cen, rtol=0, atol=1e-15)
    # every point lies in its element's bounding box
    lo, hi = m.coords[m.elems].min(axis=1), m.coords[m.elems].max(axis=1)
    assert np.all(X >= lo[:, None, :] - 1e-15) and np.all(X <= hi[:, None, :] + 1e-15)


def test_volume_integrals_unit_cube():
    # Section 3.4: mass of rho = x1^2 + x2^2 and its first moments over the unit cube
    m = _cube(4)
    vol, _ = oracle.volumes(3, m.elems, m.coords)
    ip, w = oracle.quad_rule(3, 3)
    X = oracle.quad_points(3, m.elems, m.coords, ip)
    rho = X[..., 0] ** 2 + X[..., 1] ** 2
    mass = oracle.gi(rho[..., None], w, vol)[0]
    assert mass == pytest.approx(2.0 / 3.0, abs=1e-14)
    M = oracle.gi((rho[..., None] * X), w, vol)          # int x_i rho
    np.testing.assert_allclose(M, [5.0 / 12.0, 5.0 / 12.0, 1.0 / 3.0], rtol=0, atol=1e-14)
    one = oracle.gi(np.ones((m.ne, len(w), 1)), w, vol)[0]
    assert one == pytest.approx(1.0, abs=1e-14)


def test_divergence_theorem_unit_cube():
    # F = (x1^2, x2^2, x3^2): flux through the boundary = int div F = int 2(x1+x2+x3) = 3
    m = _cube(3)
    nrm, ar, miss = oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
    assert miss == 0
    ip, w = oracle.quad_rule(2, 2)
    Xb = oracle.quad_points(3, m.faces, m.coords, ip)
    flux = oracle.gi(Xb ** 2, w, ar, normals=nrm)
    assert flux == pytest.approx(3.0, abs=1e-13)
    vol, _ = oracle.volumes(3, m.elems, m.coords)
    ipv, wv = oracle.quad_rule(3, 1)
    Xv = oracle.quad_points(3, m.elems, m.coords, ipv)
    div = oracle.gi(2.0 * Xv.sum(axis=2, keepdims=True), wv, vol)[0]
    assert div == pytest.approx(3.0, abs=1e-13)


def test_moment_of_inertia_volume_and_surface_agree():
    # Section 3.4: F = (x1^3 (x2^2 + x3^2)/3, x2^5/5, x2^2 x3^3/3) has
    # div F = (x1^2 + x2^2)(x2^2 + x3^2); on the unit cube I_1 = 8/15.
    errs_v, errs_s = [], []
    for n in (2, 4, 8):
        m = _cube(n, jitter=0.0)
        vol, _ = oracle.volumes(3, m.elems, m.coords)
        ip, w = oracle.quad_rule(3, 3)
        X = oracle.quad_points(3, m.elems, m.coords, ip)
        x1, x2, x3 = X[..., 0], X[..., 1], X[..., 2]
        Iv = oracle.gi(((x1 ** 2 + x2 ** 2) * (x2 ** 2 + x3 ** 2))[..., None], w, vol)[0]
        nrm, ar, _ = oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
        ipb, wb = oracle.quad_rule(2, 3)
        Y = oracle.quad_points(3, m.faces, m.coords, ipb)
        y1, y2, y3 = Y[..., 0], Y[..., 1], Y[..., 2]
        F = np.stack([y1 ** 3 * (y2 ** 2 + y3 ** 2) / 3, y2 ** 5 / 5, y2 ** 2 * y3 ** 3 / 3], axis=-1)
        Is = oracle.gi(F, wb, ar, normals=nrm)
        errs_v.append(abs(Iv - 8 / 15))
        errs_s.append(abs(Is - 8 / 15))
    # on the cube's faces F.n is a polynomial of degree <= 2: the surface rule is exact;
    # the degree-4 volume integrand converges at order 4 in h
    assert max(errs_s) < 1e-13
    assert errs_v[-1] < 1e-5 and errs_v[0] / errs_v[-1] > 100


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_load_vector_closed_forms(dim, order):
    m = meshgen.make_mesh(dim, 3 if dim == 3 else 5, order=order, jitter=0.1, seed=4)
    vol, _ = oracle.volumes(dim, m.elems, m.coords)
    gqo = 3 if order == 2 else 2
    ip, w = oracle.quad_rule(dim, gqo)
    X = oracle.quad_points(dim, m.elems, m.coords, ip)
    # f = 1: b sums to the domain measure; for P1, b_i = sum over incident elements |T|/(dim+1)
    b, b2D = oracle.rhs(dim, order, m.nn, m.elems, m.coords, ip, w, np.ones((m.ne, len(w))))
    assert b.sum() == pytest.approx(1.0, abs=1e-13)
    if order == 1:
        ref = np.zeros(m.nn)
        np.add.at(ref, m.elems.ravel(), np.repeat(vol / (dim + 1), dim + 1))
        np.testing.assert_allclose(b, ref, rtol=0, atol=1e-15)
    # f linear: b = M_0 f~ (f~ its nodal values; the rule integrates f phi_j exactly)
    fx = lambda Y: 0.3 + 1.7 * Y[..., 0] - 0.6 * Y[..., 1]
    b, _ = oracle.rhs(dim, order, m.nn, m.elems, m.coords, ip, w, fx(X))
    A = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 1.0, 0.0)
    M0 = oracle.to_dense(m.nn, A["row_ptr"], A["col_idx"], A["M"])
    np.testing.assert_allclose(b, M0 @ fx(m.coords), rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_energies_closed_forms_and_sums(dim, order):
    # u = x1 (reproduced exactly), c = 1: J1 = |Omega|/2 = 1/2, J2 = int x1^2 / 2 = 1/6;
    # f = 1: J3 = -int u = -1/2.  Local energies sum to the global quadratic forms.
    m = meshgen.make_mesh(dim, 3, order=order, jitter=0.1, seed=8)
    A = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 1.0, 0.0, want_pages=True)
    gqo = 3 if order == 2 else 2
    ip, w = oracle.quad_rule(dim, gqo)
    b, b2D = oracle.rhs(dim, order, m.nn, m.elems, m.coords, ip, w, np.ones((m.ne, len(w))))
    u = m.coords[:, 0].copy()
    J = oracle.energies(m.elems, u, A["K3D"], A["M3D"], b2D)
    assert J[:, 0].sum() == pytest.approx(0.5, abs=1e-13)
    assert J[:, 1].sum() == pytest.approx(1.0 / 6.0, abs=1e-13)
    assert J[:, 2].sum() == pytest.approx(-0.5, abs=1e-13)
    K = oracle.to_dense(m.nn, A["row_ptr"], A["col_idx"], A["K"])
    M = oracle.to_dense(m.nn, A["row_ptr"], A["col_idx"], A["M"])
    v = np.random.default_rng(1).standard_normal(m.nn)
    Jv = oracle.energies(m.elems, v, A["K3D"], A["M3D"], b2D)
    assert Jv[:, 0].sum() == pytest.approx(0.5 * v @ K @ v, rel=1e-12)
    assert Jv[:, 1].sum() == pytest.approx(0.5 * v @ M @ v, rel=1e-12)
    assert Jv[:, 2].sum() == pytest.approx(-b @ v, rel=1e-12)
    assert np.all(Jv[:, 0] >= -1e-14) and np.all(Jv[:, 1] >= 0)   # K_k PSD, M_k SPD


def test_avtamav_against_numpy():
    rng = np.random.default_rng(5)
    for n in (2, 3, 4, 10):
        v, w = rng.standard_normal((37, n)), rng.standard_normal((37, n))
        A = rng.standard_normal((37, n, n))                 # (N, cols, rows)
        ref = np.einsum("kr,kcr,kc->k", v, A, w)           # v^T A w with A[k][r, c] = A[k, c, r]
        np.testing.assert_allclose(oracle.avtamav(v, A, w), ref, rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# the paper's literal P1 listing: degree-2 rule, coefficient at every point
# --------------------------------------------------------------------------

def _literal(dim, m, ca, cb, kind):
    return oracle.assemble(dim, 1, m.nn, m.elems, m.coords, ca, cb, want_pages=True, ckind=kind)


@pytest.mark.parametrize("dim", [2, 3])
def test_literal_constant_coefficient_is_exact(dim):
    # c constant: the literal K equals the centroid K, and M the exact P1 mass
    m = meshgen.make_mesh(dim, 3, jitter=0.1, seed=2)
    lit = _literal(dim, m, 1.7, 0.0, 2)
    cen = _literal(dim, m, 1.7, 0.0, 0)
    np.testing.assert_allclose(lit["K3D"], cen["K3D"], rtol=1e-13, atol=1e-15)
    vol, _ = oracle.volumes(dim, m.elems, m.coords)
    Mexact = 1.7 * vol[:, None, None] * (1 + np.eye(dim + 1))[None] / ((dim + 1) * (dim + 2))
    np.testing.assert_allclose(lit["M3D"], Mexact, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_literal_quadratic_coefficient_stiffness_exact(dim):
    # c = a + b|x|^2 is quadratic, so the degree-2 rule gives K_k = (int_T c) G^T G exactly;
    # int_T |x|^2 = sum_jk (x_j . x_k) int lambda_j lambda_k, int lambda_j lambda_k = |T| (1 + delta_jk)/((d+1)(d+2))
    m = meshgen.make_mesh(dim, 2, jitter=0.1, seed=3)
    a, b = 0.7, 1.3
    lit = _literal(dim, m, a, b, 2)
    one = _literal(dim, m, 1.0, 0.0, 0)          # G^T G |T|
    vol, _ = oracle.volumes(dim, m.elems, m.coords)
    X = m.coords[m.elems[:, : dim + 1]]          # (ne, d+1, dim)
    gram = np.einsum("kjd,kld->kjl", X, X)
    lam2 = (1 + np.eye(dim + 1)) / ((dim + 1) * (dim + 2))
    intc = a * vol + b * vol * np.einsum("kjl,jl->k", gram, lam2)
    np.testing.assert_allclose(lit["K3D"], (intc / vol)[:, None, None] * one["K3D"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", [2, 3])
def test_literal_pages_follow_the_degree2_rule(dim, kind):
    # the literal P1 listing evaluates c at the points of the degree-2 rule (gqo = 2):
    # K_k = (sum_i w_i c(x_i)) |T| G^T G and M_k(p,q) = |T| sum_i w_i c(x_i) lam_p lam_q,
    # rebuilt here element by element with numpy (gradients from numpy.linalg.inv);
    # the rule itself is pinned to its degree of exactness above
    m = meshgen.make_mesh(dim, 2, jitter=0.1, seed=4)
    a, b = 1.2, 0.8
    lit = _literal(dim, m, a, b, kind)
    ip, w = oracle.quad_rule(dim, 2)                 # (nip, dim+1) barycentric, weights sum to 1
    for k in range(m.ne):
        X = m.coords[m.elems[k, : dim + 1]]          # (dim+1, dim)
        V = (X[:dim] - X[dim]).T                     # columns: vectors to the last vertex
        vol = abs(np.linalg.det(V)) / math.factorial(dim)
        Vi = np.linalg.inv(V)
        G = np.vstack([Vi, -Vi.sum(axis=0)])         # (dim+1, dim): row j = grad lambda_j
        xq = ip @ X                                  # (nip, dim) points
        c = a + b * np.sum(xq ** 2, axis=1) if kind == 2 else a * np.exp(b * xq.sum(axis=1))
        K = (w @ c) * vol * G @ G.T
        M = vol * np.einsum("i,ip,iq->pq", w * c, ip, ip)
        np.testing.assert_allclose(lit["K3D"][k], K, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(lit["M3D"][k], M, rtol=1e-12, atol=1e-16)


def test_literal_convergence_matches_printed_table_order():
    # c = e^{x1+x2+x3}, v = cos(pi x1) cos(pi x2) cos(pi x3) on unjittered unit cubes;
    # printed P1 3-D errors at levels 3-5: e_K 2.70e-1, 6.82e-2, 1.71e-2; e_M 5.04e-2,
    # 1.31e-2, 3.30e-3.  The cube split differs from the paper's, so the values agree in
    # order of magnitude (within 15 %) and in the rate (4 per level), not digit for digit.
    IK, IM = 19.2286024907, 0.6823216700
    printed = {3: (2.70e-1, 5.04e-2), 4: (6.82e-2, 1.31e-2), 5: (1.71e-2, 3.30e-3)}
    errs = {}
    for lev in (3, 4, 5):
        m = meshgen.kuhn_cube(2 ** lev, jitter=0.0)
        A = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0, ckind=3)
        v = np.prod(np.cos(np.pi * m.coords), axis=1)
        rows = np.repeat(np.arange(m.nn), np.diff(A["row_ptr"]))
        qk = np.sum(v[rows] * A["K"] * v[A["col_idx"]])
        qm = np.sum(v[rows] * A["M"] * v[A["col_idx"]])
        errs[lev] = (abs(qk - IK), abs(qm - IM))
        for e, p in zip(errs[lev], printed[lev]):
            assert 0.85 < e / p < 1.15, (lev, e, p)
    for i in (0, 1):
        assert 3.7 < errs[3][i] / errs[4][i] < 4.3 and 3.7 < errs[4][i] / errs[5][i] < 4.3
