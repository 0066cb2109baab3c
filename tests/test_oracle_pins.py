"""Pins of the CPU oracle to facts fixed outside it: values the paper prints,
closed forms, invariants, library routines and brute force on tiny meshes.
None of these tests uses the CUDA library."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Section 3.2: worked tetrahedron and the reference tetrahedron
# ---------------------------------------------------------------------------

def test_worked_tetrahedron(golden_dir):
    g = _golden(golden_dir, "worked_tet.json")
    coords = np.array(g["nodes_times_4"], dtype=np.float64) / 4.0
    elems = np.array([[0, 1, 2, 3]], dtype=np.int32)
    V = oracle.vectors(3, elems, coords)[0]          # [j, :] = column j
    np.testing.assert_allclose(V.T, np.array(g["vectors3D_times_4"]) / 4.0, rtol=0, atol=1e-15)
    vol, det = oracle.volumes(3, elems, coords)
    num, den = g["det_over_6"]
    assert det[0] / 6.0 == pytest.approx(num / den, abs=1e-15)
    assert vol[0] == pytest.approx(abs(num / den), abs=1e-15)
    N = oracle.simplex_normals(3, elems, coords)[0]  # [j, :] = column j
    expect = np.array([[float(Fraction(x)) for x in row] for row in g["normals3D"]])
    np.testing.assert_allclose(N.T, expect, rtol=0, atol=1e-14)


def test_reference_tetrahedron(golden_dir):
    g = _golden(golden_dir, "worked_tet.json")
    ref = np.array(g["normalsRef"], dtype=np.float64)
    x = np.array(g["reference_tet_nodes"], dtype=np.float64)
    # vertex order (e1, e2, e3, 0): the last vertex is the origin, so vectors3D = I
    # and the facet normals are normalsRef itself
    elems = np.array([[1, 2, 3, 0]], dtype=np.int32)
    vol, det = oracle.volumes(3, elems, x)
    assert vol[0] == pytest.approx(1.0 / 6.0, abs=1e-16) and det[0] == pytest.approx(1.0)
    N = oracle.simplex_normals(3, elems, x)[0]
    np.testing.assert_array_equal(N.T, ref)
    # paper's vertex order (0, e1, e2, e3): facet opposite vertex 0 has normal (1,1,1),
    # opposite e_i has -e_i
    N2 = oracle.simplex_normals(3, np.array([[0, 1, 2, 3]], np.int32), x)[0]
    np.testing.assert_allclose(N2, np.array([[1, 1, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1]]), atol=1e-15)


def test_nanson_facet_areas(golden_dir):
    # |det V| |n_j| / 2 equals the area of the facet opposite vertex j (cross product)
    g = _golden(golden_dir, "worked_tet.json")
    coords = np.array(g["nodes_times_4"], dtype=np.float64) / 4.0
    elems = np.array([[0, 1, 2, 3]], dtype=np.int32)
    _, det = oracle.volumes(3, elems, coords)
    N = oracle.simplex_normals(3, elems, coords)[0]
    for j in range(4):
        f = [q for q in range(4) if q != j]
        a, b, c = coords[f[0]], coords[f[1]], coords[f[2]]
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        assert abs(det[0]) * np.linalg.norm(N[j]) / 2.0 == pytest.approx(area, rel=1e-14)
    assert abs(det[0]) * np.linalg.norm(N[0]) / 2 == pytest.approx(0.9375, rel=1e-14)
    assert abs(det[0]) * np.linalg.norm(N[3]) / 2 == pytest.approx(math.sqrt(1075) / 32, rel=1e-14)


# ---------------------------------------------------------------------------
# Section 3.2 normals table: element / node / facet counts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("level", [1, 2, 3, 4, 5])
def test_facet_counts(golden_dir, level):
    row = [r for r in _golden(golden_dir, "facet_counts.json")["rows"] if r["level"] == level][0]
    m = meshgen.kuhn_cube(2 ** (level + 1), jitter=0.1, seed=level)
    assert m.ne == row["elements"] and m.nn == row["nodes"]
    n_all, n_bnd = oracle.count_facets(3, m.elems)
    assert n_all == row["all_faces"] and n_bnd == row["boundary_faces"]
    assert m.nfb == row["boundary_faces"]


def _p1_nnz_closed_form(dim, n):
    # a P1 pattern holds the diagonal and both directions of every mesh edge.
    # Unit square, n x n squares each cut by one diagonal: 2n(n+1) axis edges
    # and n^2 diagonals.  Unit cube, n^3 cubes x 6 Kuhn tets: 3n(n+1)^2 axis
    # edges, 3n^2(n+1) face diagonals and n^3 body diagonals.
    if dim == 2:
        return (n + 1) ** 2 + 2 * (2 * n * (n + 1) + n * n)
    return (n + 1) ** 3 + 2 * (3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3)


@pytest.mark.parametrize("dim,n", [(2, 1), (2, 4), (2, 9), (3, 1), (3, 2), (3, 5), (3, 8)])
def test_p1_pattern_size_closed_form(dim, n):
    m = meshgen.make_mesh(dim, n, jitter=0.1, seed=n)
    rp, ci = oracle.csr_pattern(m.nn, m.elems)
    assert len(ci) == rp[-1] == _p1_nnz_closed_form(dim, n)
    # the sizes of the 8^3 and 64^3 benchmark meshes
    assert _p1_nnz_closed_form(3, 8) == 9097 and _p1_nnz_closed_form(3, 64) == 4018753


# ---------------------------------------------------------------------------
# page primitives (Section 2.4) against closed forms and numpy.linalg
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3])
def test_page_primitives_vs_linalg(n):
    P = meshgen.random_pages(2000, n, seed=3)
    A, B, s, v = P["A"], P["B"], P["s"], P["v"]
    Am = np.transpose(A, (0, 2, 1))   # numpy row-major view: Am[k] is page k as an n x n matrix
    Bm = np.transpose(B, (0, 2, 1))
    Cm = np.transpose(oracle.amtam(A, B), (0, 2, 1))
    np.testing.assert_allclose(Cm, np.matmul(np.transpose(Am, (0, 2, 1)), Bm), rtol=1e-14, atol=1e-13)
    np.testing.assert_allclose(oracle.astam(s, A), s[:, None, None] * A, rtol=0, atol=0)
    np.testing.assert_allclose(oracle.avtam(v, A), np.einsum("kr,krc->kc", v, Am), rtol=1e-14, atol=1e-13)
    det = oracle.amdet(A)
    np.testing.assert_allclose(det, np.linalg.det(Am), rtol=1e-12)
    inv, det2, ns = oracle.aminv(A)
    assert ns == 0
    np.testing.assert_array_equal(det, det2)
    invm = np.transpose(inv, (0, 2, 1))
    np.testing.assert_allclose(invm, np.linalg.inv(Am), rtol=1e-11, atol=1e-13)
    eye = np.broadcast_to(np.eye(n), Am.shape)
    resid = np.abs(np.matmul(Am, invm) - eye).max(axis=(1, 2))
    assert np.all(resid <= 1e-15 * np.linalg.cond(Am) + 1e-15)


def test_page_closed_forms():
    # 2x2: det = ad - bc and inverse = [d -b; -c a]/det; rectangular amtam shapes
    A = np.array([[[1.0, 3.0], [2.0, 4.0]]])   # page (col-major) [[1,2],[3,4]]
    det = oracle.amdet(A)
    assert det[0] == -2.0
    inv, _, _ = oracle.aminv(A)
    np.testing.assert_allclose(inv[0].T, np.array([[-2.0, 1.0], [1.5, -0.5]]), atol=0)
    # singular pages are counted and produce non-finite entries
    S = np.array([[[1.0, 2.0], [2.0, 4.0]], [[2.0, 0.0], [0.0, 2.0]]])
    inv, det, ns = oracle.aminv(S)
    assert ns == 1 and det[0] == 0.0 and not np.all(np.isfinite(inv[0])) and np.all(np.isfinite(inv[1]))
    # 3x3 with a known inverse: upper triangular
    U = np.array([[1.0, 2.0, 3.0], [0.0, 1.0, 4.0], [0.0, 0.0, 1.0]])
    inv, det, _ = oracle.aminv(U.T[None])
    assert det[0] == 1.0
    np.testing.assert_allclose(inv[0].T, np.array([[1.0, -2.0, 5.0], [0.0, 1.0, -4.0], [0.0, 0.0, 1.0]]), atol=0)
    # rectangular A^T B: A 3x2 (p=3, m=2), B 3x4 -> C 2x4
    rng = np.random.default_rng(1)
    Ar = rng.standard_normal((5, 2, 3))
    Br = rng.standard_normal((5, 4, 3))
    Cr = oracle.amtam(Ar, Br)
    assert Cr.shape == (5, 4, 2)
    np.testing.assert_allclose(np.transpose(Cr, (0, 2, 1)), np.matmul(Ar, np.transpose(Br, (0, 2, 1))), rtol=1e-14)


# ---------------------------------------------------------------------------
# volumes and boundary facets on the unit square / cube
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 7), (3, 5)])
def test_volume_sum_and_boundary(dim, n):
    m = meshgen.make_mesh(dim, n, jitter=0.1, seed=11)
    vol, det = oracle.volumes(dim, m.elems, m.coords)
    assert vol.sum() == pytest.approx(1.0, abs=1e-13)
    assert np.all(vol > 0.05 / math.factorial(dim) * m.h ** dim)
    assert (det < 0).any() and (det > 0).any() or dim == 2
    nrm, ar, miss = oracle.boundary(dim, m.nn, m.elems, m.coords, m.faces)
    assert miss == 0
    assert ar.sum() == pytest.approx(2 * dim, abs=1e-13)   # cube surface 6, square perimeter 4
    # boundary nodes are not jittered: normals are exactly +-e_i and point outward
    fc = m.coords[m.faces].mean(axis=1)
    axis = np.argmax(np.abs(nrm), axis=1)
    np.testing.assert_allclose(np.abs(nrm[np.arange(m.nfb), axis]), 1.0, atol=1e-15)
    side = fc[np.arange(m.nfb), axis]
    sgn = nrm[np.arange(m.nfb), axis]
    assert np.all(((side > 0.5) & (sgn > 0)) | ((side < 0.5) & (sgn < 0)))


def test_boundary_orientation_independent_of_listing():
    m = meshgen.kuhn_cube(3, jitter=0.1, seed=5)
    nrm, ar, _ = oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
    flipped = m.faces[:, [0, 2, 1]].copy()
    nrm2, ar2, _ = oracle.boundary(3, m.nn, m.elems, m.coords, flipped)
    np.testing.assert_allclose(nrm2, nrm, atol=1e-15)
    np.testing.assert_allclose(ar2, ar, rtol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_boundary_matches_paper_normal_transform(dim):
    # the boundary normal equals the normalised facet normal V^{-T} normalsRef of the
    # owning simplex (Section 3.2 route), is orthogonal to the facet's edges, and
    # |det V| |n_j| / (dim-1)! is the facet measure; the mesh is moved by an affine
    # map so that no boundary facet is axis-aligned
    if dim == 3:
        m = meshgen.kuhn_cube(2, jitter=0.1, seed=2)
        Aff, shift = np.array([[1.0, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.1, 1.1]]), np.array([0.3, -0.2, 0.5])
    else:
        m = meshgen.make_mesh(2, 4, jitter=0.1, seed=2)
        Aff, shift = np.array([[1.0, 0.3], [-0.2, 0.8]]), np.array([0.3, -0.2])
    coords = m.coords @ Aff.T + shift
    nrm, ar, _ = oracle.boundary(dim, m.nn, m.elems, coords, m.faces)
    tn = oracle.simplex_normals(dim, m.elems, coords)
    _, det = oracle.volumes(dim, m.elems, coords)
    for f in range(m.nfb):
        fs = set(m.faces[f].tolist())
        owners = [k for k in range(m.ne) if fs <= set(m.elems[k].tolist())]
        assert len(owners) == 1
        k = owners[0]
        j = [q for q in range(dim + 1) if m.elems[k, q] not in fs][0]
        nj = tn[k, j]
        np.testing.assert_allclose(nj / np.linalg.norm(nj), nrm[f], atol=1e-13)
        assert abs(det[k]) * np.linalg.norm(nj) / math.factorial(dim - 1) == pytest.approx(ar[f], rel=1e-13)
        X = coords[m.faces[f]]
        assert np.all(np.abs((X[1:] - X[0]) @ nrm[f]) < 1e-13)


# ---------------------------------------------------------------------------
# stiffness / mass: invariants, patch test, stencil, moments
# ---------------------------------------------------------------------------

def _assembled_dense(m, ca=1.0, cb=0.0, ckind=0):
    out = oracle.assemble(m.dim, m.order, m.nn, m.elems, m.coords, ca, cb, ckind=ckind)
    K = oracle.to_dense(m.nn, out["row_ptr"], out["col_idx"], out["K"])
    M = oracle.to_dense(m.nn, out["row_ptr"], out["col_idx"], out["M"])
    return K, M, out


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_coefficient_kinds_closed_forms(dim, order):
    # the element coefficient is taken once at the vertex centroid x_c: kind 0
    # c = a + b |x_c|^2, kind 1 c = a exp(b sum_d x_c[d]) (Section 3.5.1's
    # e^{x1+x2+x3} with a = b = 1); each element page is c times the c = 1 page,
    # with x_c computed here from the vertex coordinates
    m = meshgen.make_mesh(dim, 3, order=order, jitter=0.1, seed=21)
    xc = m.coords[m.elems[:, :dim + 1]].mean(axis=1)
    one = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 1.0, 0.0, want_pages=True)
    a, b = 2.5, -0.7
    for kind, c in ((0, a + b * np.sum(xc ** 2, axis=1)), (1, a * np.exp(b * xc.sum(axis=1)))):
        out = oracle.assemble(dim, order, m.nn, m.elems, m.coords, a, b, want_pages=True, ckind=kind)
        np.testing.assert_allclose(out["K3D"], c[:, None, None] * one["K3D"], rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(out["M3D"], c[:, None, None] * one["M3D"], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("dim,order,n", [(2, 1, 6), (3, 1, 3), (2, 2, 4), (3, 2, 2)])
@pytest.mark.parametrize("cb", [0.0, 1.0])
def test_K_M_invariants(dim, order, n, cb):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=7)
    K, M, out = _assembled_dense(m, 1.0, cb)
    scale = np.abs(K).max()
    np.testing.assert_allclose(K, K.T, atol=1e-14 * scale)
    np.testing.assert_allclose(M, M.T, atol=1e-14 * np.abs(M).max())
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-13 * scale)       # constants in the kernel
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 * scale and abs(ev[0]) < 1e-12 * scale and ev[1] > 1e-6 * scale
    assert np.linalg.eigvalsh(M).min() > 0
    # 1^T M 1 = sum_k c_k vol_k
    _, _, vol, coef = oracle.element_pages(dim, order, m.elems, m.coords, 1.0, cb)
    assert M.sum() == pytest.approx(float((coef * vol).sum()), rel=1e-13)
    np.testing.assert_allclose(out["vol"], vol, rtol=0, atol=0)


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_linear_patch_test(dim, order):
    # u = a.x + b is reproduced exactly: (K u)_i = 0 at interior nodes for constant c,
    # u^T K u = |a|^2 sum_k c_k vol_k for any element-wise constant c
    m = meshgen.make_mesh(dim, 4, order=order, jitter=0.1, seed=3)
    a = np.array([0.7, -1.3, 0.4])[:dim]
    u = m.coords @ a + 0.25
    K, _, _ = _assembled_dense(m)
    Ku = K @ u
    x = m.coords
    interior = np.all((x > 1e-12) & (x < 1 - 1e-12), axis=1)
    np.testing.assert_allclose(Ku[interior], 0.0, atol=1e-12)
    K2, _, _ = _assembled_dense(m, 1.0, 1.0)
    _, _, vol, coef = oracle.element_pages(dim, order, m.elems, m.coords, 1.0, 1.0)
    assert u @ K2 @ u == pytest.approx(float(a @ a) * float((coef * vol).sum()), rel=1e-12)


def test_kuhn_stencil_unjittered():
    # P1 on the unjittered Kuhn mesh with c = 1: every interior row of K is the 7-point
    # Laplacian stencil times h (diag 6h, -h to the 6 axis neighbours, 0 to the other 8),
    # and every interior row of M sums to h^3
    n = 4
    h = 1.0 / n
    m = meshgen.kuhn_cube(n, jitter=0.0)
    out = oracle.assemble(3, 1, m.nn, m.elems, m.coords)
    rp, ci = out["row_ptr"], out["col_idx"]
    mm = n + 1
    checked = 0
    for node in range(m.nn):
        i, j, k = node % mm, (node // mm) % mm, node // (mm * mm)
        if not (0 < i < n and 0 < j < n and 0 < k < n):
            continue
        cols = ci[rp[node]:rp[node + 1]]
        kv = out["K"][rp[node]:rp[node + 1]]
        mv = out["M"][rp[node]:rp[node + 1]]
        assert len(cols) == 15
        axis_nb = {node + 1, node - 1, node + mm, node - mm, node + mm * mm, node - mm * mm}
        for c, v in zip(cols, kv):
            want = 6 * h if c == node else (-h if c in axis_nb else 0.0)
            assert v == pytest.approx(want, abs=1e-15)
        assert mv.sum() == pytest.approx(h ** 3, rel=1e-14)
        checked += 1
    assert checked == (n - 1) ** 3


@pytest.mark.parametrize("order", [1, 2])
def test_mass_moments(order):
    # x1 lies in the P1 and P2 spaces, so 1^T M x1 = int x1 = 1/2 and x1^T M x1 = 1/3 exactly
    m = meshgen.kuhn_cube(3, order=order, jitter=0.1, seed=9)
    _, M, _ = _assembled_dense(m)
    one = np.ones(m.nn)
    x1 = m.coords[:, 0]
    assert one @ M @ one == pytest.approx(1.0, abs=1e-14)
    assert one @ M @ x1 == pytest.approx(0.5, abs=1e-14)
    assert x1 @ M @ x1 == pytest.approx(1.0 / 3.0, abs=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_p2_quadratics_exact(dim):
    # P2 reproduces quadratics: u^T K u = int |grad u|^2, u^T M u = int u^2 (c = 1)
    m = meshgen.make_mesh(dim, 3, order=2, jitter=0.1, seed=4)
    K, M, _ = _assembled_dense(m)
    x = m.coords
    u = x[:, 0] ** 2
    assert u @ K @ u == pytest.approx(4.0 / 3.0, rel=1e-12)
    assert u @ M @ u == pytest.approx(1.0 / 5.0, rel=1e-12)
    w = x[:, 0] * x[:, 1]
    assert w @ K @ w == pytest.approx(2.0 / 3.0, rel=1e-12)
    assert w @ M @ w == pytest.approx(1.0 / 9.0, rel=1e-12)


# ---------------------------------------------------------------------------
# brute force: Lagrange bases from a Vandermonde solve and a collapsed
# Gauss-Legendre rule, dense assembly, on 1-2 cells
# ---------------------------------------------------------------------------

def _monomials(dim, order):
    exps = [e for e in np.ndindex(*([order + 1] * dim)) if sum(e) <= order]
    return [np.array(e) for e in exps]


def _simplex_rule(dim, npts=5):
    # collapsed (Duffy) tensor Gauss-Legendre rule on the unit simplex
    g, w = np.polynomial.legendre.leggauss(npts)
    g, w = 0.5 * (g + 1), 0.5 * w
    pts, wts = [], []
    if dim == 2:
        for a, wa in zip(g, w):
            for b, wb in zip(g, w):
                pts.append([a, b * (1 - a)])
                wts.append(wa * wb * (1 - a))
    else:
        for a, wa in zip(g, w):
            for b, wb in zip(g, w):
                for c, wc in zip(g, w):
                    pts.append([a, b * (1 - a), c * (1 - a) * (1 - b)])
                    wts.append(wa * wb * wc * (1 - a) ** 2 * (1 - b))
    return np.array(pts), np.array(wts)


def _brute_force(m, ca, cb):
    dim, order = m.dim, m.order
    mons = _monomials(dim, order)
    rp, rw = _simplex_rule(dim)
    K = np.zeros((m.nn, m.nn))
    M = np.zeros((m.nn, m.nn))
    for k in range(m.ne):
        nodes = m.coords[m.elems[k]]
        Vd = np.array([[np.prod(xn ** e) for e in mons] for xn in nodes])
        Cf = np.linalg.solve(Vd, np.eye(len(mons)))      # phi_j = sum_m Cf[m, j] x^e_m
        v0 = nodes[0]
        J = (nodes[1:dim + 1] - v0).T
        jac = abs(np.linalg.det(J))
        verts = nodes[:dim + 1]
        xc = verts.mean(axis=0)
        c = ca + cb * float(xc @ xc)
        for xi, wq in zip(rp, rw):
            x = v0 + J @ xi
            phi = np.array([np.prod(x ** e) for e in mons]) @ Cf
            grad = np.zeros((dim, len(mons)))
            for q, e in enumerate(mons):
                for d in range(dim):
                    if e[d] > 0:
                        e2 = e.copy()
                        e2[d] -= 1
                        grad[d, q] = e[d] * np.prod(x ** e2)
            gphi = grad @ Cf
            idx = m.elems[k]
            K[np.ix_(idx, idx)] += c * wq * jac * (gphi.T @ gphi)
            M[np.ix_(idx, idx)] += c * wq * jac * np.outer(phi, phi)
    return K, M


@pytest.mark.parametrize("dim,order,n", [(2, 1, 2), (3, 1, 1), (2, 2, 1), (3, 2, 1)])
def test_brute_force_dense_assembly(dim, order, n):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.0)
    # interior jitter is zero on 1-cell meshes; shear the mesh so elements are generic
    Aff = np.array([[1.0, 0.3, -0.2], [0.1, 1.2, 0.25], [-0.15, 0.05, 0.9]])[:dim, :dim]
    m.coords = np.ascontiguousarray(m.coords @ Aff.T)
    Kb, Mb = _brute_force(m, 1.3, 0.7)
    K, M, out = _assembled_dense(m, 1.3, 0.7)
    np.testing.assert_allclose(K, Kb, atol=1e-12 * np.abs(Kb).max())
    np.testing.assert_allclose(M, Mb, atol=1e-12 * np.abs(Mb).max())
    # pattern: exactly the pairs of nodes sharing an element
    pairs = {(int(a), int(b)) for e in m.elems for a in e for b in e}
    got = {(r, int(c)) for r in range(m.nn) for c in out["col_idx"][out["row_ptr"][r]:out["row_ptr"][r + 1]]}
    assert got == pairs


def test_brute_force_pages_jittered():
    m = meshgen.kuhn_cube(2, order=2, jitter=0.1, seed=1)
    sub = meshgen.Mesh(3, 2, 2, m.coords, m.elems[:5].copy(), m.faces, m.nn_vertices)
    Kb, Mb = _brute_force(sub, 0.5, 2.0)
    K3, M3, _, _ = oracle.element_pages(3, 2, sub.elems, sub.coords, 0.5, 2.0)
    for k in range(5):
        idx = sub.elems[k]
        Kk = np.zeros((m.nn, m.nn))
        Mk = np.zeros((m.nn, m.nn))
        Kk[np.ix_(idx, idx)] = K3[k].T
        Mk[np.ix_(idx, idx)] = M3[k].T
    K, M = np.zeros((m.nn, m.nn)), np.zeros((m.nn, m.nn))
    for k in range(5):
        idx = sub.elems[k]
        K[np.ix_(idx, idx)] += K3[k].T
        M[np.ix_(idx, idx)] += M3[k].T
    np.testing.assert_allclose(K, Kb, atol=1e-12 * np.abs(Kb).max())
    np.testing.assert_allclose(M, Mb, atol=1e-12 * np.abs(Mb).max())


def test_reference_tet_textbook_matrices():
    # reference tet: K = (1/6) G^T G with G = [[-1,1,0,0],[-1,0,1,0],[-1,0,0,1]],
    # M = (1/6)(1 + delta_ij)/20
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    K3, M3, vol, _ = oracle.element_pages(3, 1, np.array([[0, 1, 2, 3]], np.int32), x)
    G = np.array([[-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]], dtype=np.float64)
    np.testing.assert_allclose(K3[0].T, G.T @ G / 6.0, atol=1e-16)
    np.testing.assert_allclose(M3[0].T, (np.ones((4, 4)) + np.eye(4)) / 120.0, atol=1e-17)


# ---------------------------------------------------------------------------
# Section 3.5.1: convergence of the discrete quadratic forms to the printed
# closed-form I_K, I_M (coefficient exp(sum x) at the element centroid)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,ns", [(2, [8, 16, 32]), (3, [4, 8, 16])])
def test_quadratic_form_convergence(golden_dir, dim, ns):
    g = _golden(golden_dir, "quadratic_forms.json")[f"{dim}d"]
    eK, eM = [], []
    for n in ns:
        m = meshgen.make_mesh(dim, n, order=1, jitter=0.0)
        out = oracle.assemble(dim, 1, m.nn, m.elems, m.coords, 1.0, 1.0, ckind=1)
        x = m.coords
        if dim == 2:
            v = np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
        else:
            v = np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * np.cos(np.pi * x[:, 2])
        rows = np.repeat(np.arange(m.nn), np.diff(out["row_ptr"]))
        qk = float(np.sum(v[rows] * out["K"] * v[out["col_idx"]]))
        qm = float(np.sum(v[rows] * out["M"] * v[out["col_idx"]]))
        eK.append(abs(qk - g["I_K"]))
        eM.append(abs(qm - g["I_M"]))
    for a, b in zip(eK, eK[1:]):
        assert 3.0 < a / b < 5.0
    for a, b in zip(eM, eM[1:]):
        assert 3.0 < a / b < 5.0
    assert eK[-1] < 0.05 * g["I_K"] and eM[-1] < 0.05 * g["I_M"]


# ---------------------------------------------------------------------------
# facet list: the counts of the paper's normals table (Section 3.2) and
# brute-force incidence on a tiny mesh
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("level,n_all,n_bnd", [(1, 864, 192), (2, 6528, 768), (3, 50688, 3072)])
def test_facet_list_counts_match_printed_table(level, n_all, n_bnd):
    m = meshgen.kuhn_cube(2 ** (level + 1), jitter=0.0)   # level L: (2^(L+1))^3 cubes x 6 tets
    faces, owner, nbr, nb = oracle.facets(3, m.elems)
    assert (len(faces), nb) == (n_all, n_bnd)
    assert np.sum(nbr < 0) == nb


def test_facet_list_brute_force_tiny():
    m = meshgen.kuhn_cube(1)
    faces, owner, nbr, nb = oracle.facets(3, m.elems)
    # every facet's vertices are its owner's vertices without the opposite one
    for f, (k, j), p in zip(faces, owner, nbr):
        verts = [v for i, v in enumerate(m.elems[k]) if i != j]
        assert list(f) == verts
        if p >= 0:
            assert p > k and set(f) <= set(m.elems[p])
        else:   # a boundary facet of the unit cube lies in one of its faces
            X = m.coords[f]
            assert np.any(np.all(np.isclose(X, 0.0), axis=0) | np.all(np.isclose(X, 1.0), axis=0))
    # each element's 4 facets appear exactly once overall
    seen = {}
    for (k, j), p in zip(owner, nbr):
        seen[(k, j)] = True
    assert len(seen) == len(faces)
    # brute force pairing count: interior facets counted twice across elements
    triples = [tuple(sorted(v for i, v in enumerate(e) if i != j)) for e in m.elems for j in range(4)]
    assert len(set(triples)) == len(faces)


@pytest.mark.parametrize("dim,order,n", [(3, 1, 5), (3, 2, 3), (2, 1, 9), (2, 2, 6)])
def test_threaded_timing_entry_is_bit_identical(dim, order, n):
    # the CPU baseline's all-cores entry runs the pinned steps over element
    # ranges and row blocks; every value must equal the sequential assembly's
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=4)
    pat = oracle.csr_pattern(m.nn, m.elems)
    a = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 0.7, 1.3, pattern=pat)
    for nt in (1, 3, 7):
        b = oracle.assemble_threads(dim, order, m.nn, m.elems, m.coords, 0.7, 1.3, pattern=pat, nthreads=nt)
        for k in ("K", "M", "vol"):
            assert np.array_equal(a[k], b[k]), (k, nt)
