"""Pins of the oracle's amt, avtav, amsm, amsv, smamt and svamt (Section 2.4)
to facts outside it: the normals the paper prints for its worked tetrahedron
(normals3D = amsm(amt(vectors3D_inv), normalsRef), Section 3.2), the printed
determinant through the transposed Jacobian smamt(dshape, coords3D)
(Section 3.5), numpy contractions on random pages, and identities between
independent oracle paths.  Page arrays are numpy (N, cols, rows): a page
r x c is stored column by column."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _pages(M):          # one matrix -> a one-page array
    return np.ascontiguousarray(np.asarray(M, dtype=np.float64).T[None])


def _matrix(P):         # page 0 of a page array -> the matrix
    return P[0].T


def test_worked_tetrahedron_normals_by_amsm_amt(golden_dir):
    g = _golden(golden_dir, "worked_tet.json")
    V = np.array(g["vectors3D_times_4"], dtype=np.float64) / 4.0
    Vinv = _matrix(oracle.aminv(_pages(V))[0])
    VinvT = _matrix(oracle.amt(_pages(Vinv)))
    np.testing.assert_allclose(VinvT, np.linalg.inv(V).T, rtol=0, atol=1e-15)
    R = np.array(g["normalsRef"], dtype=np.float64)          # 3 x 4
    N = _matrix(oracle.amsm(_pages(VinvT), R.T.copy()))       # S passed column by column
    expect = np.array([[float(Fraction(x)) for x in row] for row in g["normals3D"]])
    np.testing.assert_allclose(N, expect, rtol=0, atol=1e-14)


def test_worked_tetrahedron_jacobian_by_smamt(golden_dir):
    # tjac = smamt(dshape, coords3D): the reference gradients of the P1 basis
    # times the transposed vertex coordinates; its rows are the edge vectors
    # from vertex 0 and |det| = 6 |T| with |T| the printed volume 25/64
    g = _golden(golden_dir, "worked_tet.json")
    X = np.array(g["nodes_times_4"], dtype=np.float64) / 4.0   # 4 vertices x 3
    dshape = np.array([[-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]], dtype=np.float64)   # 3 x 4
    coords3D = X.T                                              # 3 x 4 page (column j = vertex j)
    tjac = _matrix(oracle.smamt(dshape.T.copy(), _pages(coords3D)))
    np.testing.assert_allclose(tjac, X[1:] - X[0], rtol=0, atol=1e-15)
    num, den = g["det_over_6"]
    assert abs(oracle.amdet(_pages(tjac))[0]) == pytest.approx(6 * abs(num / den), abs=1e-14)


@pytest.mark.parametrize("m,p,n", [(2, 2, 2), (3, 3, 3), (3, 4, 5), (1, 10, 8), (4, 1, 3)])
def test_amsm_smamt_against_numpy(m, p, n):
    rng = np.random.default_rng(m * 100 + p * 10 + n)
    N = 37
    A = rng.standard_normal((N, p, m))            # pages m x p
    S = rng.standard_normal((n, p))               # the p x n matrix, column by column
    C = oracle.amsm(A, S)
    Am = np.transpose(A, (0, 2, 1))               # (N, m, p) as matrices
    Sm = S.T                                      # p x n
    np.testing.assert_allclose(np.transpose(C, (0, 2, 1)), Am @ Sm, rtol=1e-14, atol=1e-14)
    # smamt(S', B) = S' B_k^T with S' m x p and pages n x p
    Sp = rng.standard_normal((p, m))              # the m x p matrix, column by column
    B = rng.standard_normal((N, p, n))            # pages n x p
    D = oracle.smamt(Sp, B)
    np.testing.assert_allclose(np.transpose(D, (0, 2, 1)), Sp.T @ np.transpose(B, (0, 1, 2)),
                               rtol=1e-14, atol=1e-14)


def test_identities_between_oracle_paths():
    rng = np.random.default_rng(5)
    N, m, p, n = 23, 3, 4, 2
    A = rng.standard_normal((N, p, m))            # pages m x p
    S = rng.standard_normal((n, p))               # p x n
    # amt is an involution
    np.testing.assert_array_equal(oracle.amt(oracle.amt(A)), A)
    # amsm(A, S) = amtam(amt(A), S copied to every page)
    Sc = np.broadcast_to(S, (N, n, p)).copy()
    np.testing.assert_allclose(oracle.amsm(A, S), oracle.amtam(oracle.amt(A), Sc), rtol=1e-14, atol=1e-15)
    # smamt(S, B) = amt(amsm(B, S^T)) for S m x p, B pages n x p
    Sp = rng.standard_normal((p, m))
    B = rng.standard_normal((N, p, n))
    lhs = oracle.smamt(Sp, B)
    rhs = oracle.amt(oracle.amsm(B, np.ascontiguousarray(Sp.T)))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-14, atol=1e-15)
    # amsv(A, s) = amsm with one column = svamt(s, A) (the same values as a row)
    s = rng.standard_normal(p)
    y = oracle.amsv(A, s)
    np.testing.assert_allclose(y, oracle.amsm(A, s[None, :])[:, 0, :], rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(oracle.svamt(s, A), y)
    # avtav: a.a = |a|^2, orthogonal pairs give 0, and it is avtamav with the identity
    a = rng.standard_normal((N, 3))
    np.testing.assert_allclose(oracle.avtav(a, a), np.sum(a * a, axis=1), rtol=1e-15)
    e1 = np.tile([1.0, 0.0, 0.0], (N, 1))
    e2 = np.tile([0.0, 1.0, 0.0], (N, 1))
    np.testing.assert_array_equal(oracle.avtav(e1, e2), np.zeros(N))
    b = rng.standard_normal((N, 3))
    Id = np.broadcast_to(np.eye(3), (N, 3, 3)).copy()
    np.testing.assert_allclose(oracle.avtav(a, b), oracle.avtamav(a, Id, b), rtol=1e-14, atol=1e-15)
