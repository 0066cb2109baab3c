"""Per-element error bounds of the mixed-precision (FP32) P1 element path.

Test helper, not a test module.  It states, for every element, how far the
mixed-precision element matrices K_k, M_k and the volume may lie from the exact
(FP64) values, following the operation sequence of the kernels' geometry and
element-matrix code step by step (a first-order running error analysis with
u = 2^-24; second-order terms are covered by a 1 % margin).

Quantities of the exact geometry (vectors3D of Section 3.2, last-node
convention): V_j = x_j - x_d, cofactor vectors C_j (rows of adj V; C_0 =
V_1 x V_2 in 3-D), det = V_0 . C_0, the permanent perm of |V|, the 2x2
permanents pm_jc of the minors behind C_jc, Q = sum_jc |V_jc| |C_jc| and
r = perm / |det| (the guard of the fast path compares |det| with perm / 4).

Fast path (plain FP32, taken when |det| >= perm / 4):
  edge vectors     |dV_jc| <= eta_jc = 2u |V_jc| + 4u^2 X   (X = max |x|)
  cofactors        |dC_jc| <= (the eta-perturbation of the 2x2 minor) + 2u pm_jc
  det (3-D)        |d det| <= sum_jc eta_jc |C_jc| + 5u perm     (<= 11u perm)
  det (2-D, Kahan) |d det| <= sum eta |C| + 2u |det|
Float-pair path (taken when |det| < perm / 4): the edge vectors are exact to
O(u^2) and det is compensated, so |d det| <= 2u |det| + 64 u^2 perm (+ X terms);
its cofactors are within 4u pm_jc, below the fast-path figure.
Element matrices: s = c / (dim! |det|); K_ab = s (C_a . C_b) for a, b < d, the
last row and column from the zero row sums; M_k = c |det| / dim! (1 + delta) /
((d+1)(d+2)); vol = |det| / dim!.  Relative error of s: theta_det + theta_c +
3u; of M: theta_det + theta_c + 3u; of vol: theta_det + 2u.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -24
MARGIN = 1.01


def _geometry(dim, coords, elems):
    x = coords[elems[:, :dim + 1]]                       # ne x (d+1) x dim
    V = x[:, :dim, :] - x[:, dim:dim + 1, :]             # rows V_j = x_j - x_d
    A = np.abs(V)
    X = np.abs(x).max(axis=(1, 2))
    if dim == 3:
        C = np.stack([np.cross(V[:, 1], V[:, 2]), np.cross(V[:, 2], V[:, 0]), np.cross(V[:, 0], V[:, 1])], axis=1)
        pm = np.empty_like(C)
        for j, (p, q) in enumerate(((1, 2), (2, 0), (0, 1))):
            for c in range(3):
                c1, c2 = (c + 1) % 3, (c + 2) % 3
                t1 = A[:, p, c1] * A[:, q, c2]
                t2 = A[:, p, c2] * A[:, q, c1]
                pm[:, j, c] = t1 + t2
        det = np.einsum("ec,ec->e", V[:, 0], C[:, 0])
        perm = np.einsum("ec,ec->e", A[:, 0], pm[:, 0])
    else:
        C = np.stack([np.stack([V[:, 1, 1], -V[:, 1, 0]], -1), np.stack([-V[:, 0, 1], V[:, 0, 0]], -1)], axis=1)
        pm = np.abs(C)                                   # each 2-D cofactor is one entry of V
        det = V[:, 0, 0] * V[:, 1, 1] - V[:, 0, 1] * V[:, 1, 0]
        perm = A[:, 0, 0] * A[:, 1, 1] + A[:, 0, 1] * A[:, 1, 0]
    return x, V, A, C, pm, det, perm, X


def p1_bounds(dim, coords, elems, ca, cb):
    """Exact element quantities and the bounds of the mixed path (coefficient
    c = ca + cb |x_c|^2 at the vertex centroid).  Returns a dict of arrays:
    r, det, vol, K (ne x nlb x nlb exact), K_bound (entrywise absolute),
    the masks fast / slow of the elements that certainly take each path, and
    the relative bounds theta_vol, theta_M (for the path each element takes),
    theta_vol_fast (fast path) and theta_det_exact (float-pair path)."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    x, V, A, C, pm, det, perm, X = _geometry(dim, coords, elems)
    ne, nv = len(elems), dim + 1
    eta = 2 * U * A + 4 * U * U * X[:, None, None]
    adet = np.abs(det)
    r = perm / adet
    # cofactor bounds (fast path; the float-pair path is below them)
    if dim == 3:
        EC = np.empty_like(C)
        for j, (p, q) in enumerate(((1, 2), (2, 0), (0, 1))):
            for c in range(3):
                c1, c2 = (c + 1) % 3, (c + 2) % 3
                pert = (eta[:, p, c1] * A[:, q, c2] + eta[:, q, c2] * A[:, p, c1] +
                        eta[:, p, c2] * A[:, q, c1] + eta[:, q, c1] * A[:, p, c2])
                EC[:, j, c] = pert + 2 * U * pm[:, j, c]
        d_fast = np.einsum("ejc,ejc->e", eta, np.abs(C)) + 5 * U * perm
    else:
        EC = np.stack([np.stack([eta[:, 1, 1], eta[:, 1, 0]], -1), np.stack([eta[:, 0, 1], eta[:, 0, 0]], -1)], 1)
        d_fast = np.einsum("ejc,ejc->e", eta, np.abs(C)) + 2 * U * adet
    d_exact = 2 * U * adet + 64 * U * U * perm + 8 * U * U * X * np.abs(C).sum(axis=(1, 2))
    th_det_fast = MARGIN * d_fast / adet
    th_det_exact = MARGIN * d_exact / adet
    # coefficient at the centroid from the float heads of the coordinates
    xc = x.mean(axis=1)
    ex = 2 * U * np.abs(x).sum(axis=1)                   # |dx_c,i|
    r2 = (xc * xc).sum(axis=1)
    c = ca + cb * r2
    dc = abs(cb) * ((2 * np.abs(xc) * ex).sum(axis=1) + 3 * U * r2) + 2 * U * (abs(ca) + abs(cb) * r2)
    th_c = MARGIN * dc / np.abs(c)
    fact = 6.0 if dim == 3 else 2.0
    vol = adet / fact
    s = c / (fact * adet)
    # the path each element takes: fast below r = 4 (computed r within ~1e-6 of the exact)
    fast = r < 4.0 * (1 - 1e-4)
    slow = r > 4.0 * (1 + 1e-4)
    th_det = np.where(fast, th_det_fast, np.where(slow, th_det_exact, np.maximum(th_det_fast, th_det_exact)))
    th_s = th_det + th_c + 3 * U
    # K entries: a, b < d by a dot product, the last row/column from row sums
    K = np.zeros((ne, nv, nv))
    EK = np.zeros((ne, nv, nv))
    d = dim
    for a in range(d):
        for b in range(d):
            N = np.einsum("ec,ec->e", C[:, a], C[:, b])
            EN = (np.einsum("ec,ec->e", EC[:, a], np.abs(C[:, b])) + np.einsum("ec,ec->e", np.abs(C[:, a]), EC[:, b])
                  + dim * U * np.einsum("ec,ec->e", np.abs(C[:, a]), np.abs(C[:, b])))
            K[:, a, b] = s * N
            EK[:, a, b] = MARGIN * (np.abs(s) * EN + np.abs(K[:, a, b]) * (th_s + U))
    for a in range(d):
        K[:, a, d] = -K[:, a, :d].sum(axis=1)
        EK[:, a, d] = EK[:, a, :d].sum(axis=1) + 2 * U * np.abs(K[:, a, :d]).sum(axis=1)
        K[:, d, a] = K[:, a, d]
        EK[:, d, a] = EK[:, a, d]
    K[:, d, d] = -K[:, :d, d].sum(axis=1)
    EK[:, d, d] = EK[:, :d, d].sum(axis=1) + 2 * U * np.abs(K[:, :d, d]).sum(axis=1)
    return {"r": r, "det": det, "vol": vol, "K": K, "K_bound": MARGIN * EK, "fast": fast, "slow": slow,
            "theta_vol": th_det + 2 * U, "theta_M": th_det + th_c + 3 * U,
            "theta_vol_fast": th_det_fast + 2 * U, "theta_det_exact": th_det_exact}


def band_simplices(dim, n, seed=0, base=(37.0, -11.0, 5.0), h=1.0 / 64):
    """n disjoint simplices whose ratio |det| / perm(|V|) spreads from about 1
    down to about 1/200: a randomly rotated and stretched reference simplex of
    size h near `base`, one vertex pulled towards the opposite facet by a
    log-uniform factor.  Returns (coords nn x dim, elems n x (dim+1))."""
    rng = np.random.default_rng(seed)
    coords, elems = [], []
    for k in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
        S = np.diag(rng.uniform(0.7, 1.4, dim))
        P = np.vstack([np.zeros(dim), np.eye(dim)]) @ (S @ Q).T * h
        t = 10 ** rng.uniform(-2.6, 0.0)
        j = rng.integers(dim + 1)                        # the vertex pulled towards its facet
        others = [i for i in range(dim + 1) if i != j]
        ctr = P[others].mean(axis=0)
        P[j] = ctr + t * (P[j] - ctr)
        P = P + np.asarray(base[:dim]) + rng.uniform(-1, 1, dim)
        coords.extend(P)
        elems.append(list(range((dim + 1) * k, (dim + 1) * (k + 1))))
    return np.array(coords), np.array(elems, dtype=np.int32)


# ---------------------------------------------------------------------------
# A step-by-step FP32 emulation of the fast path (numpy float32, one rounding
# per operation; a fused multiply-add is formed in float64, exact for float32
# products, and rounded once).  It lets a CPU test check the bounds above
# against the same operation sequence the kernels run.
# ---------------------------------------------------------------------------

def _f(x):
    return np.asarray(x, dtype=np.float32)


def _fma(a, b, c):
    return _f(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def emulate_fast_p1(dim, coords, elems, ca, cb):
    """K pages (ne x nlb x nlb), volumes and the M off-diagonal scale as the
    fast path computes them, and a mask of the elements the guard keeps on it."""
    coords = np.asarray(coords, dtype=np.float64)
    h = _f(coords)
    lo = _f(coords - h.astype(np.float64))
    xh, xl = h[elems[:, :dim + 1]], lo[elems[:, :dim + 1]]
    d = dim
    V = _f(_f(xh[:, :d] - xh[:, d:d + 1]) + _f(xl[:, :d] - xl[:, d:d + 1]))
    ne = len(elems)
    C = np.zeros((ne, d, 3), dtype=np.float32)
    if dim == 3:
        perm = np.zeros(ne, dtype=np.float32)
        for c in range(3):
            c1, c2 = (c + 1) % 3, (c + 2) % 3
            p12 = _f(V[:, 1, c2] * V[:, 2, c1])
            p20 = _f(V[:, 2, c2] * V[:, 0, c1])
            p01 = _f(V[:, 0, c2] * V[:, 1, c1])
            C[:, 0, c] = _fma(V[:, 1, c1], V[:, 2, c2], -p12)
            C[:, 1, c] = _fma(V[:, 2, c1], V[:, 0, c2], -p20)
            C[:, 2, c] = _fma(V[:, 0, c1], V[:, 1, c2], -p01)
            perm = _fma(np.abs(V[:, 0, c]), _f(np.abs(_f(V[:, 1, c1] * V[:, 2, c2])) + np.abs(p12)), perm)
        det = _fma(V[:, 0, 0], C[:, 0, 0], _fma(V[:, 0, 1], C[:, 0, 1], _f(V[:, 0, 2] * C[:, 0, 2])))
        sx = xh[:, 3]
        for j in range(3):
            sx = _f(sx + xh[:, j])
        xc = _f(sx * np.float32(0.25))
        fast = np.abs(det) >= _f(np.float32(0.25) * perm)
    else:
        V00, V01, V10, V11 = V[:, 0, 0], V[:, 0, 1], V[:, 1, 0], V[:, 1, 1]
        C[:, 0, 0], C[:, 0, 1], C[:, 1, 0], C[:, 1, 1] = V11, -V10, -V01, V00
        w = _f(V01 * V10)
        e = _fma(-V01, V10, w)
        det = _f(_fma(V00, V11, -w) + e)
        xc = _f(_f(_f(xh[:, 0] + xh[:, 1]) + xh[:, 2]) * np.float32(1.0 / 3.0))
        fast = np.abs(det) >= _f(np.float32(0.25) * _f(np.abs(_f(V00 * V11)) + np.abs(_f(V01 * V10))))
    r2 = _f(xc[:, 0] * xc[:, 0])
    for i in range(1, dim):
        r2 = _fma(xc[:, i], xc[:, i], r2)
    cf = _fma(np.full(ne, cb, np.float32), r2, np.full(ne, ca, np.float32))
    adet = np.abs(det)
    fact = np.float32(6.0 if dim == 3 else 2.0)
    rcp = _f(1.0 / _f(fact * adet).astype(np.float64))
    sc = _f(cf * rcp)
    nv = d + 1
    K = np.zeros((ne, nv, nv), dtype=np.float32)
    for a in range(d):
        for b in range(a, d):
            t = _f(C[:, a, 0] * C[:, b, 0])
            t = _fma(C[:, a, 1], C[:, b, 1], t)
            t = _fma(C[:, a, 2], C[:, b, 2], t)
            K[:, a, b] = K[:, b, a] = _f(sc * t)
    for a in range(d):
        s = K[:, a, 0]
        for b in range(1, d):
            s = _f(s + K[:, a, b])
        K[:, a, d] = K[:, d, a] = -s
    s = K[:, 0, d]
    for a in range(1, d):
        s = _f(s + K[:, a, d])
    K[:, d, d] = -s
    moff = np.float32(1.0 / ((d + 1) * (d + 2)) / float(fact))
    mscale = _f(_f(cf * adet) * moff)
    vol = _f(adet * np.float32(1.0 / float(fact)))
    return {"K": K.astype(np.float64), "mscale": mscale.astype(np.float64), "vol": vol.astype(np.float64),
            "fast": fast}
