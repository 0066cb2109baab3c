"""The seeded input generators hold the recipes stated for the workloads:
counts, jitter only on interior nodes and within its bound, P2 mid-edge nodes
at the midpoints in the documented local order, conforming meshes (every
interior facet shared by exactly two elements), the page-array distribution,
and the batch and serving mixes (type split, arrival rate, repeat share,
coefficient range).  Plain numpy; no oracle or library call."""
import math
from collections import Counter
from itertools import combinations

import numpy as np
import pytest

import meshgen


def _facet_multiplicities(elems, dim):
    c = Counter()
    for e in elems[:, : dim + 1]:
        for f in combinations(sorted(e.tolist()), dim):
            c[f] += 1
    return c


@pytest.mark.parametrize("dim,n", [(2, 1), (2, 5), (3, 1), (3, 3)])
def test_counts_conformity_and_boundary(dim, n):
    m = meshgen.make_mesh(dim, n, jitter=0.1, seed=3)
    if dim == 3:
        assert (m.ne, m.nn, m.nfb) == (6 * n ** 3, (n + 1) ** 3, 12 * n * n)
    else:
        assert (m.ne, m.nn, m.nfb) == (2 * n * n, (n + 1) ** 2, 4 * n)
    mult = _facet_multiplicities(m.elems, dim)
    assert set(mult.values()) <= {1, 2}
    boundary = {f for f, k in mult.items() if k == 1}
    assert boundary == {tuple(sorted(f.tolist())) for f in m.faces}
    X = m.coords[m.faces]                                   # every boundary facet lies in a face of the box
    assert np.all(np.any(np.all(np.isclose(X, 0.0), axis=1) | np.all(np.isclose(X, 1.0), axis=1), axis=1))


@pytest.mark.parametrize("dim", [2, 3])
def test_jitter_moves_interior_nodes_only_within_the_bound(dim):
    n = 6
    h = 1.0 / n
    m0 = meshgen.make_mesh(dim, n, jitter=0.0)
    m1 = meshgen.make_mesh(dim, n, jitter=0.1, seed=7)
    d = np.abs(m1.coords - m0.coords)
    on_boundary = np.any(np.isclose(m0.coords, 0.0) | np.isclose(m0.coords, 1.0), axis=1)
    assert np.all(d[on_boundary] == 0.0)
    assert np.all(d[~on_boundary] <= 0.1 * h + 1e-15)
    assert d[~on_boundary].max() > 0.05 * h                  # it does move them
    np.testing.assert_array_equal(m1.coords, meshgen.make_mesh(dim, n, jitter=0.1, seed=7).coords)


@pytest.mark.parametrize("dim", [2, 3])
def test_p2_nodes_at_edge_midpoints_in_local_order(dim):
    m = meshgen.make_mesh(dim, 3, order=2, jitter=0.1, seed=5)
    edges = [(0, 1), (1, 2), (0, 2)] if dim == 2 else [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    assert m.elems.shape[1] == dim + 1 + len(edges)
    nv = len(np.unique(m.elems[:, : dim + 1]))
    for q, (a, b) in enumerate(edges):
        mid = m.elems[:, dim + 1 + q]
        assert np.all(mid >= nv)                             # numbered after the vertices
        np.testing.assert_array_equal(m.coords[mid], 0.5 * (m.coords[m.elems[:, a]] + m.coords[m.elems[:, b]]))
    # one node per geometric edge: elements sharing an edge share its node
    seen = {}
    for e in m.elems:
        for q, (a, b) in enumerate(edges):
            key = tuple(sorted((int(e[a]), int(e[b]))))
            assert seen.setdefault(key, int(e[dim + 1 + q])) == int(e[dim + 1 + q])


def test_random_pages_distribution():
    P = meshgen.random_pages(20000, 3, seed=1)
    A = P["A"]
    assert A.shape == (20000, 3, 3) and P["v"].shape == (20000, 3)
    diag = A[:, [0, 1, 2], [0, 1, 2]]
    off = A[:, [0, 1], [1, 2]]
    assert abs(diag.mean() - 3.0) < 0.03 and abs(off.mean()) < 0.03 and abs(off.std() - 1.0) < 0.03
    assert P["s"].min() >= 0.5 and P["s"].max() <= 2.0


def test_batch_mix():
    specs = meshgen.batch_specs(256, 1e3, 1e6, seed=0)
    kinds = Counter((s["dim"], s["order"]) for s in specs)
    assert kinds == {(2, 1): 64, (2, 2): 64, (3, 1): 64, (3, 2): 64}
    ne = np.array([2 * s["n"] ** 2 if s["dim"] == 2 else 6 * s["n"] ** 3 for s in specs], dtype=float)
    assert ne.min() >= 0.5e3 and ne.max() <= 2e6
    # log-uniform draws: the log element counts spread over the whole range
    q = np.quantile(np.log10(ne), [0.25, 0.5, 0.75])
    assert 3.3 < q[0] < 4.2 and 4.1 < q[1] < 4.9 and 4.8 < q[2] < 5.7


def test_serving_stream():
    reqs = meshgen.serving_requests(10000, rate_per_s=500.0, seed=0, size_levels=16)
    t = np.array([r["t_arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() - 1.0 / 500.0) < 0.05 / 500.0        # exponential gaps, mean 1/rate
    assert abs(np.diff(t).std() / np.diff(t).mean() - 1.0) < 0.05    # coefficient of variation 1
    ab = np.array([r["coeff"] for r in reqs])
    assert ab.min() >= 0.5 and ab.max() <= 2.0
    # a repeat names an earlier request's mesh; about 20 % of the requests repeat
    first = {}
    repeats = 0
    for r in reqs:
        key = tuple(sorted(r["mesh"].items()))
        if key in first:
            repeats += 1
        else:
            first[key] = r["id"]
    assert abs(repeats / len(reqs) - 0.2) < 0.02
    kinds = Counter((r["mesh"]["dim"], r["mesh"]["order"]) for r in reqs)
    assert all(abs(v / len(reqs) - 0.25) < 0.03 for v in kinds.values())
    assert math.isclose(sum(kinds.values()), len(reqs))
