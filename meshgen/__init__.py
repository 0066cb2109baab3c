"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only *generates inputs*: structured simplicial meshes of the unit
square / unit cube (node coordinates, element connectivity, boundary facets),
P2 mid-edge node numbering, random page arrays and batch/serving request
mixes.  It holds none of the method's arithmetic (no Jacobians, volumes,
element matrices, sparsity patterns or normals), so neither the CUDA path nor
the oracle depends on the other through it.

Conventions (the paper's mesh data model, Section 3, "coords" and "elems"):
  * ``coords`` is ``nn x dim`` float64, C order, i.e. the ``dim x nn``
    column-major array of the C ABI (each node's coordinates contiguous).
  * ``elems`` is ``ne x nlb`` int32, C order, 0-based, i.e. the ``nlb x ne``
    column-major array of the C ABI (each element's node list contiguous).
  * boundary ``faces`` are ``nfb x dim`` int32 (triangles in 3-D, edges in 2-D),
    listed without any orientation guarantee.

Mesh recipes (readings of what the paper leaves unstated):
  * 3-D: an ``n x n x n`` grid of cubes, each split into 6 tetrahedra by the
    Kuhn/Freudenthal rule: for every permutation ``pi`` of the axes the tet
    ``(c, c+e_pi0, c+e_pi0+e_pi1, c+(1,1,1))``.  The same split in every cube
    makes the mesh conforming.  Node id ``i + (n+1) j + (n+1)^2 k``.
    With ``n = 2**(L+1)`` this reproduces the element/node/face counts of the
    paper's level-L meshes (Section 3.2, tables of volumes and normals).
  * 2-D: an ``n x n`` grid of squares, each split into two triangles along the
    (0,0)-(1,1) diagonal.  Node id ``i + (n+1) j``.
  * jitter: strictly interior nodes move by i.i.d. U(-jitter*h, +jitter*h) per
    coordinate (numpy PCG64 ``default_rng(seed)``); boundary nodes stay put.
  * P2: mid-edge nodes are numbered after the vertices in lexicographic order
    of their (sorted) vertex pair and placed at the midpoint of the jittered
    vertices, so the geometry stays affine.  Local order of the extra nodes:
    2-D (1,2),(2,3),(1,3); 3-D (1,2),(2,3),(1,3),(1,4),(2,4),(3,4)
    (1-based local vertex numbers).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "kuhn_cube", "unit_square", "make_mesh", "random_pages",
    "batch_specs", "serving_requests", "P2_EDGES_2D", "P2_EDGES_3D",
]

# local vertex pairs (0-based) of the P2 mid-edge nodes, in local order
P2_EDGES_2D = ((0, 1), (1, 2), (0, 2))
P2_EDGES_3D = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))

_PERMS = tuple(itertools.permutations(range(3)))  # lexicographic order


@dataclass
class Mesh:
    dim: int
    order: int            # 1 = P1, 2 = P2
    n: int                # cells per side
    coords: np.ndarray    # nn x dim float64
    elems: np.ndarray     # ne x nlb int32
    faces: np.ndarray     # nfb x dim int32 (boundary facets, vertex nodes)
    nn_vertices: int      # number of vertex (P1) nodes; P2 adds edge nodes after them
    meta: dict = field(default_factory=dict)

    @property
    def nn(self) -> int:
        return int(self.coords.shape[0])

    @property
    def ne(self) -> int:
        return int(self.elems.shape[0])

    @property
    def nlb(self) -> int:
        return int(self.elems.shape[1])

    @property
    def nfb(self) -> int:
        return int(self.faces.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / self.n


def _jitter(coords: np.ndarray, interior: np.ndarray, h: float, jitter: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.0, 1.0, size=coords.shape) * (jitter * h)
    d[~interior] = 0.0
    return coords + d


def _add_p2(coords: np.ndarray, elems: np.ndarray, edges_local) -> tuple[np.ndarray, np.ndarray]:
    nv = coords.shape[0]
    pairs = np.stack([np.sort(elems[:, [a, b]], axis=1) for a, b in edges_local], axis=1)  # ne x nE x 2
    flat = pairs.reshape(-1, 2).astype(np.int64)
    keys = flat[:, 0] * nv + flat[:, 1]
    uniq, inv = np.unique(keys, return_inverse=True)
    ea = (uniq // nv).astype(np.int64)
    eb = (uniq % nv).astype(np.int64)
    mid = 0.5 * (coords[ea] + coords[eb])
    new_coords = np.concatenate([coords, mid], axis=0)
    edge_nodes = (nv + inv).reshape(elems.shape[0], len(edges_local)).astype(np.int32)
    return new_coords, np.concatenate([elems, edge_nodes], axis=1).astype(np.int32)


def kuhn_cube(n: int, jitter: float = 0.1, seed: int = 0, order: int = 1) -> Mesh:
    """Unit cube, ``n^3`` cubes x 6 Kuhn tetrahedra (6 n^3 tets, (n+1)^3 vertices)."""
    if n < 1:
        raise ValueError("n >= 1")
    m = n + 1
    g = np.arange(m, dtype=np.float64) / n
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()          # node id = i + m j + m^2 k
    coords = np.stack([g[ii], g[jj], g[kk]], axis=1)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
    h = 1.0 / n
    if jitter:
        coords = _jitter(coords, interior[:, None].repeat(3, axis=1), h, jitter, seed)

    def nid(i, j, k):
        return i + m * j + m * m * k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cube order: x fastest
    ci, cj, ck = ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(), ck.transpose(2, 1, 0).ravel()
    tets = []
    for p in _PERMS:
        off = np.zeros(3, dtype=np.int64)
        verts = [nid(ci, cj, ck)]
        for ax in p:
            off[ax] += 1
            verts.append(nid(ci + off[0], cj + off[1], ck + off[2]))
        tets.append(np.stack(verts, axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)   # 6 tets per cube, cube-major

    # boundary triangles: every boundary square split along its low-low/high-high diagonal
    faces = []
    r = np.arange(n)
    A, B = np.meshgrid(r, r, indexing="ij")
    A, B = A.ravel(), B.ravel()
    for ax in range(3):
        ua, ub = [a for a in range(3) if a != ax]
        for side in (0, n):
            def node(da, db, A=A, B=B, ax=ax, ua=ua, ub=ub, side=side):
                idx = [None, None, None]
                idx[ax] = np.full_like(A, side)
                idx[ua] = A + da
                idx[ub] = B + db
                return nid(idx[0], idx[1], idx[2])
            p00, p10, p01, p11 = node(0, 0), node(1, 0), node(0, 1), node(1, 1)
            faces.append(np.stack([p00, p10, p11], axis=1))
            faces.append(np.stack([p00, p01, p11], axis=1))
    faces = np.concatenate(faces, axis=0).astype(np.int32)
    nv = coords.shape[0]
    if order == 2:
        coords, elems = _add_p2(coords, elems, P2_EDGES_3D)
    elif order != 1:
        raise ValueError("order must be 1 or 2")
    return Mesh(3, order, n, np.ascontiguousarray(coords), np.ascontiguousarray(elems),
                np.ascontiguousarray(faces), nv, {"kind": "kuhn_cube", "jitter": jitter, "seed": seed})


def unit_square(n: int, jitter: float = 0.1, seed: int = 0, order: int = 1) -> Mesh:
    """Unit square, ``n^2`` squares x 2 triangles (2 n^2 triangles, (n+1)^2 vertices)."""
    if n < 1:
        raise ValueError("n >= 1")
    m = n + 1
    g = np.arange(m, dtype=np.float64) / n
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()                           # node id = i + m j
    coords = np.stack([g[ii], g[jj]], axis=1)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n)
    h = 1.0 / n
    if jitter:
        coords = _jitter(coords, interior[:, None].repeat(2, axis=1), h, jitter, seed)
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    a = ci + m * cj
    b = a + 1
    c = a + 1 + m
    d = a + m
    elems = np.stack([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], axis=1).reshape(-1, 3).astype(np.int32)
    r = np.arange(n)
    edges = [np.stack([r, r + 1], 1),                              # y = 0
             np.stack([r + m * n, r + 1 + m * n], 1),              # y = 1
             np.stack([m * r, m * (r + 1)], 1),                    # x = 0
             np.stack([n + m * r, n + m * (r + 1)], 1)]            # x = 1
    faces = np.concatenate(edges, axis=0).astype(np.int32)
    nv = coords.shape[0]
    if order == 2:
        coords, elems = _add_p2(coords, elems, P2_EDGES_2D)
    elif order != 1:
        raise ValueError("order must be 1 or 2")
    return Mesh(2, order, n, np.ascontiguousarray(coords), np.ascontiguousarray(elems),
                np.ascontiguousarray(faces), nv, {"kind": "unit_square", "jitter": jitter, "seed": seed})


def make_mesh(dim: int, n: int, order: int = 1, jitter: float = 0.1, seed: int = 0) -> Mesh:
    return kuhn_cube(n, jitter, seed, order) if dim == 3 else unit_square(n, jitter, seed, order)


def random_pages(N: int, n: int, seed: int = 0, dtype=np.float64, m: int | None = None):
    """Page-array inputs for the primitive sweep.

    Returns a dict with ``A``, ``B`` (``N x m x n`` arrays whose entries are
    i.i.d. N(0,1), plus 3 on the diagonal), ``s`` (N scalars U(0.5, 2)) and
    ``v`` (``N x n`` vectors N(0,1)).  Arrays are C-ordered with the page index
    slowest; page ``k`` viewed as a column-major ``n x m`` matrix is
    ``A[k].T`` (i.e. ``A[k, c, r]`` holds entry (r, c)).
    """
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, m, n))
    B = rng.standard_normal((N, m, n))
    for r in range(min(m, n)):
        A[:, r, r] += 3.0
        B[:, r, r] += 3.0
    s = rng.uniform(0.5, 2.0, size=N)
    v = rng.standard_normal((N, n))
    return {k: np.ascontiguousarray(x.astype(dtype)) for k, x in (("A", A), ("B", B), ("s", s), ("v", v))}


def _structured_n(dim: int, order: int, target: float) -> int:
    # elements per mesh: 2 n^2 (triangles) or 6 n^3 (tets); P2 uses the same cell counts
    per = 2.0 if dim == 2 else 6.0
    n = max(1, int(round((target / per) ** (1.0 / dim))))
    return n


def batch_specs(count: int = 256, lo: float = 1e3, hi: float = 1e6, seed: int = 0):
    """Mesh mix of the batched uneven workload: an equal split of 2-D/3-D x P1/P2,
    element counts log-uniform in [lo, hi] rounded to the nearest structured n.
    Returns a list of dicts ``{dim, order, n, seed}``."""
    rng = np.random.default_rng(seed)
    specs = []
    kinds = [(2, 1), (2, 2), (3, 1), (3, 2)]
    for q in range(count):
        dim, order = kinds[q % 4]
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        specs.append({"dim": dim, "order": order, "n": _structured_n(dim, order, target),
                      "seed": int(rng.integers(0, 2**31 - 1))})
    return specs


def serving_requests(count: int = 10000, rate_per_s: float = 1000.0, lo: float = 1e3, hi: float = 2e6,
                     repeat_frac: float = 0.2, seed: int = 0, size_levels: int = 0):
    """Poisson arrival stream of assembly requests.  Each request names a mesh
    spec (as in :func:`batch_specs`); a ``repeat_frac`` share repeats an earlier
    mesh with a new coefficient ``c(x) = a + b |x|^2``, ``a, b ~ U(0.5, 2)``.
    ``size_levels`` > 0 snaps each drawn element count to a geometric ladder of
    that many levels per decade before choosing n (fewer distinct mesh sizes
    to generate; the draws themselves are unchanged)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    kinds = [(2, 1), (2, 2), (3, 1), (3, 2)]
    for q in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        a, b = rng.uniform(0.5, 2.0, size=2)
        if reqs and rng.uniform() < repeat_frac:
            src = reqs[int(rng.integers(0, len(reqs)))]
            spec = dict(src["mesh"])
        else:
            dim, order = kinds[int(rng.integers(0, 4))]
            target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
            if size_levels > 0:
                target = 10.0 ** (round(math.log10(target) * size_levels) / size_levels)
            spec = {"dim": dim, "order": order, "n": _structured_n(dim, order, target),
                    "seed": int(rng.integers(0, 2**31 - 1))}
        reqs.append({"id": q, "t_arrival": t, "mesh": spec, "coeff": (float(a), float(b))})
    return reqs
