"""GPU edge cases: single-element meshes of every type through every entry
point, isolated nodes, empty reductions, degenerate elements in batches, and
the documented size limits (rejected before any work)."""
import ctypes as C

import numpy as np
import pytest
import torch

import meshgen
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MIX = 1e-5


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _single(dim, order):
    """One reference simplex (scaled, shifted), P2 mid-edge nodes appended."""
    if dim == 2:
        X = np.array([[0.1, 0.2], [1.3, 0.25], [0.4, 1.1]])
        edges = [(0, 1), (1, 2), (0, 2)]
    else:
        X = np.array([[0.1, 0.2, 0.3], [1.3, 0.25, 0.35], [0.4, 1.1, 0.3], [0.2, 0.3, 1.4]])
        edges = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    el = list(range(dim + 1))
    if order == 2:
        for a, b in edges:
            X = np.vstack([X, 0.5 * (X[a] + X[b])])
            el.append(len(X) - 1)
    return X, np.array([el], dtype=np.int32)


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_single_element_everywhere(vla, dim, order):
    X, E = _single(dim, order)
    # an isolated node at the end: an empty CSR row, a zero load
    X = np.vstack([X, np.full((1, dim), 7.0)])
    gm = vla.Mesh(_dev(X), _dev(E), order=order)
    ref = oracle.assemble(dim, order, len(X), E, X, 1.1, 0.3, want_pages=True)
    for prec, tol in ((vla.PREC_FP64, TOL64), (vla.PREC_MIXED, TOL_MIX)):
        out = gm.assemble(1.1, 0.3, precision=prec, pages=True)
        for key in ("K", "M", "vol", "K3D", "M3D"):
            got = out[key].cpu().numpy()
            assert np.linalg.norm(got - ref[key]) <= tol * np.linalg.norm(ref[key]), (prec, key)
    rp, ci = gm.csr()
    assert rp[-1].item() == rp[-2].item()          # the isolated node's row is empty
    faces, owner, nbr, nb = gm.facets()
    assert faces.shape[0] == nb == dim + 1 and bool((nbr < 0).all())
    ip, w = vla.quad_rule(dim, 2)
    b, b2D = gm.rhs(2, torch.ones((1, len(w)), dtype=torch.float64, device="cuda"))
    assert b[-1].item() == 0.0
    vol = ref["vol"][0]
    assert b.sum().item() == pytest.approx(vol, rel=1e-13)
    pg = gm.assemble(1.0, 0.0, precision=vla.PREC_FP64, pages=True)
    u = torch.from_numpy(X[:, 0].copy()).cuda()
    _, tot = gm.energies(u, pg["K3D"], pg["M3D"], b2D)
    Jr = oracle.energies(E, X[:, 0], pg["K3D"].cpu().numpy(), pg["M3D"].cpu().numpy(), b2D.cpu().numpy())
    np.testing.assert_allclose(tot.cpu().numpy(), Jr.sum(axis=0), rtol=1e-12, atol=1e-15)


def test_batch_of_single_elements_and_flat_ones(vla):
    meshes = []
    for dim, order in ((2, 1), (2, 2), (3, 1), (3, 2)):
        X, E = _single(dim, order)
        meshes.append(vla.Mesh(_dev(X), _dev(E), order=order))
    # a flat tetrahedron (all four vertices in one plane): det 0, counted per job
    Xf = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.float64)
    flat = vla.Mesh(_dev(Xf), _dev(np.array([[0, 1, 2, 3]], np.int32)))
    jobs = [(g, g.outputs(), vla.COEFF_POLY, 1.0, 0.5) for g in meshes] + [(flat, flat.outputs(), 0, 1.0, 0.0)]
    for form in ("fused", "split"):
        b = vla.Batch(jobs, precision=vla.PREC_FP64, count_singular=True, form=form)
        b.run()
        torch.cuda.synchronize()
        assert b.n_singular.cpu().tolist() == [0, 0, 0, 0, 1]
        for g, o, *_ in jobs[:4]:
            ref = g.assemble(1.0, 0.5, precision=vla.PREC_FP64)
            assert torch.equal(o["K"], ref["K"]) and torch.equal(o["M"], ref["M"])
        assert flat.outputs is not None and b.outs[4]["vol"][0].item() == 0.0
        b.close()


def test_server_single_element_request(vla):
    X, E = _single(3, 2)
    srv = vla.Server(1 << 28)
    try:
        t = srv.submit(X, E, order=2, key=5, ca=1.0, cb=0.0)
        res = srv.poll(t, timeout=60.0)
        assert res is not None and res.status == 0 and res.ne == 1
        got = srv.result(t, res)
        ref = oracle.assemble(3, 2, len(X), E, X, 1.0, 0.0)
        assert np.linalg.norm(got["K"].cpu().numpy() - ref["K"]) <= TOL_MIX * np.linalg.norm(ref["K"])
        srv.release(t)
    finally:
        srv.close()


def test_empty_reductions_and_batches(vla):
    sizes = torch.empty(0, dtype=torch.float64, device="cuda")
    fip = torch.empty((0, 1, 2), dtype=torch.float64, device="cuda")
    assert vla.gi(fip, [1.0], sizes).cpu().tolist() == [0.0, 0.0]
    with pytest.raises(ValueError):
        vla.Batch([])
    out = vla.amtam(torch.empty((0, 3, 3), device="cuda"), torch.empty((0, 3, 3), device="cuda"))
    assert out.shape == (0, 3, 3)


def test_row_length_limit(vla):
    # a fan: one centre node in 300 triangles has a CSR row of 302 entries (> 255)
    n = 300
    ang = np.linspace(0.0, 2 * np.pi, n + 1)[:-1]
    X = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
    E = np.array([[0, 1 + i, 1 + (i + 1) % n] for i in range(n)], dtype=np.int32)
    with pytest.raises(vla.VlaError) as e:
        vla.Mesh(_dev(X), _dev(E))
    assert e.value.status == -8


def test_element_count_limit_rejected_before_work(vla):
    # ne >= 2^27 is refused from the sizes alone (the arrays are never read)
    L = vla.lib()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    h = C.c_void_p()
    st = L.vla_mesh_create(3, 1, 4, 1 << 27, C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), 0, None,
                           None, C.byref(h))
    assert st == -8 and not h.value


@pytest.mark.parametrize("dim,order,n", [(3, 1, 4), (2, 1, 7), (3, 2, 2), (2, 2, 4)])
def test_vertex_order_and_node_labels_do_not_matter(vla, dim, order, n):
    # every element's vertices in a random order (about half of them with a
    # negative determinant; P2 mid-edge nodes moved with their edges), the
    # global node labels permuted at random, the boundary facets listed in
    # reverse order: the outputs still match the oracle on the same arrays
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=n)
    rng = np.random.default_rng(5)
    nv = dim + 1
    edges = [(0, 1), (1, 2), (0, 2)] if dim == 2 else [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    E = np.empty_like(m.elems)
    flipped = 0
    for k in range(m.ne):
        s = rng.permutation(nv)
        flipped += int(np.sum([s[a] > s[b] for a in range(nv) for b in range(a + 1, nv)]) % 2)
        row = list(m.elems[k, s])
        if order == 2:
            edge_node = {frozenset(e): m.elems[k, nv + t] for t, e in enumerate(edges)}
            row += [edge_node[frozenset((s[p], s[q]))] for p, q in edges]
        E[k] = row
    assert 0 < flipped < m.ne
    lab = rng.permutation(m.nn).astype(np.int32)
    E2 = lab[E].astype(np.int32)
    X2 = np.empty_like(m.coords)
    X2[lab] = m.coords
    F2 = np.ascontiguousarray(lab[m.faces][:, ::-1]).astype(np.int32)
    gm = vla.Mesh(_dev(X2), _dev(E2), _dev(F2), order=order)
    ref = oracle.assemble(dim, order, m.nn, E2, X2, 1.0, 1.0)
    rp, ci = gm.csr()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref["row_ptr"])
    np.testing.assert_array_equal(ci.cpu().numpy(), ref["col_idx"])
    o64 = gm.assemble(1.0, 1.0, precision=vla.PREC_FP64, boundary=True)
    omx = gm.assemble(1.0, 1.0, precision=vla.PREC_MIXED, boundary=True)
    for key in ("K", "M", "vol"):
        r = ref[key]
        assert np.abs(o64[key].cpu().numpy() - r).max() <= TOL64 * np.abs(r).max(), key
        assert np.linalg.norm(omx[key].cpu().numpy() - r) <= TOL_MIX * np.linalg.norm(r), key
    assert (o64["vol"] > 0).all()
    rn, ra, miss = oracle.boundary(dim, m.nn, E2, X2, F2)
    assert miss == 0
    np.testing.assert_allclose(o64["normals"].cpu().numpy(), rn, rtol=0, atol=1e-13)
    np.testing.assert_allclose(o64["areas"].cpu().numpy(), ra, rtol=1e-13)
    gm.close()


def _p2_nodes(X, E, dim):
    """Mid-edge nodes appended for every element edge (one node per edge,
    shared by the elements around it), in the element's local edge order."""
    edges = [(0, 1), (1, 2), (0, 2)] if dim == 2 else [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    pts = [np.asarray(x, dtype=np.float64) for x in X]
    mid, rows = {}, []
    for el in E:
        row = [int(v) for v in el]
        for a, b in edges:
            key = (min(el[a], el[b]), max(el[a], el[b]))
            if key not in mid:
                mid[key] = len(pts)
                pts.append(0.5 * (pts[key[0]] + pts[key[1]]))
            row.append(mid[key])
        rows.append(row)
    return np.array(pts), np.array(rows, dtype=np.int32)


def _high_valence_mesh(dim, order, n):
    # 2-D: a fan of n triangles around node 0; 3-D: a book of n tetrahedra
    # around the edge (0, 1).  Node 0 (and 1) lies in n elements
    rng = np.random.default_rng(n)
    ang = np.linspace(0.0, 2 * np.pi, n + 1)[:-1] + rng.uniform(-0.2, 0.2, n) * np.pi / n
    rad = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, n)
    if dim == 2:
        X = np.vstack([[0.05, -0.03], np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)])
        E = np.array([[0, 1 + i, 1 + (i + 1) % n] for i in range(n)], dtype=np.int32)
    else:
        ring = np.stack([rad * np.cos(ang), rad * np.sin(ang), 0.05 * rng.uniform(-1.0, 1.0, n)], axis=1)
        X = np.vstack([[0.02, 0.01, -1.0], [-0.03, 0.02, 1.1], ring])
        E = np.array([[0, 1, 2 + i, 2 + (i + 1) % n] for i in range(n)], dtype=np.int32)
    if order == 2:
        X, E = _p2_nodes(X, E, dim)
    return X, E


@pytest.mark.parametrize("dim,order,n", [(2, 1, 100), (2, 2, 60), (3, 1, 80), (3, 2, 40)])
def test_high_valence_rows(vla, dim, order, n):
    # incidence lists longer than a warp (the build walks them 32 at a time)
    # and pairs with n contributions (node 0 with its neighbours on the fan's
    # centre or the book's spine): pattern bit-exact, values as everywhere
    X, E = _high_valence_mesh(dim, order, n)
    gm = vla.Mesh(_dev(X), _dev(E), order=order)
    ref = oracle.assemble(dim, order, len(X), E, X, 1.0, 0.5)
    rp, ci = gm.csr()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref["row_ptr"])
    np.testing.assert_array_equal(ci.cpu().numpy(), ref["col_idx"])
    assert np.diff(ref["row_ptr"]).max() > 32
    o64 = gm.assemble(1.0, 0.5, precision=vla.PREC_FP64)
    omx = gm.assemble(1.0, 0.5, precision=vla.PREC_MIXED)
    for key in ("K", "M", "vol"):
        r = ref[key]
        assert np.abs(o64[key].cpu().numpy() - r).max() <= TOL64 * np.abs(r).max(), key
        assert np.linalg.norm(omx[key].cpu().numpy() - r) <= TOL_MIX * np.linalg.norm(r), key
    gm.close()


@pytest.mark.parametrize("dim,order,n", [(3, 1, 22), (3, 2, 12), (2, 1, 120), (2, 2, 60)])
def test_tile_node_capacity_second_pass(vla, monkeypatch, dim, order, n):
    # the tile builder first bounds a tile's distinct vertex nodes tightly and,
    # when a tile has more, runs its pass again under the bound no tile can
    # exceed; VLA_TILE_NODE_CAP=64 forces the tight bound down so that every
    # larger tile takes the second pass: the pattern, the tiles and every
    # output stay the same bit for bit
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=n)
    X, E = _dev(m.coords), _dev(m.elems)
    runs = []
    for cap in (None, "64"):
        if cap is not None:
            monkeypatch.setenv("VLA_TILE_NODE_CAP", cap)
        g = vla.Mesh(X, E, order=order)
        rp, ci = g.csr()
        omx = g.assemble(1.0, 1.0, precision=vla.PREC_MIXED)
        o64 = g.assemble(1.0, 1.0, precision=vla.PREC_FP64)
        runs.append(([rp.cpu(), ci.cpu(), omx["K"].cpu(), omx["M"].cpu(), o64["K"].cpu(), o64["M"].cpu()],
                     (g.n_tiles, g.tile_elems, g.n_codes, g.smem_bytes)))
        g.close()
    monkeypatch.delenv("VLA_TILE_NODE_CAP")
    (a, ia), (b, ib) = runs
    assert ia == ib
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    if (dim, order) == (3, 1):
        # every vertex of this mesh is in at most 24 tetrahedra, so a tile of
        # more than 6 x 64 elements has more than 64 vertex nodes: the second
        # pass did run
        assert ia[1] / ia[0] > 6 * 64


def test_builds_on_several_streams_and_threads(vla):
    # a host thread's builds share its kept scratch memory; builds on
    # alternating streams of one thread, a facet query between them, and
    # builds on two threads at once must give the same meshes as one build
    # on the current stream
    import threading
    specs = [(3, 1, 12), (2, 2, 20), (3, 2, 5), (2, 1, 60)]
    meshes = [meshgen.make_mesh(d, n, order=o, jitter=0.1, seed=n) for d, o, n in specs]
    args = [(_dev(m.coords), _dev(m.elems), o) for m, (_, o, _) in zip(meshes, specs)]

    def summary(g):
        rp, ci = g.csr()
        o = g.assemble(1.0, 1.0, precision=vla.PREC_MIXED)
        return [rp.cpu(), ci.cpu(), o["K"].cpu(), o["M"].cpu(), o["vol"].cpu()]

    ref = []
    for X, E, o in args:
        g = vla.Mesh(X, E, order=o)
        ref.append(summary(g))
        g.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep in range(2):
        for k, (X, E, o) in enumerate(args):
            s = streams[(k + rep) % 2]
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                g = vla.Mesh(X, E, order=o, stream=s)
                g.facets(stream=s)
                got = summary(g)
            torch.cuda.synchronize()
            for a, b in zip(got, ref[k]):
                assert torch.equal(a, b)
            g.close()
    out, errors = {}, []

    def worker(t):
        try:
            s = torch.cuda.Stream()
            for k in range(t, len(args), 2):
                X, E, o = args[k]
                with torch.cuda.stream(s):
                    g = vla.Mesh(X, E, order=o, stream=s)
                    out[k] = summary(g)
                    torch.cuda.synchronize()
                    g.close()
        except Exception as e:   # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    for k in range(len(args)):
        for a, b in zip(out[k], ref[k]):
            assert torch.equal(a, b)
