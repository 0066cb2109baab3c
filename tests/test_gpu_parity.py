"""GPU parity: every CUDA entry point against the CPU FP64 oracle on the same
seeded inputs.

Tolerances:
  integer work (CSR pattern): bit-exact;
  FP64 paths: |gpu - ref| <= 1e-12 * max(|ref|, max over the row of |ref|)
  (an FP64 sum of <= 24 terms of one row's magnitude errs by ~24u ~ 5e-15 of it);
  mixed FP32/compensated paths: relative Frobenius error <= 1e-5 per output;
  FP32 page primitives: relative Frobenius error per page <= 1e-5 (scaled by
  the page condition number for inverses).
"""
import math

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


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---------------------------------------------------------------------------
# page primitives
# ---------------------------------------------------------------------------

def _to_layout(A, layout):
    # A: numpy (N, cols, rows) page layout -> tensor in the requested layout
    if layout == 0:
        return A
    return np.ascontiguousarray(np.transpose(A, (1, 2, 0)))


def _from_layout(X, layout):
    if layout == 0:
        return X
    return np.ascontiguousarray(np.transpose(X, (2, 0, 1)))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("N", [0, 1, 77, 128 * 37 + 55])
def test_page_primitives(vla, layout, dt, n, N):
    P = meshgen.random_pages(max(N, 1), n, seed=N + n)
    A, B, s, v = (P[k][:N].astype(dt) for k in ("A", "B", "s", "v"))
    tA, tB = _dev(_to_layout(A, layout)), _dev(_to_layout(B, layout))
    ts = _dev(s)
    tv = _dev(v if layout == 0 else np.ascontiguousarray(v.T))
    tol = TOL64 if dt == np.float64 else TOL_MIX
    C = _from_layout(vla.amtam(tA, tB, layout=layout).cpu().numpy(), layout)
    S = _from_layout(vla.astam(ts, tA, layout=layout).cpu().numpy(), layout)
    Y = vla.avtam(tv, tA, layout=layout).cpu().numpy()
    Y = Y if layout == 0 else Y.T
    D = vla.amdet(tA, layout=layout).cpu().numpy()
    inv, det, ns = vla.aminv(tA, layout=layout)
    I = _from_layout(inv.cpu().numpy(), layout)
    torch.cuda.synchronize()
    if N == 0:
        assert C.size == 0 and int(ns.item()) == 0
        return
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    Cr = oracle.amtam(A64, B64)
    Sr = oracle.astam(s.astype(np.float64), A64)
    Yr = oracle.avtam(v.astype(np.float64), A64)
    Dr = oracle.amdet(A64)
    Ir, Dr2, nsr = oracle.aminv(A64)
    scale = np.abs(A64).max(axis=(1, 2)) * np.abs(B64).max(axis=(1, 2)) * n
    assert np.all(np.abs(C - Cr).max(axis=(1, 2)) <= 4 * tol * scale)
    assert np.all(np.abs(S - Sr) <= tol * np.abs(Sr) + 1e-300)
    assert np.all(np.abs(Y - Yr).max(axis=1) <= 4 * tol * np.abs(v).max(axis=1) * np.abs(A64).max(axis=(1, 2)) * n)
    dscale = np.abs(A64).max(axis=(1, 2)) ** n * 6
    assert np.all(np.abs(D - Dr) <= 4 * tol * dscale)
    assert np.all(np.abs(det.cpu().numpy() - D) <= 4 * tol * dscale)
    cond = np.linalg.cond(np.transpose(A64, (0, 2, 1)))
    err = np.abs(I - Ir).max(axis=(1, 2)) / np.abs(Ir).max(axis=(1, 2))
    assert np.all(err <= 8 * tol * cond)
    assert int(ns.item()) == nsr == 0


@pytest.mark.parametrize("layout", [0, 1])
def test_singular_pages_counted(vla, layout):
    N = 128 * 3 + 5
    P = meshgen.random_pages(N, 3, seed=9)
    A = P["A"].copy()
    sing = [0, 100, 128 * 2 + 3, N - 1]
    for k in sing:
        A[k, 2, :] = 2.0 * A[k, 0, :]          # dependent columns -> det exactly 0 in any order
        A[k] = np.round(A[k] * 4) / 4
        A[k, 2, :] = 2.0 * A[k, 0, :]
    inv, det, ns = vla.aminv(_dev(_to_layout(A, layout)), layout=layout)
    _, dref, nref = oracle.aminv(A)
    assert int(ns.item()) == nref == len(sing)
    I = _from_layout(inv.cpu().numpy(), layout)
    for k in sing:
        assert det.cpu().numpy()[k] == 0.0 and not np.all(np.isfinite(I[k]))


def test_page_primitives_rectangular_shapes(vla):
    rng = np.random.default_rng(5)
    for (p, m, n) in [(2, 3, 2), (3, 2, 3), (3, 3, 2), (2, 2, 3)]:
        A = rng.standard_normal((300, m, p))
        B = rng.standard_normal((300, n, p))
        C = vla.amtam(_dev(A), _dev(B)).cpu().numpy()
        np.testing.assert_allclose(C, oracle.amtam(A, B), rtol=0, atol=1e-13)
    for (p, n) in [(2, 3), (3, 2)]:
        A = rng.standard_normal((300, n, p))
        v = rng.standard_normal((300, p))
        np.testing.assert_allclose(vla.avtam(_dev(v), _dev(A)).cpu().numpy(), oracle.avtam(v, A), atol=1e-13)


def test_page_primitives_misaligned_pointer(vla):
    # a view starting 8 bytes into the allocation cannot use the bulk-copy path
    P = meshgen.random_pages(1000, 3, seed=2)
    buf = torch.empty(1000 * 9 + 1, dtype=torch.float64, device="cuda")
    buf[1:] = _dev(P["A"]).reshape(-1)
    A = buf[1:].view(1000, 3, 3)
    D = vla.amdet(A).cpu().numpy()
    np.testing.assert_allclose(D, oracle.amdet(P["A"]), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("op", ["amtam", "aminv", "astam", "avtam", "amdet", "amtam_f32"])
def test_page_primitives_full_size_sampled(vla, op):
    # N = 1e8 pages of 3x3 FP64 (the largest sweep point), generated on the device;
    # a seeded sample of 1e5 pages is checked against the oracle
    N = 100_000_000
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((N, 3, 3), generator=g, dtype=torch.float64, device="cuda")
    A[:, [0, 1, 2], [0, 1, 2]] += 3.0
    idx = np.random.default_rng(0).choice(N, 100_000, replace=False)
    Ai = A[torch.from_numpy(idx).cuda()].cpu().numpy()
    sel = torch.from_numpy(idx).cuda()
    if op == "amtam":
        B = torch.randn((N, 3, 3), generator=g, dtype=torch.float64, device="cuda")
        C = vla.amtam(A, B)
        Bi = B[sel].cpu().numpy()
        Ci = C[sel].cpu().numpy()
        np.testing.assert_allclose(Ci, oracle.amtam(Ai, Bi), rtol=0, atol=1e-12 * np.abs(Ci).max())
        del B, C
    elif op == "amtam_f32":   # the FP32 sweep point: the same pages rounded to float
        A32 = A.float()
        del A
        B32 = torch.randn((N, 3, 3), generator=g, dtype=torch.float32, device="cuda")
        C = vla.amtam(A32, B32)
        Ai, Bi, Ci = (x[sel].double().cpu().numpy() for x in (A32, B32, C))
        ref = oracle.amtam(Ai, Bi)   # FP64 of the FP32 inputs: only the float products' rounding differs
        assert np.abs(Ci - ref).max() <= 1e-5 * np.abs(ref).max()
        del A32, B32, C
        torch.cuda.empty_cache()
        return
    elif op == "astam":
        sc = 0.5 + 1.5 * torch.rand(N, generator=g, dtype=torch.float64, device="cuda")
        C = vla.astam(sc, A)
        np.testing.assert_allclose(C[sel].cpu().numpy(), oracle.astam(sc[sel].cpu().numpy(), Ai), rtol=1e-15, atol=0)
        del sc, C
    elif op == "avtam":
        v = torch.randn((N, 3), generator=g, dtype=torch.float64, device="cuda")
        y = vla.avtam(v, A)
        yr = oracle.avtam(v[sel].cpu().numpy(), Ai)
        np.testing.assert_allclose(y[sel].cpu().numpy(), yr, rtol=0, atol=1e-12 * np.abs(yr).max())
        del v, y
    elif op == "amdet":
        d = vla.amdet(A)
        dr = oracle.amdet(Ai)
        np.testing.assert_allclose(d[sel].cpu().numpy(), dr, rtol=0, atol=1e-12 * np.abs(dr).max())
        del d
    else:
        inv, det, ns = vla.aminv(A)
        Ii = inv[sel].cpu().numpy()
        Ir, Dr, _ = oracle.aminv(Ai)
        cond = np.linalg.cond(np.transpose(Ai, (0, 2, 1)))
        err = np.abs(Ii - Ir).max(axis=(1, 2)) / np.abs(Ir).max(axis=(1, 2))
        assert np.all(err <= 8e-12 * cond)
        del inv, det
    del A
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# meshes: pattern, assembly, boundary, facet normals
# ---------------------------------------------------------------------------

def _gpu_mesh(vla, m):
    return vla.Mesh(_dev(m.coords), _dev(m.elems), _dev(m.faces) if m.nfb else None, order=m.order)


def _check_fp64(got, ref, rp):
    # |got - ref| <= 1e-12 max(|ref|, max over the row of |ref|)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    rowmax = np.zeros(len(rp) - 1)
    np.maximum.at(rowmax, rows, np.abs(ref))
    bound = TOL64 * np.maximum(np.abs(ref), rowmax[rows])
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{bad.sum()} entries off, worst {np.abs(got - ref).max():.3e}"


CASES = [(2, 1, 5), (2, 1, 37), (3, 1, 3), (3, 1, 9), (2, 2, 4), (2, 2, 17), (3, 2, 2), (3, 2, 5)]


@pytest.mark.parametrize("dim,order,n", CASES)
def test_pattern_bit_exact(vla, dim, order, n):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=n)
    gm = _gpu_mesh(vla, m)
    rp, ci = gm.csr()
    rpr, cir = oracle.csr_pattern(m.nn, m.elems)
    np.testing.assert_array_equal(rp.cpu().numpy(), rpr)
    np.testing.assert_array_equal(ci.cpu().numpy(), cir)
    assert gm.nnz == len(cir)
    rpv, civ = gm.csr_view()   # the mesh's own arrays, no copy
    assert torch.equal(rpv, rp) and torch.equal(civ, ci)
    rpb, cib = gm.block()
    assert torch.equal(rpb, rp) and torch.equal(cib, ci)


@pytest.mark.parametrize("dim,order,n", CASES)
@pytest.mark.parametrize("kind,ca,cb", [(0, 1.0, 0.0), (0, 1.0, 1.0), (1, 1.0, 1.0), (1, 2.5, -0.7)])
def test_assembly_fp64(vla, dim, order, n, kind, ca, cb):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=3 * n + order)
    gm = _gpu_mesh(vla, m)
    out = gm.assemble(ca, cb, kind=kind, precision=vla.PREC_FP64, pages=True, count_singular=True)
    ref = oracle.assemble(dim, order, m.nn, m.elems, m.coords, ca, cb, want_pages=True, ckind=kind)
    _check_fp64(out["K"].cpu().numpy(), ref["K"], ref["row_ptr"])
    _check_fp64(out["M"].cpu().numpy(), ref["M"], ref["row_ptr"])
    np.testing.assert_allclose(out["vol"].cpu().numpy(), ref["vol"], rtol=TOL64, atol=0)
    Kp, Mp = out["K3D"].cpu().numpy(), out["M3D"].cpu().numpy()
    for P, R in ((Kp, ref["K3D"]), (Mp, ref["M3D"])):
        err = np.abs(P - R).max(axis=(1, 2)) / np.abs(R).max(axis=(1, 2))
        assert err.max() <= TOL64
    assert int(out["n_singular"].item()) == 0


@pytest.mark.parametrize("dim,order,n", CASES)
def test_assembly_mixed(vla, dim, order, n):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=5 * n + order)
    gm = _gpu_mesh(vla, m)
    out = gm.assemble(1.0, 1.0, precision=vla.PREC_MIXED, pages=True)
    ref = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 1.0, 1.0, want_pages=True)
    for key in ("K", "M", "vol"):
        e = _rel_fro(out[key].cpu().numpy(), ref[key])
        assert e <= TOL_MIX, (key, e)
    for key in ("K3D", "M3D"):
        assert _rel_fro(out[key].cpu().numpy(), ref[key]) <= TOL_MIX


def test_config0_fp64_with_pages(vla):
    # 8x8x8 cubes x 6 tets, interior jitter 0.1h, seed 0, c = 1, FP64, pages
    m = meshgen.kuhn_cube(8, jitter=0.1, seed=0)
    assert (m.ne, m.nn) == (3072, 729)
    gm = _gpu_mesh(vla, m)
    assert gm.nnz == 9097
    out = gm.assemble(1.0, 0.0, precision=vla.PREC_FP64, pages=True)
    ref = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 0.0, want_pages=True)
    _check_fp64(out["K"].cpu().numpy(), ref["K"], ref["row_ptr"])
    _check_fp64(out["M"].cpu().numpy(), ref["M"], ref["row_ptr"])
    np.testing.assert_allclose(out["vol"].cpu().numpy(), ref["vol"], rtol=TOL64)
    assert out["vol"].sum().item() == pytest.approx(1.0, abs=1e-13)
    np.testing.assert_allclose(out["K3D"].cpu().numpy(), ref["K3D"], rtol=0, atol=TOL64 * np.abs(ref["K3D"]).max())
    np.testing.assert_allclose(out["M3D"].cpu().numpy(), ref["M3D"], rtol=0, atol=TOL64 * np.abs(ref["M3D"]).max())


def test_config2_full_size_mixed(vla):
    # 64^3 cubes x 6 tets (1,572,864 tets, 274,625 nodes), c = 1 + |x|^2, mixed precision,
    # boundary normals and areas of the 49,152 boundary triangles: every output vs the oracle
    m = meshgen.kuhn_cube(64, jitter=0.1, seed=0)
    gm = _gpu_mesh(vla, m)
    assert (gm.ne, gm.nn, gm.nnz, gm.nfb) == (1572864, 274625, 4018753, 49152)
    # the benchmark's launch: assembly and boundary facets in one launch
    out = gm.assemble(1.0, 1.0, precision=vla.PREC_MIXED, boundary=True)
    nrm, ar = out["normals"], out["areas"]
    n2, a2 = gm.boundary(precision=vla.PREC_MIXED)
    assert torch.equal(nrm, n2) and torch.equal(ar, a2)
    ref = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0)
    rn, ra, _ = oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
    rp, ci = gm.csr()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref["row_ptr"])
    np.testing.assert_array_equal(ci.cpu().numpy(), ref["col_idx"])
    errs = {k: _rel_fro(out[k].cpu().numpy(), ref[k]) for k in ("K", "M", "vol")}
    errs["normals"] = _rel_fro(nrm.cpu().numpy(), rn)
    errs["areas"] = _rel_fro(ar.cpu().numpy(), ra)
    for k, e in errs.items():
        assert e <= TOL_MIX, (k, e)
    # the FP64 form on the same mesh meets the FP64 bound
    o64 = gm.assemble(1.0, 1.0, precision=vla.PREC_FP64)
    _check_fp64(o64["K"].cpu().numpy(), ref["K"], ref["row_ptr"])
    _check_fp64(o64["M"].cpu().numpy(), ref["M"], ref["row_ptr"])


@pytest.mark.parametrize("dim,order,n", [(3, 1, 4), (2, 2, 6), (3, 2, 3)])
def test_boundary_and_facet_normals(vla, dim, order, n):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=n)
    # a general affine map makes the boundary normals non-trivial
    Aff = np.array([[1.0, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.1, 1.1]])[:dim, :dim]
    m.coords = np.ascontiguousarray(m.coords @ Aff.T + 0.25)
    gm = _gpu_mesh(vla, m)
    rn, ra, miss = oracle.boundary(dim, m.nn, m.elems, m.coords, m.faces)
    assert miss == 0
    n64, a64 = gm.boundary(precision=vla.PREC_FP64)
    np.testing.assert_allclose(n64.cpu().numpy(), rn, rtol=0, atol=1e-13)
    np.testing.assert_allclose(a64.cpu().numpy(), ra, rtol=1e-13)
    nmx, amx = gm.boundary(precision=vla.PREC_MIXED)
    assert _rel_fro(nmx.cpu().numpy(), rn) <= TOL_MIX and _rel_fro(amx.cpu().numpy(), ra) <= TOL_MIX
    sn = gm.simplex_normals().cpu().numpy()
    snr = oracle.simplex_normals(dim, m.elems, m.coords)
    err = np.abs(sn - snr).max(axis=(1, 2)) / np.abs(snr).max(axis=(1, 2))
    assert err.max() <= TOL64


@pytest.mark.parametrize("dim,order,n", [(2, 1, 5), (3, 1, 4), (2, 2, 6), (3, 2, 3), (3, 1, 17)])
def test_assembly_with_boundary_one_launch(vla, dim, order, n):
    # vla_assemble_with_boundary equals vla_assemble followed by vla_boundary, bit for bit
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=7 * n)
    gm = _gpu_mesh(vla, m)
    rn, ra, _ = oracle.boundary(dim, m.nn, m.elems, m.coords, m.faces)
    for prec in (vla.PREC_FP64, vla.PREC_MIXED):
        one = gm.assemble(0.7, 1.3, precision=prec, pages=True, count_singular=True, boundary=True)
        two = gm.assemble(0.7, 1.3, precision=prec, pages=True, count_singular=True)
        nrm, ar = gm.boundary(precision=prec)
        for key in ("K", "M", "vol", "K3D", "M3D", "n_singular"):
            assert torch.equal(one[key], two[key]), key
        assert torch.equal(one["normals"], nrm) and torch.equal(one["areas"], ar)
        tol = 1e-13 if prec == vla.PREC_FP64 else TOL_MIX
        assert _rel_fro(one["normals"].cpu().numpy(), rn) <= tol
        assert _rel_fro(one["areas"].cpu().numpy(), ra) <= tol
    # a mesh given without boundary facets: the fused call is the plain assembly
    bare = vla.Mesh(_dev(m.coords), _dev(m.elems), None, order=m.order)
    one = bare.assemble(1.0, 0.0, precision=vla.PREC_MIXED, boundary=True)
    assert one["normals"].numel() == 0 and one["areas"].numel() == 0
    assert torch.equal(one["K"], bare.assemble(1.0, 0.0, precision=vla.PREC_MIXED)["K"])


def test_worked_tetrahedron_normals(vla):
    coords = np.array([[7, 3, -1], [7, -2, 4], [10, 3, 4], [4, 3, 4]], dtype=np.float64) / 4.0
    elems = np.array([[0, 1, 2, 3]], dtype=np.int32)
    gm = vla.Mesh(_dev(coords), _dev(elems))
    N = gm.simplex_normals().cpu().numpy()[0].T
    expect = np.array([[0, 0, -2 / 3, 2 / 3], [0, 4 / 5, -2 / 5, -2 / 5], [4 / 5, 0, -2 / 5, -2 / 5]])
    np.testing.assert_allclose(N, expect, atol=1e-15)
    vol = gm.assemble(precision=vla.PREC_FP64)["vol"].cpu().numpy()
    assert vol[0] == pytest.approx(25 / 64, abs=1e-15)


def test_assembly_deterministic(vla):
    m = meshgen.kuhn_cube(12, jitter=0.1, seed=4)
    gm = _gpu_mesh(vla, m)
    for prec in (vla.PREC_MIXED, vla.PREC_FP64):
        a = gm.assemble(1.0, 1.0, precision=prec)
        b = gm.assemble(1.0, 1.0, precision=prec)
        for k in ("K", "M", "vol"):
            assert torch.equal(a[k], b[k])
    # an independently built handle of the same mesh gives the same bits
    gm2 = _gpu_mesh(vla, m)
    c = gm2.assemble(1.0, 1.0, precision=vla.PREC_MIXED)
    d = gm.assemble(1.0, 1.0, precision=vla.PREC_MIXED)
    assert torch.equal(c["K"], d["K"]) and torch.equal(c["M"], d["M"])


def test_sliver_elements_mixed_precision(vla):
    # tetrahedra flattened towards a face plane (vol/h^3 from 1e-2 down to 1e-6), far
    # from the origin; the compensated determinant keeps the mixed-precision error of
    # K, M and vol within the stated bound relative to the FP64 oracle
    rng = np.random.default_rng(7)
    coords, elems = [], []
    for q, eps in enumerate([1e-2, 1e-3, 1e-4, 1e-5, 1e-6] * 4):
        base = np.array([37.0, -11.0, 5.0]) + rng.uniform(-1, 1, 3)
        h = 1.0 / 64
        P = np.array([[0, 0, 0], [h, 0, 0], [0.3 * h, h, 0], [0.4 * h, 0.3 * h, eps * h]]) + base
        coords.extend(P)
        elems.append([4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3])
    coords = np.array(coords)
    elems = np.array(elems, dtype=np.int32)
    gm = vla.Mesh(_dev(coords), _dev(elems))
    out = gm.assemble(1.0, 0.0, precision=vla.PREC_MIXED, pages=True)
    ref = oracle.assemble(3, 1, len(coords), elems, coords, 1.0, 0.0, want_pages=True)
    Kp, Kr = out["K3D"].cpu().numpy(), ref["K3D"]
    for k in range(len(elems)):
        assert _rel_fro(Kp[k], Kr[k]) <= TOL_MIX, (k, _rel_fro(Kp[k], Kr[k]))
    assert _rel_fro(out["vol"].cpu().numpy(), ref["vol"]) <= TOL_MIX
    np.testing.assert_allclose(out["vol"].cpu().numpy(), ref["vol"], rtol=1e-5)


# ---------------------------------------------------------------------------
# edge cases and error reporting
# ---------------------------------------------------------------------------

def test_single_element_and_isolated_node(vla):
    coords = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [5, 5, 5]], dtype=np.float64)
    elems = np.array([[0, 1, 2, 3]], dtype=np.int32)   # node 4 belongs to no element: empty row
    gm = vla.Mesh(_dev(coords), _dev(elems))
    rp, ci = gm.csr()
    rpr, cir = oracle.csr_pattern(5, elems)
    np.testing.assert_array_equal(rp.cpu().numpy(), rpr)
    for prec in (vla.PREC_FP64, vla.PREC_MIXED):
        out = gm.assemble(2.0, 0.0, precision=prec)
        ref = oracle.assemble(3, 1, 5, elems, coords, 2.0, 0.0)
        assert _rel_fro(out["K"].cpu().numpy(), ref["K"]) <= (1e-14 if prec == 0 else TOL_MIX)


def test_degenerate_element_counts_singular(vla):
    coords = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.float64)
    elems = np.array([[0, 1, 2, 4], [0, 1, 2, 3]], dtype=np.int32)   # second tet is flat
    gm = vla.Mesh(_dev(coords), _dev(elems))
    out = gm.assemble(precision=vla.PREC_FP64, count_singular=True)
    assert int(out["n_singular"].item()) == 1
    assert out["vol"].cpu().numpy()[1] == 0.0


def test_invalid_meshes_rejected(vla):
    coords = _dev(np.zeros((4, 3)))
    with pytest.raises(vla.VlaError) as e:
        vla.Mesh(coords, _dev(np.array([[0, 1, 2, 4]], np.int32)))
    assert e.value.status == -2
    with pytest.raises(vla.VlaError) as e:
        vla.Mesh(coords, _dev(np.array([[0, 1, 1, 3]], np.int32)))
    assert e.value.status == -7
    good = _dev(np.array([[0, 1, 2, 3]], np.int32))
    with pytest.raises(vla.VlaError) as e:
        vla.Mesh(coords, good, faces=_dev(np.array([[0, 1, 9]], np.int32)))
    assert e.value.status == -2
    with pytest.raises(vla.VlaError) as e:
        vla.Mesh(_dev(np.zeros((5, 3))), good, faces=_dev(np.array([[0, 1, 4]], np.int32)))
    assert e.value.status == -7


# ---------------------------------------------------------------------------
# the paper's literal P1 listing: degree-2 rule, coefficient at every point
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 5), (2, 33), (3, 3), (3, 9)])
@pytest.mark.parametrize("kind", [2, 3])
def test_literal_quadrature_fp64_and_mixed(vla, dim, n, kind):
    m = meshgen.make_mesh(dim, n, order=1, jitter=0.1, seed=7 * n + kind)
    gm = _gpu_mesh(vla, m)
    ref = oracle.assemble(dim, 1, m.nn, m.elems, m.coords, 1.2, 0.8, want_pages=True, ckind=kind)
    out = gm.assemble(1.2, 0.8, kind=kind, precision=vla.PREC_FP64, pages=True)
    _check_fp64(out["K"].cpu().numpy(), ref["K"], ref["row_ptr"])
    _check_fp64(out["M"].cpu().numpy(), ref["M"], ref["row_ptr"])
    for key in ("K3D", "M3D"):
        P, R = out[key].cpu().numpy(), ref[key]
        assert (np.abs(P - R).max(axis=(1, 2)) / np.abs(R).max(axis=(1, 2))).max() <= TOL64
    mixed = gm.assemble(1.2, 0.8, kind=kind, precision=vla.PREC_MIXED, pages=True)
    for key in ("K", "M", "vol", "K3D", "M3D"):
        assert _rel_fro(mixed[key].cpu().numpy(), ref[key]) <= TOL_MIX, key


def test_literal_quadrature_limits(vla):
    p2 = _gpu_mesh(vla, meshgen.make_mesh(3, 2, order=2))
    with pytest.raises(vla.VlaError) as e:
        p2.assemble(1.0, 1.0, kind=vla.COEFF_EXP_IP)
    assert e.value.status == -8
    p1 = _gpu_mesh(vla, meshgen.kuhn_cube(2))
    with pytest.raises(vla.VlaError):
        vla.Batch([(p1, p1.outputs(), vla.COEFF_EXP_IP, 1.0, 1.0)])


# ---------------------------------------------------------------------------
# facet list (integer work: bit-exact against the oracle)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,order,n", [(2, 1, 6), (2, 2, 4), (3, 1, 4), (3, 2, 3), (3, 1, 16)])
def test_facet_list_bit_exact(vla, dim, order, n):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=n)
    gm = _gpu_mesh(vla, m)
    faces, owner, nbr, nb = gm.facets()
    rf, ro, rn, rnb = oracle.facets(dim, m.elems)
    np.testing.assert_array_equal(faces.cpu().numpy(), rf)
    np.testing.assert_array_equal(owner.cpu().numpy(), ro)
    np.testing.assert_array_equal(nbr.cpu().numpy(), rn)
    assert nb == rnb == m.nfb


def test_facet_counts_full_size(vla):
    # level 5 of the paper's normals table: 1,572,864 tets -> 3,170,304 faces, 49,152 on the boundary
    m = meshgen.kuhn_cube(64, jitter=0.1, seed=0)
    gm = _gpu_mesh(vla, m)
    faces, owner, nbr, nb = gm.facets()
    assert (faces.shape[0], nb) == (3170304, 49152)
    # the boundary facets are the mesh's boundary triangles (as vertex sets)
    bf = np.sort(faces[nbr < 0].cpu().numpy(), axis=1)
    ref = np.sort(m.faces, axis=1)
    assert set(map(tuple, bf)) == set(map(tuple, ref))
