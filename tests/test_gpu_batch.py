"""GPU: batched assembly of many meshes in one persistent launch, the
autotuner, and the device error word of bounded waits.

Every batch job must be bit-identical to vla_assemble on its mesh alone (the
summation order of each CSR value and page entry depends only on the mesh),
and the single-mesh path is itself checked against the FP64 oracle in
test_gpu_parity.py; small jobs are also compared with the oracle directly.
"""
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


def _gpu_mesh(vla, m):
    return vla.Mesh(_dev(m.coords), _dev(m.elems), _dev(m.faces) if m.nfb else None, order=m.order)


def _rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# a mix of every element type and of tile counts from 1 to many
MIX_SPECS = [(2, 1, 3), (3, 2, 2), (3, 1, 9), (2, 2, 11), (3, 1, 1), (2, 1, 40), (3, 2, 4), (2, 2, 2),
             (3, 1, 14), (2, 1, 7), (3, 2, 1), (2, 2, 23)]


def _mix(vla, specs, seed0=0):
    meshes, gms = [], []
    for q, (dim, order, n) in enumerate(specs):
        m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=seed0 + q)
        meshes.append(m)
        gms.append(_gpu_mesh(vla, m))
    return meshes, gms


def _coeffs(q):
    return (0 if q % 3 else 1), 0.5 + 0.25 * (q % 5), 0.1 * (q % 4)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("form", ["fused", "split", "tuned"])
def test_batch_bit_identical_to_single(vla, precision, graph, form):
    meshes, gms = _mix(vla, MIX_SPECS)
    jobs = []
    for q, gm in enumerate(gms):
        kind, ca, cb = _coeffs(q)
        jobs.append((gm, gm.outputs(pages=(q % 4 == 1)), kind, ca, cb))
    b = vla.Batch(jobs, precision=precision, graph=graph, count_singular=True,
                  form=None if form == "tuned" else form, tune=form == "tuned")
    if form != "tuned":
        assert b.split == (form == "split")
    assert b.count == len(jobs) and b.graph == graph
    assert b.n_work == sum(gm.n_tiles for gm in gms)
    assert b.elements == sum(m.ne for m in meshes)
    for rep in range(2):   # a second run (graph replay) gives the same bits
        b.run()
        torch.cuda.synchronize()
        for q, gm in enumerate(gms):
            kind, ca, cb = _coeffs(q)
            ref = gm.assemble(ca, cb, kind=kind, precision=precision, pages=(q % 4 == 1))
            got = b.outs[q]
            for key in ("K", "M", "vol") + (("K3D", "M3D") if q % 4 == 1 else ()):
                assert torch.equal(got[key], ref[key]), (q, key, rep)
    assert int(b.n_singular.abs().sum().item()) == 0
    b.check()
    b.close()


def test_batch_against_oracle(vla):
    specs = [(2, 1, 6), (2, 2, 5), (3, 1, 4), (3, 2, 2)]
    meshes, gms = _mix(vla, specs, seed0=40)
    for precision, tol in ((0, None), (1, TOL_MIX)):
        jobs = [(gm, gm.outputs(pages=True), 0, 1.0, 1.0) for gm in gms]
        vla.Batch(jobs, precision=precision).run()
        torch.cuda.synchronize()
        for (m, (_, out, *_)) in zip(meshes, jobs):
            ref = oracle.assemble(m.dim, m.order, m.nn, m.elems, m.coords, 1.0, 1.0, want_pages=True)
            for key, rk in (("K", "K"), ("M", "M"), ("vol", "vol"), ("K3D", "K3D"), ("M3D", "M3D")):
                got = out[key].cpu().numpy()
                if tol is None:
                    scale = np.abs(ref[rk]).max()
                    assert np.abs(got - ref[rk]).max() <= TOL64 * scale, key
                else:
                    assert _rel_fro(got, ref[rk]) <= tol, key


def test_batch_set_job_and_one_shot(vla):
    meshes, gms = _mix(vla, MIX_SPECS[:6], seed0=7)
    jobs = [(gm, gm.outputs(), 0, 1.0, 0.0) for gm in gms]
    b = vla.Batch(jobs, precision=1, graph=True)
    b.run()
    # new coefficient and new outputs for job 2, same mesh, stream ordered
    fresh = gms[2].outputs()
    b.set_job(2, fresh, kind=0, ca=1.7, cb=0.6)
    b.run()
    torch.cuda.synchronize()
    ref = gms[2].assemble(1.7, 0.6, precision=1)
    assert torch.equal(fresh["K"], ref["K"]) and torch.equal(fresh["M"], ref["M"])
    ref0 = gms[0].assemble(1.0, 0.0, precision=1)
    assert torch.equal(b.outs[0]["K"], ref0["K"])
    # one-shot batch (stream-ordered tables)
    outs = vla.batch_assemble([(gm, gm.outputs(), 1, 1.0, 0.5) for gm in gms], precision=1)
    torch.cuda.synchronize()
    for gm, o in zip(gms, outs):
        r = gm.assemble(1.0, 0.5, kind=1, precision=1)
        assert torch.equal(o["K"], r["K"]) and torch.equal(o["vol"], r["vol"])
    with pytest.raises(vla.VlaError):
        b.set_job(0, gms[0].outputs(), kind=7)   # unknown coefficient kind
    b.close()


def test_batch_singular_counts_per_job(vla):
    coords = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.float64)
    flat = vla.Mesh(_dev(coords), _dev(np.array([[0, 1, 2, 4], [0, 1, 2, 3]], dtype=np.int32)))
    good = _gpu_mesh(vla, meshgen.kuhn_cube(2, seed=1))
    b = vla.Batch([(good, good.outputs(), 0, 1.0, 0.0), (flat, flat.outputs(), 0, 1.0, 0.0)],
                  precision=0, count_singular=True)
    b.run()
    torch.cuda.synchronize()
    assert b.n_singular.cpu().tolist() == [0, 1]
    b.run()   # counts are reset by every run
    torch.cuda.synchronize()
    assert b.n_singular.cpu().tolist() == [0, 1]


def test_batch_uneven_config_scaled(vla):
    # the uneven mix of the batched workload (2-D/3-D x P1/P2, log-uniform sizes),
    # 32 meshes of 1e3..1e5 elements: every job bit-identical to its single assembly
    specs = meshgen.batch_specs(32, lo=1e3, hi=1e5, seed=3)
    gms = [_gpu_mesh(vla, meshgen.make_mesh(s["dim"], s["n"], order=s["order"], seed=s["seed"])) for s in specs]
    jobs = [(gm, gm.outputs(), 0, 1.0, 1.0) for gm in gms]
    b = vla.Batch(jobs, precision=1, graph=True)
    b.run()
    torch.cuda.synchronize()
    for gm, (_, out, *_) in zip(gms, jobs):
        ref = gm.assemble(1.0, 1.0, precision=1)
        assert torch.equal(out["K"], ref["K"]) and torch.equal(out["M"], ref["M"])
    b.check()


def test_batch_uneven_full_size(vla):
    # the batched workload at full size, in the launch the benchmark times: 256
    # meshes (2-D/3-D x P1/P2, 1e3..1e6 elements, 45 M elements), c = 1 + |x|^2,
    # mixed precision, one graph-captured launch per element type.  Every job
    # equals its single-mesh assembly bit for bit; every mesh's K rows sum to
    # zero and its volumes to the domain's; the smallest mesh of each type is
    # checked against the FP64 oracle
    specs = meshgen.batch_specs(256, 1e3, 1e6, seed=0)
    meshes = [meshgen.make_mesh(s["dim"], s["n"], order=s["order"], jitter=0.1, seed=s["seed"]) for s in specs]
    assert sum(m.ne for m in meshes) == 45000030
    gms = [_gpu_mesh(vla, m) for m in meshes]
    jobs = [(gm, gm.outputs(), 0, 1.0, 1.0) for gm in gms]
    b = vla.Batch(jobs, precision=1, graph=True, form="split")
    b.run()
    torch.cuda.synchronize()
    b.check()
    smallest = {}
    for q, (m, gm, (_, out, *_)) in enumerate(zip(meshes, gms, jobs)):
        ref = gm.assemble(1.0, 1.0, precision=1)
        for key in ("K", "M", "vol"):
            assert torch.equal(out[key], ref[key]), (q, key)
        rp, _ = gm.csr()
        rows = torch.repeat_interleave(torch.arange(gm.nn, device=rp.device), rp[1:] - rp[:-1])
        rsum = torch.zeros(gm.nn, dtype=torch.float64, device=rp.device).index_add_(0, rows, out["K"])
        rmax = torch.zeros(gm.nn, dtype=torch.float64, device=rp.device).scatter_reduce_(
            0, rows, out["K"].abs(), "amax", include_self=False)
        assert (rsum.abs() <= 1e-5 * rmax).all(), q
        assert abs(out["vol"].sum().item() - 1.0) <= 1e-6, q
        key = (m.dim, m.order)
        if key not in smallest or m.ne < smallest[key][0].ne:
            smallest[key] = (m, out)
    for m, out in smallest.values():
        ref = oracle.assemble(m.dim, m.order, m.nn, m.elems, m.coords, 1.0, 1.0)
        for key in ("K", "M", "vol"):
            assert _rel_fro(out[key].cpu().numpy(), ref[key]) <= TOL_MIX, (m.dim, m.order, key)
    b.close()
    for gm in gms:
        gm.close()


@pytest.mark.parametrize("dim,order,n", [(3, 1, 16), (3, 2, 16)])
def test_fp64_two_pass_equals_one_launch(vla, dim, order, n):
    # an FP64 call on a tetrahedral mesh of >= 20,000 elements computes every
    # element's record once and then the tiles (two passes); a batch of that
    # mesh runs the one-launch form: the same bits, pages, volumes and
    # singular count too
    m = meshgen.kuhn_cube(n, jitter=0.1, seed=4) if (dim, order) == (3, 1) else \
        meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=4)
    assert m.ne >= 20000
    gm = _gpu_mesh(vla, m)
    for kind, ca, cb in ((0, 1.0, 1.0), (1, 0.7, 0.3)):
        two = gm.assemble(ca, cb, kind=kind, precision=0, pages=True, count_singular=True)
        jobs = [(gm, gm.outputs(pages=True), kind, ca, cb)]
        b = vla.Batch(jobs, precision=0, count_singular=True)
        b.run()
        torch.cuda.synchronize()
        one = jobs[0][1]
        for key in ("K", "M", "vol", "K3D", "M3D"):
            assert torch.equal(two[key], one[key]), (kind, key)
        assert int(two["n_singular"].item()) == int(b.n_singular.abs().sum().item()) == 0
        b.close()
    ref = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 1.0, 1.0)
    two = gm.assemble(1.0, 1.0, precision=0)
    for key in ("K", "M", "vol"):
        r = ref[key]
        assert np.abs(two[key].cpu().numpy() - r).max() <= TOL64 * np.abs(r).max(), key
    gm.close()


def test_tile_budget_does_not_change_results(vla):
    m = meshgen.kuhn_cube(10, seed=2)
    ref = None
    try:
        for budget in (64, 200, 800, 1200):
            vla.tune_set(3, 1, 1, tile_budget=budget, ctas_per_sm=1 + budget % 3)
            gm = _gpu_mesh(vla, m)
            out = gm.assemble(1.0, 1.0, precision=1)
            if ref is None:
                ref = out
                n_tiles = gm.n_tiles
            else:
                assert torch.equal(out["K"], ref["K"]) and torch.equal(out["M"], ref["M"])
                assert torch.equal(out["vol"], ref["vol"])
        assert gm.n_tiles < n_tiles
    finally:
        vla.tune_set(3, 1, 1, tile_budget=0, ctas_per_sm=0)


@pytest.mark.parametrize("dim,order,n", [(3, 1, 8), (2, 1, 30), (3, 2, 4), (2, 2, 12)])
def test_small_mesh_tiling_does_not_change_results(vla, dim, order, n):
    # under the default budget a small mesh is cut into about two tiles per SM;
    # its outputs equal those of the same mesh cut at the full budget, bit for bit
    m = meshgen.kuhn_cube(n, jitter=0.1, seed=0) if (dim, order) == (3, 1) else \
        meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=3)
    fine = _gpu_mesh(vla, m)
    full_budget = {(2, 1): 2048, (2, 2): 1024, (3, 1): 800, (3, 2): 384}[(dim, order)]
    try:
        vla.tune_set(dim, order, 1, tile_budget=full_budget, ctas_per_sm=0)
        coarse = _gpu_mesh(vla, m)
    finally:
        vla.tune_set(dim, order, 1, tile_budget=0, ctas_per_sm=0)
    assert fine.n_tiles > coarse.n_tiles
    for prec in (0, 1):
        a = fine.assemble(1.0, 1.0, precision=prec, pages=True)
        b = coarse.assemble(1.0, 1.0, precision=prec, pages=True)
        for key in ("K", "M", "vol", "K3D", "M3D"):
            assert torch.equal(a[key], b[key]), (prec, key)
    fine.close()
    coarse.close()


def test_autotune_picks_a_candidate(vla):
    m = meshgen.kuhn_cube(16, seed=0)
    try:
        budget, ctas, us = vla.autotune(_dev(m.coords), _dev(m.elems), order=1, precision=1, reps=3)
        assert budget in (400, 600, 800, 1000, 1200)
        assert ctas in (0, 1, 2, 3, 4)
        assert us > 0
        assert vla.tune_get(3, 1, 1) == (budget, ctas)
        gm = _gpu_mesh(vla, m)   # built with the tuned budget
        out = gm.assemble(1.0, 1.0, precision=1)
        ref = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0)
        assert _rel_fro(out["K"].cpu().numpy(), ref["K"]) <= TOL_MIX
    finally:
        vla.tune_set(3, 1, 1, tile_budget=0, ctas_per_sm=0)


def test_bounded_wait_expiry_is_reported(vla, monkeypatch):
    # a mesh whose kernels may not wait at all: the first wait on a bulk copy
    # runs out, the kernel records it in the error word and returns; the host
    # reads VLA_ERR_TIMEOUT and the context stays usable
    m = meshgen.kuhn_cube(6, seed=5)
    monkeypatch.setenv("VLA_DEBUG_SPIN_LIMIT", "0")
    gm = _gpu_mesh(vla, m)
    monkeypatch.delenv("VLA_DEBUG_SPIN_LIMIT")
    gm.assemble(1.0, 0.0, precision=1)
    with pytest.raises(vla.VlaError) as e:
        gm.check()
    assert e.value.status == -5
    gm.check()   # cleared
    good = _gpu_mesh(vla, m)
    out = good.assemble(1.0, 0.0, precision=1)
    good.check()
    ref = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 0.0)
    assert _rel_fro(out["K"].cpu().numpy(), ref["K"]) <= TOL_MIX
