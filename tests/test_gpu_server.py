"""GPU: the continuous-batching assembly server.

Results must equal vla_assemble on the same mesh bit for bit, whether the
request runs alone or among others (every value's summation order depends
only on its mesh); admission must respect the memory budget; resident meshes
must be reused by key.
"""
import time

import numpy as np
import pytest
import torch

import meshgen
import oracle

pytestmark = pytest.mark.gpu

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


def _single(vla, m, ca, cb, precision=1):
    gm = vla.Mesh(_dev(m.coords), _dev(m.elems), order=m.order)
    out = gm.assemble(ca, cb, precision=precision)
    rp, ci = gm.csr()
    return out, rp, ci


def _wait(srv, t, timeout=60.0):
    res = srv.poll(t, timeout=timeout)
    assert res is not None, "request did not finish"
    return res


def _rel_fro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


MESHES = [(2, 1, 9), (3, 1, 5), (2, 2, 6), (3, 2, 3), (3, 1, 11), (2, 1, 31), (2, 2, 13), (3, 2, 5)]


def test_single_request_matches_assembly_and_oracle(vla):
    m = meshgen.kuhn_cube(6, seed=11)
    srv = vla.Server(1 << 30)
    try:
        t = srv.submit(m.coords, m.elems, order=1, key=1, ca=1.3, cb=0.7)
        res = _wait(srv, t)
        assert res.status == 0 and res.new_mesh == 1 and res.batch_size >= 1
        assert res.t_submit <= res.t_admit <= res.t_ready <= res.t_start <= res.t_done
        got = srv.result(t, res, pattern=True)
        ref, rp, ci = _single(vla, m, 1.3, 0.7)
        assert torch.equal(got["K"], ref["K"]) and torch.equal(got["M"], ref["M"])
        assert torch.equal(got["vol"], ref["vol"])
        assert torch.equal(got["row_ptr"], rp) and torch.equal(got["col_idx"], ci)
        orc = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.3, 0.7)
        assert _rel_fro(got["K"].cpu().numpy(), orc["K"]) <= TOL_MIX
        srv.release(t)
        st = srv.stats()
        assert st["n_done"] == 1 and st["n_resident"] == 1
    finally:
        srv.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_result_same_alone_and_in_the_mix(vla, precision):
    target = meshgen.make_mesh(3, 7, order=2, seed=21)
    others = [meshgen.make_mesh(d, n, order=o, seed=30 + q) for q, (d, o, n) in enumerate(MESHES * 3)]
    srv = vla.Server(4 << 30, precision=precision, ingest_workers=4)
    try:
        t = srv.submit(target.coords, target.elems, order=2, key=-1, ca=0.9, cb=1.1)
        alone = srv.result(t, _wait(srv, t))
        srv.release(t)
        # the same mesh again (a new private copy), among 24 others submitted at once
        tickets = []
        for q, m in enumerate(others[:12]):
            tickets.append((m, 0.5 + q * 0.1, 1.0, srv.submit(m.coords, m.elems, order=m.order, key=-1,
                                                              ca=0.5 + q * 0.1, cb=1.0)))
        tt = srv.submit(target.coords, target.elems, order=2, key=-1, ca=0.9, cb=1.1)
        for q, m in enumerate(others[12:]):
            tickets.append((m, 0.5 + q * 0.1, 1.0, srv.submit(m.coords, m.elems, order=m.order, key=-1,
                                                              ca=0.5 + q * 0.1, cb=1.0)))
        mixed = srv.result(tt, _wait(srv, tt))
        for k in ("K", "M", "vol"):
            assert torch.equal(alone[k], mixed[k]), k
        for m, ca, cb, tk in tickets:
            res = _wait(srv, tk)
            got = srv.result(tk, res)
            ref, _, _ = _single(vla, m, ca, cb, precision)
            assert torch.equal(got["K"], ref["K"]) and torch.equal(got["M"], ref["M"])
            srv.release(tk)
        srv.release(tt)
        st = srv.stats()
        assert st["n_done"] == 2 + len(others) and st["n_failed"] == 0
        assert st["used_bytes"] == 0   # nothing resident (private meshes), every output released
    finally:
        srv.close()


def test_resident_mesh_reused_by_key(vla):
    m = meshgen.unit_square(20, seed=3, order=2)
    srv = vla.Server(1 << 30)
    try:
        t1 = srv.submit(m.coords, m.elems, order=2, key=77, keep_resident=True, ca=1.0, cb=0.0)
        r1 = _wait(srv, t1)
        assert r1.new_mesh == 1
        srv.release(t1)
        # same key, new coefficient: the arrays are not read again (pass garbage to prove it)
        junk_c = np.zeros((1, 2))
        junk_e = np.zeros((1, 6), dtype=np.int32)
        t2 = srv.submit(junk_c, junk_e, order=2, key=77, ca=1.5, cb=0.8)
        r2 = _wait(srv, t2)
        assert r2.new_mesh == 0 and r2.status == 0
        got = srv.result(t2, r2)
        ref, _, _ = _single(vla, m, 1.5, 0.8)
        assert torch.equal(got["K"], ref["K"]) and torch.equal(got["M"], ref["M"])
        srv.release(t2)
        st = srv.stats()
        assert st["n_reused"] == 1 and st["n_ingested"] == 1
    finally:
        srv.close()


def test_budget_admission_and_eviction(vla):
    big = meshgen.kuhn_cube(12, seed=5)       # 10,368 tets
    srv = vla.Server(24 << 20, ingest_workers=2)   # room for a few such meshes only
    try:
        # a request that can never fit fails at admission
        huge = meshgen.kuhn_cube(40, seed=1)
        th = srv.submit(huge.coords, huge.elems, key=-1)
        rh = _wait(srv, th)
        assert rh.status == -6   # VLA_ERR_BUDGET
        srv.release(th)
        tickets = [srv.submit(big.coords, big.elems, key=100 + q, keep_resident=True, ca=1.0 + q)
                   for q in range(10)]
        ref, _, _ = _single(vla, big, 1.0, 0.0)
        for q, t in enumerate(tickets):
            r = _wait(srv, t)
            assert r.status == 0
            got = srv.result(t, r)
            assert _rel_fro(got["K"].cpu().numpy(), (1.0 + q) * ref["K"].cpu().numpy()) <= 1e-6
            srv.release(t)
        st = srv.stats()
        assert st["peak_bytes"] <= st["budget_bytes"]
        assert st["n_evicted"] >= 1   # resident meshes made room for later ones
        assert st["n_failed"] == 1
    finally:
        srv.close()


def test_requests_are_batched(vla):
    meshes = [meshgen.make_mesh(d, n, order=o, seed=q) for q, (d, o, n) in enumerate(MESHES)]
    srv = vla.Server(1 << 30)
    try:
        for q, m in enumerate(meshes):   # make them resident
            t = srv.submit(m.coords, m.elems, order=m.order, key=q)
            _wait(srv, t)
            srv.release(t)
        before = srv.stats()["n_batches"]
        ts = [srv.submit(m.coords, m.elems, order=m.order, key=q % len(meshes), ca=2.0)
              for q, m in enumerate(meshes * 4)]
        rs = [_wait(srv, t) for t in ts]
        assert all(r.status == 0 and r.new_mesh == 0 for r in rs)
        st = srv.stats()
        assert st["n_batches"] - before < len(ts)
        assert max(r.batch_size for r in rs) >= 2
        for t in ts:
            srv.release(t)
    finally:
        srv.close()


def test_poisson_stream_small(vla):
    # the serving workload's shape at small scale: Poisson arrivals, mixed mesh kinds,
    # 20% repeats of a resident mesh with a new coefficient a + b|x|^2
    reqs = meshgen.serving_requests(60, rate_per_s=400.0, lo=1e3, hi=3e4, seed=5)
    cache = {}

    def mesh_of(spec):
        k = (spec["dim"], spec["order"], spec["n"], spec["seed"])
        if k not in cache:
            cache[k] = meshgen.make_mesh(spec["dim"], spec["n"], order=spec["order"], seed=spec["seed"])
        return k, cache[k]

    srv = vla.Server(2 << 30)
    keys = {}
    try:
        t0 = time.monotonic()
        out = []
        for r in reqs:
            k, m = mesh_of(r["mesh"])
            key = keys.setdefault(k, len(keys))
            delay = t0 + r["t_arrival"] - time.monotonic()
            if delay > 0:
                time.sleep(delay)
            a, b = r["coeff"]
            out.append((m, a, b, srv.submit(m.coords, m.elems, order=m.order, key=key, ca=a, cb=b)))
        lat = []
        for m, a, b, t in out:
            res = _wait(srv, t)
            assert res.status == 0
            lat.append(res.t_done - res.t_submit)
            got = srv.result(t, res)
            ref, _, _ = _single(vla, m, a, b)
            assert torch.equal(got["K"], ref["K"]) and torch.equal(got["vol"], ref["vol"])
            srv.release(t)
        assert np.percentile(lat, 99) < 30.0
        assert srv.stats()["n_reused"] >= 1
    finally:
        srv.close()
