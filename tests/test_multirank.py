"""The multi-rank harness of bench.py on CPU: two gloo ranks over 127.0.0.1.

Every rank assembles an independent copy of the workload (no collective on
the data path); only the timing barrier and the max-over-ranks reduction
cross ranks, and the whole-job value counts the units of all ranks.  Under
torchrun the reference arm runs on rank 0 alone and the other ranks exit
without work.
"""
import argparse
import json
import os
import socket
import sys

import pytest

pytestmark = pytest.mark.timeout(300)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws, local = bench._dist()
    assert (r, ws, local) == (rank, 2, rank)
    assert dist.get_backend() == "gloo"
    bench._barrier(dist)
    # rank 1 is the slow one: the job time is its time, the value counts both ranks' units
    ms = bench._max_over_ranks(dist, 3.0 if rank == 1 else 2.0)
    value = bench._job_value(ws, 1000, ms)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value}, f)
    dist.destroy_process_group()


def _reference_worker(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import contextlib
    import io
    import bench
    buf = io.StringIO()
    args = argparse.Namespace(n=3, steps=2, warmup=1)
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(args)
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(f"{rc}\n{buf.getvalue()}")


def _spawn(fn, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(fn, args=(_free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")


def test_two_rank_timing_and_value(tmp_path):
    _spawn(_worker, tmp_path)
    for rank in (0, 1):
        d = json.loads((tmp_path / f"rank{rank}.json").read_text())
        assert d["ms"] == 3.0                      # max over ranks, seen by every rank
        assert d["value"] == pytest.approx(2 * 1000 / 3e-3)


def test_reference_arm_rank0_only(tmp_path):
    pytest.importorskip("numpy")
    _spawn(_reference_worker, tmp_path)
    rc0, out0 = (tmp_path / "ref0.txt").read_text().split("\n", 1)
    rc1, out1 = (tmp_path / "ref1.txt").read_text().split("\n", 1)
    assert rc0 == "0" and rc1 == "0"
    assert out1.strip() == ""                      # rank 1 prints nothing
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2   # the launch it was given; rank 0 does the work
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["value"] > 0 and line["unit"] == "elements/s"


def _block_worker(rank, port, out_dir):
    # each rank owns the rows bench.py would give it, takes the elements with a
    # node in those rows (the halo duplicated) and assembles them with the
    # oracle; rank 0 gathers the row blocks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import bench
    import meshgen
    import oracle
    dist.init_process_group("gloo")
    out = {}
    for name, (dim, order, n) in {"p1tet": (3, 1, 6), "p2tri": (2, 2, 7)}.items():
        m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=5)
        r0, r1 = bench._row_block(m.nn, rank, 2)
        touch = ((m.elems >= r0) & (m.elems < r1)).any(axis=1)
        sub = m.elems[touch]
        ref = oracle.assemble(dim, order, m.nn, sub, m.coords, 0.7, 1.3)
        rp = ref["row_ptr"]
        a, b = rp[r0], rp[r1]
        out[name] = (r0, r1, int(touch.sum()), rp[r0:r1 + 1] - a, ref["col_idx"][a:b], ref["K"][a:b], ref["M"][a:b])
    got = [None, None]
    dist.all_gather_object(got, out)
    if rank == 0:
        import pickle
        with open(os.path.join(out_dir, "blocks.pkl"), "wb") as f:
            pickle.dump(got, f)
    dist.destroy_process_group()


def test_row_blocks_concatenate_to_the_whole_csr(tmp_path):
    import pickle
    import numpy as np
    sys.path.insert(0, ROOT)
    import meshgen
    import oracle
    _spawn(_block_worker, tmp_path)
    blocks = pickle.loads((tmp_path / "blocks.pkl").read_bytes())
    for name, (dim, order, n) in {"p1tet": (3, 1, 6), "p2tri": (2, 2, 7)}.items():
        m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=5)
        whole = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 0.7, 1.3)
        parts = [blocks[r][name] for r in (0, 1)]
        assert parts[0][0] == 0 and parts[0][1] == parts[1][0] and parts[1][1] == m.nn   # the blocks tile the rows
        assert parts[0][2] + parts[1][2] > m.ne                                          # halo elements duplicated
        rp = np.concatenate([parts[0][3], parts[1][3][1:] + parts[0][3][-1]])
        ci = np.concatenate([p[4] for p in parts])
        K = np.concatenate([p[5] for p in parts])
        M = np.concatenate([p[6] for p in parts])
        assert np.array_equal(rp, whole["row_ptr"]) and np.array_equal(ci, whole["col_idx"])
        # the same terms in the same (ascending element) order: the values are the whole-mesh values exactly
        assert np.array_equal(K, whole["K"]) and np.array_equal(M, whole["M"])
