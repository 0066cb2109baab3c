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
