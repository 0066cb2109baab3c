"""Benchmark: P1 tetrahedral stiffness + mass assembly into CSR on the unit cube.

Workload (default): 64^3 cubes x 6 Kuhn tetrahedra = 1,572,864 tets, 274,625
nodes, 4,018,753 CSR nonzeros, interior nodes jittered by U(-0.1h, 0.1h)
(seed 0), coefficient c(x) = 1 + |x|^2 at the element centroid, mixed
precision (FP32 element matrices, compensated determinant and CSR sums, FP64
outputs), plus outward unit normals and areas of the 49,152 boundary
triangles.  One step = vla_assemble_with_boundary (K, M, volumes, and the
boundary facets in the same persistent launch) on a resident mesh.

  value   elements/s over all ranks, inputs resident in HBM, CUDA events
          around each step, L2 flushed (512 MiB write) before every step.
  e2e     the same metric host to host through the public API: pinned host
          coords/elems/faces -> device, mesh build (CSR pattern + tiles),
          assembly, boundary, CSR + values + volumes + normals -> pinned host.
  roofline  the assembly kernel against the measured HBM copy bandwidth, with
          the algorithmic bytes per element of the method (elements 16 B,
          coordinates 24 nn/ne B, element-to-nonzero map 64 B, K and M values
          16 nnz/ne B, volume 8 B) plus 48 B per boundary facet (three node
          indices, the opposite node, normal and area).
  cpu_baseline  the FP64 oracle (plain C) on the same mesh, one host thread
          and all host cores (core count read at run time).
  errors  every output (K, M, volumes, normals, areas) against the FP64
          oracle of the cpu_baseline leg.
  latency p50/p99 of the step over --latency-reps calls: L2 flushed, warm,
          and host call plus synchronize.
  --precision fp64: the plain FP64 form, its roofline against the FP64 pipe
          (cuBLAS DGEMM measured in the same run) beside HBM.

Other workloads (--workload): pages (page primitives at N = 1e8), batch (256
meshes of all four element types in one persistent launch), serve (a Poisson
request stream through the server), next (the rows beyond the assembly core,
one timed call each on the bench mesh), small (p50/p99 latency of the FP64
call with element pages on the 3,072-tet mesh), build (mesh build latency by
size).

Multi-GPU (torchrun): the one mesh is split by rows -- rank r of N owns the
contiguous node rows [nn r / N, nn (r+1) / N) and assembles the sub-mesh of
the elements touching them (halo elements duplicated), which gives it those
rows of K and M complete; no collective on the data path (strong scaling,
value = elements of the whole mesh / slowest rank's step time).  The
reference arm runs on rank 0 alone.  BENCH_DIST_BACKEND=gloo runs the
multi-rank harness without NCCL (ranks may then share a GPU: a functional
check of the row-block path, not a timing).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def _src_hash():
    h = hashlib.sha256()
    for f in ("vla_assemble.cu", "vla_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2404_16039_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_from_profile(kernel_hash):
    p = os.path.join(ROOT, "profiles", "assemble_p1tet64_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def _dist():
    """(dist module or None, rank, world size, local rank) from the torchrun
    environment; NCCL on GPUs, gloo otherwise (the CPU tests of this harness)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        local = int(os.environ.get("LOCAL_RANK", "0"))
        cuda = torch.cuda.is_available()
        if cuda:
            local %= torch.cuda.device_count()   # more ranks than GPUs only in a gloo check of this harness
            torch.cuda.set_device(local)
        # BENCH_DIST_BACKEND=gloo runs the harness without NCCL (a check of the multi-rank path on fewer GPUs)
        dist.init_process_group(os.environ.get("BENCH_DIST_BACKEND") or ("nccl" if cuda else "gloo"))
        return dist, dist.get_rank(), ws, local
    return None, 0, 1, 0


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(ws, units_per_rank, ms):
    """Whole-job throughput: every rank processes units_per_rank in (at most) ms."""
    return ws * units_per_rank / (ms * 1e-3)


def _row_block(nn, rank, ws):
    """The contiguous rows [r0, r1) rank `rank` of `ws` owns."""
    return nn * rank // ws, nn * (rank + 1) // ws


def _alg_bytes_per_el(ne, nn, nnz):
    return 16.0 + 24.0 * nn / ne + 64.0 + 16.0 * nnz / ne + 8.0


FACET_BYTES = 48.0   # a P1 tet boundary facet: 3 node indices + opposite node (16 B), normal + area (32 B)


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(m, seconds=10.0):
    """The oracle as it stands on the same mesh, CSR pattern built once: one
    host thread (orc_assemble), then every host core (the same pinned element
    and scatter steps over element ranges and row blocks, bit-identical
    results).  Also returns the oracle's outputs of the first pass, which the
    error report compares against."""
    import oracle
    pat = oracle.csr_pattern(m.nn, m.elems)
    ref = None
    t0 = time.perf_counter()
    reps = 0
    while True:
        r = oracle.assemble(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0, pattern=pat)
        b = oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
        if ref is None:
            ref = dict(r, normals=b[0], areas=b[1])
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt1 = (time.perf_counter() - t0) / reps
    cores = _host_cores()
    t0 = time.perf_counter()
    reps_n = 0
    while True:
        oracle.assemble_threads(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0, pattern=pat, nthreads=cores)
        oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
        reps_n += 1
        if time.perf_counter() - t0 >= seconds / 2:
            break
    dtn = (time.perf_counter() - t0) / reps_n
    base = {"value": m.ne / dt1, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} full passes of the oracle assembly (K, M, volumes, CSR scatter) plus boundary "
                      f"facets on the same {m.ne}-tet mesh, CSR pattern precomputed, 1 host thread",
            "all_cores": {"value": m.ne / dtn, "unit": "elements/s", "cores": cores,
                          "sample": f"{reps_n} passes, element pages over element ranges and the CSR scatter over "
                                    f"row blocks on {cores} host threads (same results bit for bit), boundary "
                                    f"facets on one"}}
    return base, ref


def _errors(ref, got):
    """Error of every output against the FP64 oracle: K and M entrywise, each
    entry scaled by max(|ref|, max over its row of |ref|), and by relative
    Frobenius norm; volumes and areas relative per entry; unit normals
    absolute per component."""
    rp = ref["row_ptr"]
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    out = {}
    for k in ("K", "M"):
        r, g = ref[k], got[k]
        rowmax = np.zeros(len(rp) - 1)
        np.maximum.at(rowmax, rows, np.abs(r))
        scale = np.maximum(np.abs(r), rowmax[rows])
        out[k] = {"max_entry_rel_rowscale": float((np.abs(g - r) / scale).max()),
                  "rel_fro": float(np.linalg.norm(g - r) / np.linalg.norm(r))}
    for k in ("vol", "areas"):
        r, g = ref[k], got[k]
        out[k] = {"max_rel": float((np.abs(g - r) / np.abs(r)).max()),
                  "rel_fro": float(np.linalg.norm(g - r) / np.linalg.norm(r))}
    r, g = ref["normals"].reshape(-1), got["normals"].reshape(-1)
    out["normals"] = {"max_abs": float(np.abs(g - r).max()), "rel_fro": float(np.linalg.norm(g - r) /
                                                                             np.linalg.norm(r))}
    return out


def _fp64_peak(dev):
    """FP64 throughput of this GPU measured with cuBLAS DGEMM (torch.matmul,
    4096^3, best of 5, CUDA events), GFLOP/s."""
    import torch
    n = 4096
    a = torch.randn((n, n), dtype=torch.float64, device=dev)
    b = torch.randn((n, n), dtype=torch.float64, device=dev)
    c = a @ b
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e9


# FP64 flops one P1 tetrahedron needs in the FP64 form (add, sub, mul, div 1; FMA 2): edge vectors 9,
# centroid 12, cofactors 27, det 5, coefficient 7, scale 2, six stiffness dot products and scalings 36,
# zero-row-sum column and diagonal 8, mass scale 2, volume 1, and 20 CSR additions (10 entries of K and M).
MIXED_LABEL = ("mixed: f32 element matrices; det and inverse in plain f32 where |det| >= perm(|V|)/4 (error <= "
               "11u perm), from error-free float-pair edge vectors with a compensated det below; compensated "
               "float-float CSR sums; f64 outputs")

FP64_FLOPS_PER_TET = 129
FP64_FLOPS_PER_TET_EVAL = 108   # the per-evaluation part, repeated by every row tile an element touches (one-launch form)


def run_reference(args):
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return 0
    import meshgen
    m = meshgen.kuhn_cube(args.n, jitter=0.1, seed=0)
    import oracle
    pat = oracle.csr_pattern(m.nn, m.elems)
    cores = _host_cores()
    per_step = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.assemble_threads(3, 1, m.nn, m.elems, m.coords, 1.0, 1.0, pattern=pat, nthreads=cores)
        oracle.boundary(3, m.nn, m.elems, m.coords, m.faces)
        if i >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    dt = sum(per_step) / len(per_step)
    val = m.ne / dt
    line = {"metric": "elements/sec for P1 tet K+M to CSR", "value": val, "unit": "elements/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(_config(m, "fp64 oracle"),
                           l2=f"host run, no flush: each step reads and writes over "
                              f"{int(_alg_bytes_per_el(m.ne, m.nn, len(pat[1])) * m.ne / 1e6)} MB of mesh "
                              f"arrays and CSR values, more than the host caches hold"),
            "cpu_baseline": {"value": val, "unit": "elements/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step one full oracle pass over the {m.ne}-tet mesh: element pages "
                                       f"over element ranges and the CSR scatter over row blocks on {cores} host "
                                       f"threads, boundary facets on one"},
            "e2e": {"value": val, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(m, precision):
    return {"workload": f"P1 tet K+M -> CSR + boundary normals/areas, unit cube {m.n}^3 cubes x 6 Kuhn tets "
                        f"({m.ne} tets, {m.nn} nodes), interior jitter U(-0.1h,0.1h) seed 0, c(x)=1+|x|^2 "
                        f"at the centroid",
            "ne": m.ne, "nn": m.nn, "nfb": m.nfb, "precision": precision,
            "l2": "flushed before every timed step (512 MiB write)"}


def run_pages(args):
    """Page-primitive sweep (amtam, astam, avtam, amdet, aminv): N pages of n x n,
    FP32/FP64, page-major layout, inputs generated on the device; GB/s of each
    call (bytes the operation must move / CUDA-event time, L2 flushed)."""
    import torch
    import paper_2404_16039_gb300 as vla
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, src = _peaks()
    rows = []
    for N in [int(x) for x in args.pages_n.split(",")]:
        for dt, sz in ((torch.float32, 4), (torch.float64, 8)):
            for n in (2, 3):
                g = torch.Generator(device="cuda").manual_seed(0)
                A = torch.randn((N, n, n), generator=g, dtype=dt, device=dev)
                A[:, list(range(n)), list(range(n))] += 3.0
                B = torch.randn((N, n, n), generator=g, dtype=dt, device=dev)
                s_ = torch.empty(N, dtype=dt, device=dev).uniform_(0.5, 2.0, generator=g)
                v = torch.randn((N, n), generator=g, dtype=dt, device=dev)
                out = torch.empty_like(A)
                det = torch.empty(N, dtype=dt, device=dev)
                y = torch.empty((N, n), dtype=dt, device=dev)
                ops = {
                    "amtam": (lambda: vla.amtam(A, B, out=out), 3 * n * n * sz),
                    "astam": (lambda: vla.astam(s_, A, out=out), (2 * n * n + 1) * sz),
                    "avtam": (lambda: vla.avtam(v, A, out=y), (n * n + 2 * n) * sz),
                    "amdet": (lambda: vla.amdet(A, out=det), (n * n + 1) * sz),
                    "aminv": (lambda: vla.aminv(A, out=out, det=det, count_singular=False), (2 * n * n + 1) * sz),
                }
                for name, (fn, bpp) in ops.items():
                    for _ in range(3):
                        fn()
                    ts = []
                    for _ in range(args.steps):
                        flush.zero_()
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        fn()
                        b.record()
                        torch.cuda.synchronize()
                        ts.append(a.elapsed_time(b))
                    ms = float(np.median(ts))
                    gbs = N * bpp / (ms * 1e-3) / 1e9
                    rows.append({"op": name, "n": n, "dtype": "f32" if sz == 4 else "f64", "N": N, "ms": ms,
                                 "GBps": gbs, "frac_hbm": gbs / peaks["hbm_gbs"]})
                del A, B, out, det, y, s_, v
                torch.cuda.empty_cache()
    print(json.dumps({"workload": "page primitives, page-major layout", "peak_hbm_gbs": peaks["hbm_gbs"],
                      "peak_source": src, "results": rows}), flush=True)
    return 0


def _nlb(dim, order):
    return dim + 1 if order == 1 else (dim + 1) * (dim + 2) // 2


def _alg_bytes_mesh(dim, order, ne, nn, nnz):
    """Bytes the method must move for one assembly of a mesh: elements (4 nlb),
    coordinates (8 dim per node), element-to-nonzero map (4 nlb^2), K and M
    values (16 per nonzero), volumes (8)."""
    nlb = _nlb(dim, order)
    return (4 * nlb + 4 * nlb * nlb + 8) * ne + 8 * dim * nn + 16 * nnz


def _time_steps(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_batch(args):
    """Batched uneven assembly: 256 meshes (2-D/3-D x P1/P2, element counts
    log-uniform in [1e3, 1e6]) in one persistent, graph-captured launch, tile
    budget and CTA residency autotuned per element type."""
    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla
    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    specs = meshgen.batch_specs(args.batch_count, args.batch_lo, args.batch_hi, seed=0)
    meshes = [meshgen.make_mesh(s["dim"], s["n"], order=s["order"], jitter=0.1, seed=s["seed"]) for s in specs]
    gen_s = time.perf_counter() - t0
    print(f"generated {len(meshes)} meshes in {gen_s:.1f} s", file=sys.stderr, flush=True)
    tuned = {}
    for dim, order in ((2, 1), (2, 2), (3, 1), (3, 2)):
        cand = [m for m in meshes if (m.dim, m.order) == (dim, order) and m.ne <= 300000]
        smp = max(cand, key=lambda m: m.ne) if cand else meshgen.make_mesh(dim, 8, order=order)
        b, c, us = vla.autotune(torch.from_numpy(smp.coords).to(dev), torch.from_numpy(smp.elems).to(dev),
                                order=order, precision=vla.PREC_MIXED, reps=3)
        tuned[f"{dim}d_p{order}"] = {"tile_budget": b, "ctas_per_sm": c, "sample_ne": smp.ne, "sample_us": us}
    t0 = time.perf_counter()
    gms = [vla.Mesh(torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.elems).to(dev), order=m.order)
           for m in meshes]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    ne = sum(g.ne for g in gms)
    alg = sum(_alg_bytes_mesh(g.dim, g.order, g.ne, g.nn, g.nnz) for g in gms)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out_mix = [g.outputs() for g in gms]
    out_64 = [g.outputs() for g in gms]
    bm = vla.Batch([(g, o, vla.COEFF_POLY, 1.0, 1.0) for g, o in zip(gms, out_mix)], precision=vla.PREC_MIXED,
                   graph=True, tune=args.batch_form == "auto",
                   form=None if args.batch_form == "auto" else args.batch_form)
    b64 = vla.Batch([(g, o, vla.COEFF_POLY, 1.0, 1.0) for g, o in zip(gms, out_64)], precision=vla.PREC_FP64,
                    graph=True, tune=True)
    forms = {}
    for form in ("fused", "split"):
        bf = vla.Batch([(g, o, vla.COEFF_POLY, 1.0, 1.0) for g, o in zip(gms, out_mix)], precision=vla.PREC_MIXED,
                       graph=True, form=form)
        forms[form] = float(np.median(_time_steps(bf.run, max(3, args.steps // 4), 3, flush,
                                                  torch.cuda.current_stream())))
        bf.close()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    _barrier(dist)
    sampler.start()
    time.sleep(0.3)
    ms_mix = _time_steps(bm.run, args.steps, args.warmup, flush, stream)
    clocks = sampler.stop()
    ms_64 = _time_steps(b64.run, max(3, args.steps // 4), 3, flush, stream)

    def loop():   # the same work as one launch per mesh
        for g, o in zip(gms, out_mix):
            g.assemble(1.0, 1.0, precision=vla.PREC_MIXED, K=o["K"], M=o["M"], vol=o["vol"])

    ms_loop = _time_steps(loop, max(3, args.steps // 4), 3, flush, stream)
    bm.check()
    b64.check()
    # accuracy of the mixed form against the FP64 form (itself within 1e-12 of the FP64 oracle)
    err = {"K": 0.0, "M": 0.0, "vol": 0.0}
    for a, b in zip(out_mix, out_64):
        for k in err:
            d = torch.linalg.vector_norm(a[k] - b[k]).item() / max(torch.linalg.vector_norm(b[k]).item(), 1e-300)
            err[k] = max(err[k], d)
    ms = _max_over_ranks(dist, float(np.median(ms_mix)))
    value = _job_value(ws, ne, ms)
    peaks, src = _peaks()
    achieved = alg / (float(np.median(ms_mix)) * 1e-3) / 1e9

    # end to end: pinned host meshes -> device, mesh builds, one-shot batch, K/M/vol -> pinned host
    hin = [(torch.from_numpy(m.coords).pin_memory(), torch.from_numpy(m.elems).pin_memory()) for m in meshes]
    hout = [{k: torch.empty(g.nnz if k != "vol" else g.ne, dtype=torch.float64).pin_memory()
             for k in ("K", "M", "vol")} for g in gms]
    h2d = sum(c.numel() * 8 + e.numel() * 4 for c, e in hin)
    d2h = sum(sum(t.numel() * 8 for t in o.values()) for o in hout)

    def e2e_step():
        ms_ = []
        for (c, e), m in zip(hin, meshes):
            ms_.append(vla.Mesh(c.to(dev, non_blocking=True), e.to(dev, non_blocking=True), order=m.order))
        outs = [g.outputs() for g in ms_]
        vla.batch_assemble([(g, o, vla.COEFF_POLY, 1.0, 1.0) for g, o in zip(ms_, outs)], precision=vla.PREC_MIXED)
        for o, h in zip(outs, hout):
            for k in h:
                h[k].copy_(o[k], non_blocking=True)
        torch.cuda.synchronize()
        for g in ms_:
            g.close()

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    e2e_s = _max_over_ranks(dist, (time.perf_counter() - t0) / args.e2e_steps)
    kinds = {}
    for g in gms:
        k = f"{g.dim}d_p{g.order}"
        kinds.setdefault(k, {"meshes": 0, "elements": 0, "max_smem": 0, "min_budget": 1 << 30})
        kinds[k]["meshes"] += 1
        kinds[k]["elements"] += g.ne
        kinds[k]["max_smem"] = max(kinds[k]["max_smem"], g.smem_bytes)
        kinds[k]["min_budget"] = min(kinds[k]["min_budget"], g.tile_budget)
    line = {"metric": "elements/sec for batched uneven K+M to CSR (one persistent launch)", "value": value,
            "unit": "elements/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{len(gms)} meshes from seed 0: 2-D unit-square triangles and 3-D Kuhn unit-cube "
                                   f"tets, half P1 half P2, element counts log-uniform in [{args.batch_lo:g}, "
                                   f"{args.batch_hi:g}] rounded to the structured n, interior jitter 0.1h, "
                                   f"c(x)=1+|x|^2",
                       "meshes": len(gms), "elements": ne, "nnz": sum(g.nnz for g in gms), "by_kind": kinds,
                       "precision": MIXED_LABEL,
                       "launch": ("one persistent kernel per element type" if bm.split else
                                  "one persistent kernel over the row tiles of every mesh") +
                                 ", captured in one CUDA graph" + ("; form chosen by timing both at creation"
                                                                    if args.batch_form == "auto" else ""),
                       "form_ms": forms,
                       "autotuned": tuned, "grid": bm.grid, "work_items": bm.n_work,
                       "smem_per_cta": bm.smem_bytes,
                       "l2": "flushed before every timed step (512 MiB write)"},
            "e2e": {"value": ws * ne / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "includes": "H2D of every mesh's coords/elems, mesh builds (patterns, tiles), one batched "
                                "launch, D2H of K/M/vol"},
            "roofline": {"bound": "hbm", "kernel": "k_assemble<mixed, all types, batched>", "achieved": achieved,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                         "peak_source": src, "traffic": None, "alg_bytes_per_launch": alg},
            "fp64_form": {"ms_per_step": float(np.median(ms_64)), "value": ne / (float(np.median(ms_64)) * 1e-3),
                          "note": "the same batch computed entirely in FP64 on the same GPU"},
            "mixed_vs_fp64_max_rel_fro": err,
            "unbatched_loop": {"ms_per_step": float(np.median(ms_loop)),
                               "value": ne / (float(np.median(ms_loop)) * 1e-3),
                               "note": "one vla_assemble launch per mesh, same outputs"},
            "mesh_build_s": build_s, "gpu_launches": args.steps * (sum(1 for k in kinds) if bm.split else 1),
            "clocks": clocks,
            "p50_ms": float(np.percentile(ms_mix, 50)), "p99_ms": float(np.percentile(ms_mix, 99))}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        done = 0
        order_ = sorted(range(len(meshes)), key=lambda i: meshes[i].ne)
        used = 0
        for i in order_:
            m = meshes[i]
            oracle.assemble(m.dim, m.order, m.nn, m.elems, m.coords, 1.0, 1.0)
            done += m.ne
            used += 1
            if time.perf_counter() - t0 >= args.cpu_seconds:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle assembly (pattern, K, M, volumes) of the {used} smallest meshes "
                                          f"of the batch ({done} elements), 1 host thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for b in (bm, b64):
        b.close()
    for g in gms:
        g.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Serving: a Poisson stream of assembly requests (2-D/3-D, P1/P2, element
    counts log-uniform in [1e3, 2e6], 20% repeating a resident mesh with a new
    coefficient a + b|x|^2) against a 100 GB device budget; continuous
    batching.  The sustained rate is measured closed-loop first, then the
    stream runs at 0.5x, 0.8x and 1.0x of it; the FP64 form is measured the
    same way at 0.8x of its own sustained rate."""
    import threading
    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla
    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.requests
    base = meshgen.serving_requests(N, rate_per_s=1.0, lo=1e3, hi=2e6, seed=0, size_levels=args.size_levels)
    t0 = time.perf_counter()
    cache = {}
    for r in base:
        s = r["mesh"]
        k = (s["dim"], s["order"], s["n"])
        if k not in cache:
            cache[k] = meshgen.make_mesh(s["dim"], s["n"], order=s["order"], jitter=0.1, seed=s["n"])
    gen_s = time.perf_counter() - t0
    print(f"generated {len(cache)} distinct meshes for {N} requests in {gen_s:.1f} s", file=sys.stderr, flush=True)
    # the client's inputs live in pinned host memory
    pinned = {k: (torch.from_numpy(m.coords).pin_memory(), torch.from_numpy(m.elems).pin_memory(), m.order, m.ne)
              for k, m in cache.items()}
    keys = {}
    reqs = []
    for r in base:
        s = r["mesh"]
        key = keys.setdefault((s["dim"], s["order"], s["n"], s["seed"]), len(keys))
        reqs.append((r["t_arrival"], key, pinned[(s["dim"], s["order"], s["n"])], r["coeff"]))
    n_poll = args.pollers
    hosts = [[torch.empty(1 << 20, dtype=torch.float64).pin_memory()] for _ in range(n_poll)]   # grown on demand

    def run(precision, rate, count, closed=False):
        srv = vla.Server(args.budget_gb << 30, precision=precision, ingest_workers=args.ingest_workers)
        sub = reqs[:count]
        tickets = [None] * count
        t_arr = [0.0] * count
        lat = [None] * count
        lat_host = [None] * count
        els = [0] * count
        bsz = [0] * count
        phases = [None] * count
        ingest = [None] * count
        fails = {}
        h2d = [0]
        d2h = [0] * n_poll
        lock = threading.Lock()

        def poller(p):   # requests p, p + n_poll, ...: wait, copy K/M/vol to pinned host memory, release
            host = hosts[p]
            for i in range(p, count, n_poll):
                while tickets[i] is None:
                    time.sleep(0.0002)
                res = None
                while res is None:
                    res = srv.poll(tickets[i], timeout=1.0)
                if res.status == 0:
                    n = res.nnz
                    if host[0].numel() < n:
                        host[0] = torch.empty(2 * n, dtype=torch.float64).pin_memory()
                    for ptr, cnt in ((res.K_vals, n), (res.M_vals, n), (res.vol, res.ne)):
                        host[0][:cnt].copy_(vla._view(ptr, cnt, "<f8", dev))
                        d2h[p] += 8 * cnt
                    th = time.monotonic()
                    phases[i] = (res.t_admit - res.t_submit, res.t_ready - res.t_admit, res.t_start - res.t_ready,
                                 res.t_done - res.t_start, th - res.t_done)
                    if res.new_mesh:
                        ingest[i] = (res.t_ingest - res.t_admit, res.h2d_ms * 1e-3, res.build_ms * 1e-3,
                                     res.t_ready - res.t_ingest - (res.h2d_ms + res.build_ms) * 1e-3)
                    lat[i] = res.t_done - t_arr[i]
                    lat_host[i] = th - t_arr[i]
                    els[i] = res.ne
                    bsz[i] = res.batch_size
                else:
                    with lock:
                        fails[int(res.status)] = fails.get(int(res.status), 0) + 1
                srv.release(tickets[i])

        ths = [threading.Thread(target=poller, args=(p,)) for p in range(n_poll)]
        for t_ in ths:
            t_.start()
        start = time.monotonic() + 0.05
        for i, (ta, key, (c, e, order, ne), (a, b)) in enumerate(sub):
            t_arr[i] = start if closed else start + ta / rate
            d = t_arr[i] - time.monotonic()
            if d > 0:
                time.sleep(d)
            tickets[i] = srv.submit(c, e, order=order, key=key, keep_resident=True, kind=vla.COEFF_POLY, ca=a, cb=b)
            h2d[0] += c.numel() * 8 + e.numel() * 4
        for t_ in ths:
            t_.join()
        st = srv.stats()
        srv.close()
        ok = [i for i in range(count) if lat[i] is not None]
        L = np.array([lat[i] for i in ok])
        LH = np.array([lat_host[i] for i in ok])
        wall = max(t_arr[i] + lat_host[i] for i in ok) - start
        ne_ok = int(sum(els[i] for i in ok))
        return {"requests": count, "completed": len(ok), "failed": st["n_failed"], "fail_status": fails,
                "elements": ne_ok, "wall_s": wall, "elements_per_s": ne_ok / wall, "requests_per_s": len(ok) / wall,
                "p50_ms": 1e3 * float(np.percentile(L, 50)), "p99_ms": 1e3 * float(np.percentile(L, 99)),
                "p50_ms_to_host": 1e3 * float(np.percentile(LH, 50)),
                "p99_ms_to_host": 1e3 * float(np.percentile(LH, 99)),
                "mean_batch": float(np.mean([bsz[i] for i in ok])), "max_batch": int(max(bsz[i] for i in ok)),
                "mean_phase_ms": dict(zip(("queued", "ingest", "wait_launch", "assembly", "copy_out"),
                                          (1e3 * float(np.mean([phases[i][c] for i in ok])) for c in range(5)))),
                "ingest_split_ms": dict(zip(("wait_for_ingest_thread", "h2d_device", "build_device",
                                             "build_host_rest"),
                                            (1e3 * float(np.mean([ingest[i][c] for i in ok if ingest[i]]))
                                             for c in range(4)))) if any(ingest[i] for i in ok) else None,
                "batches": st["n_batches"], "ingested": st["n_ingested"], "reused": st["n_reused"],
                "evicted": st["n_evicted"], "peak_bytes": st["peak_bytes"], "h2d_bytes": h2d[0], "d2h_bytes": sum(d2h)}

    calib = min(N, args.calib_requests)
    sus = run(vla.PREC_MIXED, 1.0, calib, closed=True)
    rate0 = sus["requests_per_s"]
    print(f"sustained (closed loop, {calib} requests): {rate0:.1f} req/s", file=sys.stderr, flush=True)
    sampler = ClockSampler(local)
    sampler.start()
    runs = {}
    for f in args.rate_fracs:
        runs[f"{f:g}x"] = dict(run(vla.PREC_MIXED, f * rate0, N), rate_per_s=f * rate0)
        print(f"{f:g}x: {json.dumps(runs[f'{f:g}x'])}", file=sys.stderr, flush=True)
    clocks = sampler.stop()
    sus64 = run(vla.PREC_FP64, 1.0, calib, closed=True)
    r64 = dict(run(vla.PREC_FP64, 0.8 * sus64["requests_per_s"], N), rate_per_s=0.8 * sus64["requests_per_s"])
    head = runs[f"{args.rate_fracs[-1]:g}x"]
    line = {"metric": "serving: elements/sec and p50/p99 latency of K+M+vol requests", "value": head["elements_per_s"],
            "unit": "elements/s", "n_gpus": ws, "steps": N, "warmup": 0, "ms_per_step": 1e3 * head["wall_s"] / N,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Poisson stream of {N} assembly requests (seed 0): 2-D/3-D x P1/P2 meshes with "
                                   f"element counts log-uniform in [1e3, 2e6] (snapped to {args.size_levels} sizes "
                                   f"per decade), 20% repeating a resident mesh with c(x)=a+b|x|^2, a,b~U(0.5,2)",
                       "budget_gb": args.budget_gb, "ingest_workers": args.ingest_workers,
                       "client": f"inputs in pinned host memory, {n_poll} client threads copying results to pinned "
                                 f"host memory",
                       "rates": "fractions of the sustained closed-loop rate", "sustained_req_per_s": rate0,
                       "precision": "mixed", "results": "K, M, vol copied to pinned host memory by the client"},
            "latency": {"p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
                        "p50_ms_to_host": head["p50_ms_to_host"], "p99_ms_to_host": head["p99_ms_to_host"]},
            "runs": runs, "closed_loop": sus, "fp64_form": {"closed_loop": sus64, "at_0.8x": r64},
            "e2e": {"value": head["elements_per_s"], "unit": "elements/s",
                    "h2d_bytes_per_step": int(head["h2d_bytes"] / N), "d2h_bytes_per_step": int(head["d2h_bytes"] / N),
                    "note": "the serving measurement is end to end: host arrays in, host results out"},
            "gpu_launches": None, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_build(args):
    """Mesh build latency by size: `vla_mesh_create` (validation, CSR pattern,
    row tiles; synchronous) on device-resident inputs, for P1/P2 triangles and
    tetrahedra from hundreds to 1.57 M elements.  Per size one untimed build,
    then the median and maximum of --build-reps builds by the host clock
    around the call (the call synchronises).  `value` is the median for the
    bench mesh (64^3 x 6 Kuhn tets).  VLA_POOL_KEEP (bytes of freed device
    memory the library keeps mapped between calls) is reported as set."""
    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cases = [(3, 1, 5), (3, 1, 12), (3, 1, 25), (3, 1, 50), (3, 1, 64), (3, 2, 6), (3, 2, 20), (2, 1, 30),
             (2, 1, 300), (2, 2, 100)]
    rows, value = [], None
    for dim, order, n in cases:
        m = meshgen.kuhn_cube(n, jitter=0.1, seed=0) if (dim, order) == (3, 1) else \
            meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=1)
        c, e = torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.elems).to(dev)
        f = torch.from_numpy(m.faces).to(dev) if m.nfb else None
        ts = []
        for r in range(args.build_reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = vla.Mesh(c, e, f, order=order)
            ts.append((time.perf_counter() - t0) * 1e3)
            g.close()
        ts = ts[1:]
        row = {"dim": dim, "order": order, "ne": int(m.ne), "nn": int(m.nn), "median_ms": float(np.median(ts)),
               "max_ms": float(np.max(ts))}
        rows.append(row)
        if (dim, order, n) == (3, 1, 64):
            value = row["median_ms"]
        print(json.dumps(row), file=sys.stderr, flush=True)
    line = {"metric": "mesh build latency (vla_mesh_create) of the 64^3 x 6 Kuhn cube", "value": value, "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.build_reps, "warmup": 1, "data": "synthetic",
            "config": {"workload": "vla_mesh_create on device-resident inputs, sizes " +
                                   ", ".join(f"{r['ne']} {'tets' if r['dim'] == 3 else 'triangles'} P{r['order']}"
                                             for r in rows),
                       "pool_keep_bytes": os.environ.get("VLA_POOL_KEEP", "default (min(8 GiB, HBM/16))")},
            "sizes": rows}
    print(json.dumps(line), flush=True)


def run_small(args):
    """The small FP64 case with element pages: Kuhn 8^3 x 6 (3,072 tets, 729
    nodes), c = 1, K, M, volumes and both page arrays in FP64 from one call,
    a latency-bound call.  Reports p50/p99 over --small-reps calls of the
    device time between CUDA events around the call with the L2 flushed
    before each (cold), the same back to back (warm), and the host wall time
    of the call plus a synchronize."""
    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m = meshgen.kuhn_cube(8, jitter=0.1, seed=0)
    gm = vla.Mesh(torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.elems).to(dev),
                  torch.from_numpy(m.faces).to(dev))
    K = torch.empty(gm.nnz, dtype=torch.float64, device=dev)
    M = torch.empty_like(K)
    vol = torch.empty(gm.ne, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        gm.assemble(1.0, 0.0, precision=vla.PREC_FP64, K=K, M=M, vol=vol, pages=True)

    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()

    def device_ms(flushed):
        ts = []
        for _ in range(args.small_reps):
            if flushed:
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    sampler = ClockSampler(0)
    sampler.start()
    cold = device_ms(True)
    warm = device_ms(False)
    host = []
    for _ in range(args.small_reps):
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        host.append((time.perf_counter() - t0) * 1e3)
    clocks = sampler.stop()

    def pct(x):
        return {"p50_ms": float(np.percentile(x, 50)), "p99_ms": float(np.percentile(x, 99))}

    line = {"metric": "latency of one FP64 P1 tet K+M call with element pages", "value": pct(cold)["p50_ms"],
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": args.small_reps, "warmup": warmup,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"P1 tet K+M -> CSR with K3D/M3D pages, FP64, unit cube 8^3 cubes x 6 Kuhn "
                                   f"tets ({gm.ne} tets, {gm.nn} nodes, {gm.nnz} nonzeros), interior jitter "
                                   f"U(-0.1h,0.1h) seed 0, c = 1",
                       "l2": "cold: flushed before every call (512 MiB write); warm: back to back"},
            "cold_l2": pct(cold), "warm_l2": pct(warm), "host_call_and_sync": pct(host), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_next(args):
    """The rows beyond the assembly core, each timed on the bench mesh (CUDA
    events around one call, L2 flushed before each, median of 20 after 3
    warm-ups): literal-quadrature assembly, facet list, quadrature points, GI
    integrals, load vector, local energies and avtamav; then the remaining
    page functions of Section 2.4 on 1e7 FP32 pages.  Algorithmic bytes:
    what each call must read and write once (stated per row); achieved =
    bytes / time against the measured HBM copy bandwidth."""
    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m = meshgen.kuhn_cube(args.n, jitter=0.1, seed=0)
    gm = vla.Mesh(torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.elems).to(dev),
                  torch.from_numpy(m.faces).to(dev))
    ne, nn, nnz, nfb = gm.ne, gm.nn, gm.nnz, gm.nfb
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, src = _peaks()
    hbm = peaks["hbm_gbs"]
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            flush.zero_()
            fn()
        ts = []
        for _ in range(20):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    fp64_peak = 1250.0   # GFLOP/s, the GB300's nominal dense FP64 rate (a probe measured ~1,000)

    def row(ms, units, unit, nbytes, what, fp64_flops=None, flops_what=None):
        g = nbytes / (ms * 1e-3) / 1e9
        r = {"ms": ms, "throughput": units / (ms * 1e-3), "unit": unit, "alg_bytes": int(nbytes),
             "achieved_gbs": g, "frac_of_measured_hbm": g / hbm, "bytes": what, "bound": "hbm"}
        if fp64_flops is not None:
            f = fp64_flops / (ms * 1e-3) / 1e9
            r.update({"fp64_gflops": f, "frac_of_nominal_fp64": f / fp64_peak, "flops": flops_what})
            if f / fp64_peak > g / hbm:
                r["bound"] = "fp64"
        return r

    sampler = ClockSampler(0)
    sampler.start()
    rows = {}
    K = torch.empty(nnz, dtype=torch.float64, device=dev)
    M = torch.empty_like(K)
    vol = torch.empty(ne, dtype=torch.float64, device=dev)
    bpe = _alg_bytes_per_el(ne, nn, nnz)
    for name, kind in (("assembly_centroid_coefficient", vla.COEFF_POLY),
                       ("f1_literal_quadrature_assembly", vla.COEFF_POLY_IP)):
        ms = timed(lambda: gm.assemble(1.0, 1.0, kind=kind, precision=vla.PREC_MIXED, K=K, M=M, vol=vol))
        rows[name] = row(ms, ne, "elements/s", bpe * ne, "as the main bench line (elements, coordinates, "
                         "element-to-nonzero map, K and M, volumes)")
    faces, owner, nbr, nb = gm.facets()
    nf = faces.shape[0]
    ms = timed(lambda: gm.facets())
    rows["f2_facet_list"] = row(ms, nf, "facets/s", 16 * ne + 8 * 4 * ne + nf * (12 + 8 + 4),
                                "elements 16 B and their incidence lists (4 x 8 B) per element; per facet "
                                "3 vertices, owner pair and neighbour")
    rows["f2_facet_list"]["bound"] = "latency (integer search of incidence lists; two calls: count, then fill)"
    ip, w = vla.quad_rule(3, 3)
    nip = len(w)
    X = gm.quad_points(3)
    ms = timed(lambda: gm.quad_points(3))
    rows["f4_quadrature_points_degree3"] = row(ms, ne * nip, "points/s", 16 * ne + 24 * nn + 24 * ne * nip,
                                               "elements 16 B, coordinates 24 B per node, 3 doubles per point",
                                               2.0 * ne * nip * 4 * 3, "4 vertices x 3 coordinates FMA per point")
    rho = (1.0 + X[..., 0] ** 2)[..., None].contiguous()
    gm.assemble(1.0, 1.0, precision=vla.PREC_FP64, K=K, M=M, vol=vol)
    ms = timed(lambda: vla.gi(rho, w, vol))
    rows["f4_gi_integral_degree3"] = row(ms, ne * nip, "points/s", 8 * ne * nip + 8 * ne,
                                         "one double per point and the element measure",
                                         2.0 * ne * nip + 2.0 * ne, "weight FMA per point, measure per element")
    ip2, w2 = vla.quad_rule(3, 2)
    f = torch.ones((ne, len(w2)), dtype=torch.float64, device=dev)
    b = torch.empty(nn, dtype=torch.float64, device=dev)
    b2D = torch.empty((ne, 4), dtype=torch.float64, device=dev)
    ms = timed(lambda: gm.rhs(2, f, b=b, b2D=b2D))
    rows["f3_load_vector_degree2"] = row(ms, ne, "elements/s", 8 * ne * len(w2) + 16 * ne + 24 * nn + 32 * ne
                                         + 8 * nn + 64 * ne,
                                         "f at the points, elements, coordinates, b2D, b, and the node "
                                         "gather's incidence lists (4 x 16 B per element)",
                                         (35.0 + 4 * len(w2) * 3 + 4 + 4) * ne,
                                         "measure ~35, 3 per point and basis function, scaling, gather adds")
    pg = gm.assemble(1.0, 1.0, precision=vla.PREC_FP64, pages=True)
    u = torch.from_numpy(m.coords[:, 0].copy()).to(dev)
    J = torch.empty((ne, 3), dtype=torch.float64, device=dev)
    ms = timed(lambda: gm.energies(u, pg["K3D"], pg["M3D"], b2D))
    rows["f3_local_energies"] = row(ms, ne, "elements/s", 2 * 128 * ne + 32 * ne + 16 * ne + 8 * nn + 24 * ne,
                                    "K3D and M3D pages (2 x 128 B), b2D, elements, u, J (3 doubles)",
                                    88.0 * ne, "K u and M u (2 x 16 FMA), two dots and b.u per element")
    v4 = torch.randn((ne, 4), dtype=torch.float64, device=dev)
    A4 = pg["K3D"]
    ms = timed(lambda: vla.avtamav(v4, A4, v4))
    rows["f3_avtamav_4x4_fp64"] = row(ms, ne, "pages/s", ne * 8 * (4 + 16 + 4 + 1), "v, A, w and the result",
                                      40.0 * ne, "A w (16 FMA) and v.(A w) (4 FMA) per page")
    # the remaining page functions of Section 2.4, FP32 page layout, 1e7 pages
    NP = 10_000_000
    g = torch.Generator(device=dev).manual_seed(0)
    A33 = torch.randn((NP, 3, 3), generator=g, device=dev)
    A45 = torch.randn((NP, 4, 3), generator=g, device=dev)        # pages 3 x 4
    v3 = torch.randn((NP, 3), generator=g, device=dev)
    S = torch.randn((5, 4), generator=g, device=dev)              # 4 x 5
    Sp = torch.randn((4, 3), generator=g, device=dev)             # 3 x 4
    s4 = torch.randn(4, generator=g, device=dev)
    for name, fn, nbytes, what in (
            ("pages_amt_3x3_f32", lambda: vla.amt(A33), NP * 72, "read 9 and write 9 floats"),
            ("pages_avtav_3_f32", lambda: vla.avtav(v3, v3), NP * 28, "read 2 x 3 floats (the same array), write 1"),
            ("pages_amsm_3x4_by_4x5_f32", lambda: vla.amsm(A45, S), NP * 108, "read 12, write 15 floats"),
            ("pages_amsv_3x4_f32", lambda: vla.amsv(A45, s4), NP * 60, "read 12, write 3 floats"),
            ("pages_smamt_3x4_by_3x4_f32", lambda: vla.smamt(Sp, A45), NP * 84,
             "read 12, write 9 floats (tjac = smamt(dshape, coords3D))"),
            ("pages_svamt_3x4_f32", lambda: vla.svamt(s4, A45), NP * 60, "read 12, write 3 floats")):
        ms = timed(fn)
        rows[name] = row(ms, NP, "pages/s", nbytes, what)
    del A33, A45, v3
    clocks = sampler.stop()
    line = {"metric": "rows beyond the assembly core, timed on the bench mesh", "unit": "per row",
            "n_gpus": 1, "workload": "unit cube %d^3 cubes x 6 Kuhn tets (%d tets, %d nodes, %d nonzeros, %d boundary "
            "facets), interior jitter 0.1h seed 0" % (args.n, ne, nn, nnz, nfb), "peak_gbs": hbm,
            "peak_source": src, "l2": "flushed before every timed call (512 MiB write)", "rows": rows,
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    gm.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vla", choices=["vla", "reference"])
    ap.add_argument("--n", type=int, default=64, help="cubes per side")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="p1tet", choices=["p1tet", "pages", "batch", "serve", "next", "small", "build"])
    ap.add_argument("--build-reps", type=int, default=5)
    ap.add_argument("--small-reps", type=int, default=1000)
    ap.add_argument("--latency-reps", type=int, default=1000)
    ap.add_argument("--pages-n", default="100000000")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-lo", type=float, default=1e3)
    ap.add_argument("--batch-hi", type=float, default=1e6)
    ap.add_argument("--batch-form", default="auto", choices=["auto", "fused", "split"])
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--calib-requests", type=int, default=3000)
    ap.add_argument("--pollers", type=int, default=4)
    ap.add_argument("--size-levels", type=int, default=16)
    ap.add_argument("--budget-gb", type=int, default=100)
    ap.add_argument("--ingest-workers", type=int, default=4)
    ap.add_argument("--rate-fracs", type=float, nargs="+", default=[0.5, 0.8, 1.0])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "pages":
        return run_pages(args)
    if args.workload == "batch":
        if "--e2e-steps" not in sys.argv:
            args.e2e_steps = 1
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "next":
        return run_next(args)
    if args.workload == "small":
        return run_small(args)
    if args.workload == "build":
        return run_build(args)

    import torch
    import meshgen
    import paper_2404_16039_gb300 as vla

    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = vla.PREC_MIXED if args.precision == "mixed" else vla.PREC_FP64
    m = meshgen.kuhn_cube(args.n, jitter=0.1, seed=0)
    coords = torch.from_numpy(m.coords).to(dev)
    elems = torch.from_numpy(m.elems).to(dev)
    faces = torch.from_numpy(m.faces).to(dev)
    # one row block per rank (strong scaling: the one mesh split by rows, halo elements duplicated,
    # complete rows per rank, no collective on the data path); one rank takes every row
    blk = _row_block(m.nn, rank, ws)
    gm = vla.Mesh(coords, elems, faces, rows=None if ws == 1 else blk)
    K = torch.empty(gm.nnz, dtype=torch.float64, device=dev)
    M = torch.empty(gm.nnz, dtype=torch.float64, device=dev)
    vol = torch.empty(gm.ne, dtype=torch.float64, device=dev)
    nrm = torch.empty((gm.nfb, 3), dtype=torch.float64, device=dev)
    ar = torch.empty(gm.nfb, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        gm.assemble(1.0, 1.0, precision=prec, K=K, M=M, vol=vol, boundary=True, normals=nrm, areas=ar)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the clock sampler starts first; the warm-up steps then run right before
    # the timed ones (a GPU left idle while the sampler starts slows the first
    # timed step by up to 70 us)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    _barrier(dist)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        e0, e1 = ev[i]
        e0.record(stream)
        step()   # one launch: the assembly kernel with the boundary facets after its tiles
        e1.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = _max_over_ranks(dist, sum(step_ms) / len(step_ms))
    asm = sum(step_ms) / len(step_ms)   # this rank's kernel time (the step is that one launch)
    value = m.ne / (ms * 1e-3)   # every element of the one mesh, over the slowest rank's time

    # latency of the hot step over --latency-reps calls: device time with the L2
    # flushed before each (cold) and back to back (warm), and the host time of
    # the call plus a synchronize
    def _lat(flushed):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.latency_reps)]
        for a, b in evs:
            if flushed:
                flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def _pct(x):
        return {"p50_ms": float(np.percentile(x, 50)), "p99_ms": float(np.percentile(x, 99)), "reps": len(x)}

    lat_cold = _lat(True)
    lat_warm = _lat(False)
    host = []
    for _ in range(args.latency_reps):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        host.append((time.perf_counter() - t0) * 1e3)
    latency = {"cold_l2": _pct(lat_cold), "warm_l2": _pct(lat_warm), "host_call_and_sync": _pct(host),
               "what": "one step (assembly with boundary facets, one launch) on the resident mesh; cold = 512 MiB "
                       "L2 flush before each"}
    got = {"K": K.cpu().numpy(), "M": M.cpu().numpy(), "vol": vol.cpu().numpy(), "normals": nrm.cpu().numpy(),
           "areas": ar.cpu().numpy()}

    # end to end through the public API with pinned host buffers
    hc = torch.from_numpy(m.coords).pin_memory()
    he = torch.from_numpy(m.elems).pin_memory()
    hf = torch.from_numpy(m.faces).pin_memory()
    out_host = {
        "K": torch.empty(gm.nnz, dtype=torch.float64).pin_memory(),
        "M": torch.empty(gm.nnz, dtype=torch.float64).pin_memory(),
        "vol": torch.empty(gm.ne, dtype=torch.float64).pin_memory(),
        "nrm": torch.empty((gm.nfb, 3), dtype=torch.float64).pin_memory(),
        "ar": torch.empty(gm.nfb, dtype=torch.float64).pin_memory(),
        "rp": torch.empty(gm.nn + 1, dtype=torch.int32).pin_memory(),
        "ci": torch.empty(gm.nnz, dtype=torch.int32).pin_memory(),
    }
    h2d = hc.numel() * 8 + he.numel() * 4 + hf.numel() * 4
    rp_b, ci_b = gm.block()
    d2h = rp_b.numel() * 4 + ci_b.numel() * (4 + 8 + 8) + gm.ne * 8 + gm.nfb * (3 * 8 + 8)   # what one rank copies

    split = []
    copy_stream = torch.cuda.Stream()
    ready = torch.cuda.Event()

    def e2e_step():
        # CUDA events between the phases and the host clock around each, to itemise the step
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        th = [time.perf_counter()]
        ev[0].record(stream)
        dc = hc.to(dev, non_blocking=True)
        de = he.to(dev, non_blocking=True)
        df = hf.to(dev, non_blocking=True)
        ev[1].record(stream)
        th.append(time.perf_counter())
        g2 = vla.Mesh(dc, de, df, rows=None if ws == 1 else blk)   # the build synchronises the stream
        ev[2].record(stream)
        th.append(time.perf_counter())
        # the CSR pattern is final once the mesh is built: its copy to the host
        # runs on a second stream while the assembly runs
        rp, ci = g2.block()
        ready.record(stream)
        o = g2.assemble(1.0, 1.0, precision=prec, boundary=True)
        n2, a2 = o["normals"], o["areas"]
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            out_host["rp"][: rp.numel()].copy_(rp, non_blocking=True)
            out_host["ci"][: ci.numel()].copy_(ci, non_blocking=True)
        ev[3].record(stream)
        _, _, kb, mb = g2.block((o["K"], o["M"]))
        ev[4].record(stream)
        th.append(time.perf_counter())
        out_host["K"][: kb.numel()].copy_(kb, non_blocking=True)
        out_host["M"][: mb.numel()].copy_(mb, non_blocking=True)
        out_host["vol"][: g2.ne].copy_(o["vol"], non_blocking=True)
        out_host["nrm"][: g2.nfb].copy_(n2, non_blocking=True)
        out_host["ar"][: g2.nfb].copy_(a2, non_blocking=True)
        stream.wait_stream(copy_stream)
        ev[5].record(stream)
        torch.cuda.synchronize()
        th.append(time.perf_counter())
        g2.close()
        names = ("h2d", "mesh_build", "assemble_with_boundary", "csr_views", "d2h")
        split.append({"device_ms": {n: ev[i].elapsed_time(ev[i + 1]) for i, n in enumerate(names)},
                      "host_ms": {"h2d_enqueue": (th[1] - th[0]) * 1e3, "mesh_build_call": (th[2] - th[1]) * 1e3,
                                  "assemble_boundary_csr_enqueue": (th[3] - th[2]) * 1e3,
                                  "d2h_and_sync": (th[4] - th[3]) * 1e3}})

    e2e_step()
    _barrier(dist)
    torch.cuda.synchronize()
    split.clear()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(dist, (time.perf_counter() - t0) / args.e2e_steps)
    e2e_split = {kind: {n: float(np.median([d[kind][n] for d in split])) for n in split[0][kind]}
                 for kind in ("device_ms", "host_ms")}
    e2e = {"value": m.ne / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
           "includes": "H2D of coords/elems/faces, mesh build (CSR pattern, tiles), assembly, boundary, "
                       "D2H of row_ptr/col_idx/K/M/vol/normals/areas (row_ptr/col_idx on a second stream, "
                       "during the assembly)", "split": e2e_split}

    peaks, src = _peaks()
    bpe = _alg_bytes_per_el(gm.ne, gm.nn, gm.nnz) + FACET_BYTES * gm.nfb / gm.ne
    achieved = bpe * gm.ne / (asm * 1e-3) / 1e9
    khash = _src_hash()
    roof = {"bound": "hbm", "kernel": "k_assemble<3,1,%s>" % ("mixed" if prec else "fp64"),
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": src,
            "traffic": _traffic_from_profile(khash) if prec == vla.PREC_MIXED else None,
            "alg_bytes_per_element": bpe, "kernel_ms": asm, "kernel_source_hash": khash}
    if prec == vla.PREC_FP64:
        # the plain FP64 form against the FP64 pipe: min(HBM, FP64) and which one binds
        fp64 = _fp64_peak(dev)
        # tetrahedral meshes of >= 20,000 elements take the library's two-pass FP64
        # form (every element's record once, then the tiles); otherwise each tile
        # evaluates every element it touches
        recompute = 1.0 if (gm.dim == 3 and gm.ne >= 20000) else gm.tile_elems / gm.ne
        fl = FP64_FLOPS_PER_TET * gm.ne / (asm * 1e-3) / 1e9
        fl_exec = (FP64_FLOPS_PER_TET_EVAL * recompute + FP64_FLOPS_PER_TET - FP64_FLOPS_PER_TET_EVAL) * gm.ne \
            / (asm * 1e-3) / 1e9
        hbm_roof = dict(roof)
        roof = {"bound": "fp64", "kernel": roof["kernel"], "achieved": fl, "peak": fp64, "unit": "GFLOP/s",
                "frac": fl / fp64, "peak_source": "measured in this run: cuBLAS DGEMM 4096^3 (torch.matmul, "
                                                   "best of 5)",
                "flops_per_element": FP64_FLOPS_PER_TET,
                "executed_gflops": fl_exec, "executed_frac": fl_exec / fp64, "element_recompute": recompute,
                "traffic": None, "kernel_ms": asm, "kernel_source_hash": khash, "hbm": hbm_roof}
        if hbm_roof["frac"] > roof["executed_frac"]:
            roof["bound"] = "hbm"

    line = {"metric": "elements/sec for P1 tet K+M to CSR", "value": value, "unit": "elements/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if prec == vla.PREC_MIXED else "f64", "data": "synthetic",
            "config": dict(_config(m, MIXED_LABEL if prec else "fp64"),
                           parallelism=f"rows split in {ws} contiguous blocks, one per rank (halo elements "
                                       f"duplicated, complete rows per rank, no collective on the data path)"
                           if ws > 1 else "one GPU, every row"),
            "e2e": e2e, "roofline": roof, "gpu_launches": args.steps, "clocks": clocks,
            "p50_ms": latency["cold_l2"]["p50_ms"], "p99_ms": latency["cold_l2"]["p99_ms"], "latency": latency,
            "timed_steps_ms": {"min": min(step_ms), "median": float(np.median(step_ms)), "max": max(step_ms),
                               "all": [round(x, 5) for x in step_ms]}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base, ref = cpu_baseline(m, args.cpu_seconds)
        line["cpu_baseline"] = base
        line["errors"] = dict(_errors(ref, got), against="the FP64 oracle on the same mesh and coefficient")
    if rank == 0:
        print(json.dumps(line), flush=True)
    gm.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
