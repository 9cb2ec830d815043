#!/usr/bin/env python3
"""Benchmark of the collision-operator hot path on GB300.

One step = one pass of the hot path over one batch: the fused collision kernel
Q^R(f,f) on 4096 cells (N = 32, hard spheres, M = 48 directions, Mr = 16, FP64)
followed by the moments / realizability / mask kernel on the same cells.
Prints ONE JSON line (rank 0).  Default: 1 GPU, --steps 5 --warmup 3.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas: each rank
evaluates its own 4096-cell batch (weak scaling, no data-path collective); the
reported time is the max over ranks.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(N=32, L=(3.0 + math.sqrt(2.0)) * 3.0, lam=1.0, M=48, Mtheta=4, Mr=16, cells=4096,
                eta0=1e-3, delta0=1e-4)
METRIC = "Q(f,f) cell-evals/s at N=32^3 (mixed vs FP64, L2 err); %HBM/tensor peak; p50/p99 ms"


def algorithmic_flops_per_cell(N: int, n_terms_gain: int) -> float:
    """Transforms T = 2 * (gain terms) + 3 real 3D transforms of N^3 points, each
    2.5 N^3 log2(N^3) flops, plus 4 flops per gain term per point and 3 per
    point for the loss (the per-cell count of the method)."""
    T = 2 * n_terms_gain + 3
    n3 = N ** 3
    return T * 2.5 * n3 * math.log2(n3) + 4 * n_terms_gain * n3 + 3 * n3


def fp64_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """FP64 pipe peak: 2 DFMA per clock per SM (4 flop), the unit count behind
    GB300's nominal 1.25 TFLOP/s at 2.07 GHz."""
    return sms * 4 * sm_mhz * 1e6 / 1e12


KERNEL_SOURCES = {
    "collision_f64_n32": ["collision_impl.cuh", "collision_layout.cuh", "fft.cuh", "twiddles.h", "coll_inst_d32.cu"],
    "moments_f64": ["moments.cu"],
    "conservation_f64": ["moments.cu"],
    "mixed_f16_n32": ["mixed.cu", "tcgen05.cuh"],
    "mixed_sliced_n32": ["sliced.cu", "tcgen05.cuh", "dfloat.cuh"],
    "m2d_f64_n32": ["m2d_impl.cuh", "m2d_d.cu", "fft.cuh", "twiddles.h"],
}


def mixed_mma_flops_per_cell(N: int, n_terms: int) -> float:
    """Executed tensor-core flops of the f16 hi+lo DFT-GEMM path per cell: 128-row
    tiles; per tile (4N/16) K steps against the hi matrix and (2N/16) against
    the lo matrix, each 2 * 128 * n_out * 16 flops (n_out = 2N, N for the real
    first forward pass)."""
    steps = 4 * N // 16 + 2 * N // 16
    per = lambda nout: steps * 2.0 * 128 * nout * 16
    tiles_f2 = N * N // 128
    tiles_full = 2 * (N // 2) * N // 128 + 3 * n_terms * N * N // 128
    return tiles_f2 * per(N) + tiles_full * per(2 * N)


def sliced_mma_flops_per_cell(N: int, n_terms: int) -> float:
    """Executed tensor-core flops of the fixed-point-slice path per cell: 128-row
    tiles; per tile ten slice products of (2N/16) K steps, each 2 * 128 * n_out
    * 16 flops (n_out = 2N, N for the real first forward pass)."""
    steps = 10 * (2 * N // 16)
    per = lambda nout: steps * 2.0 * 128 * nout * 16
    tiles_f2 = N * N // 128
    tiles_full = 2 * (N // 2) * N // 128 + 3 * n_terms * N * N // 128
    return tiles_f2 * per(N) + tiles_full * per(2 * N)


# the Gaussian's exponent (quadratic form, shared along a row), its exponential and the
# step's combination, per value of f
ESBGK_FP64_OPS_PER_VALUE = 11
REGIME_FP64_OPS_PER_CELL = 126     # add/sub/mul/div/sqrt of the indicator sequence (4 div, 3 sqrt)
REGIME_BYTES_PER_CELL = 4 * 8 + 8 + 1 + 1 + 4 * 8   # fields, l1, r in/out, indicators


def time_regime(torch, coll, synth, dev, ny, nx, reps):
    """Regime update (indicators + Algorithm 1) on an nx x ny grid: ms per launch (CUDA events)."""
    dx = 1.0 / 256
    F, r, l1 = synth.regime_fields(ny, nx, dx, synth.BASE_SEED + 6)
    Fd, ld, rd = (torch.from_numpy(a).to(dev) for a in (F, l1, r))
    out = torch.empty_like(rd)
    ind = torch.empty((4, ny, nx), dtype=torch.float64, device=dev)
    p = coll.coll_regime_params(1e-4, 1.0, 1.0, dx, dx, 1e-3, 2.8e-5, 1e-4)
    st = torch.cuda.Stream(device=dev)
    for _ in range(3):
        coll.regime_update(Fd, ld, rd, nx, ny, p, out, ind, stream=st)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        coll.regime_update(Fd, ld, rd, nx, ny, p, out, ind, stream=st)
    b.record(st)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps


M2D_WORKLOAD = dict(N=32, L=8.0, A=32, cells=32768)


def m2d_flops_per_cell(N: int, A: int) -> float:
    """2D operator, counted like the 3D one: 2 A + 3 real 2D transforms of N^2
    points, each 2.5 N^2 log2(N^2) flops, plus 4 flops per gain term per point
    and 3 per point for the loss."""
    n2 = N * N
    return (2 * A + 3) * 2.5 * n2 * math.log2(n2) + 4 * A * n2 + 3 * n2


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """FP32 pipe peak: 128 FFMA per clock per SM (256 flop)."""
    return sms * 256 * sm_mhz * 1e6 / 1e12


def time_m2d(torch, coll, synth, dev, reps=5):
    """2D Maxwell molecules (coll_m2d_eval_batch): FP64, float pairs and FP32 on
    32768 cells N = 32^2 (f and Q 268 MB each in FP64, larger than L2)."""
    w = M2D_WORKLOAD
    N, A, n = w["N"], w["A"], w["cells"]
    f64 = torch.from_numpy(synth.bimodal_batch_2d(n, N, w["L"])).to(dev)
    st = torch.cuda.Stream(device=dev)
    out, ref = {}, None
    for prec in ("f64", "f32x2", "f32"):
        plan = coll.Plan2D(N, w["L"], A=A, prec=prec, device=dev)
        fd = f64.to(plan.torch_dtype)
        Q = torch.empty_like(fd)
        for _ in range(3):
            plan.eval(fd, Q, stream=st)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            plan.eval(fd, Q, stream=st)
        b.record(st)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / reps
        if prec == "f64":
            ref = Q
            err = 0.0
        else:
            err = float(torch.linalg.vector_norm(Q.double() - ref) / torch.linalg.vector_norm(ref))
        out[prec] = (ms, err, plan.status())
        plan.close()
    del f64
    return out


def time_cufft_same_algorithm(torch, coll, plan_desc, f, Q_ref, chunk=512):
    """Timed comparison only: the same fast-spectral algorithm with cuFFT (torch.fft)
    in place of the hand-written transforms, FP64, unfused (per term two C2R 3D
    transforms of the half spectrum times A_t and B_t, then G += a * b).  Uses the
    plan's host-built tables; returns (ms for the whole batch, relative L2 vs Q_ref)."""
    import numpy as np
    N = plan_desc.N
    H = N // 2
    tab = coll.coll_plan_tables_host(plan_desc)                     # [T, N, N, N/2, 2]
    T = tab.shape[0]
    full = np.zeros((T, N, N, H + 1, 2))
    full[:, :, :, :H] = tab
    At = torch.from_numpy(full[..., 0]).to(f.device)
    Bt = torch.from_numpy(full[..., 1]).to(f.device)
    n = f.shape[0]
    Q = torch.empty_like(f)

    def run():
        for s0 in range(0, n, chunk):
            fc = f[s0:s0 + chunk]
            Fh = torch.fft.rfftn(fc, dim=(1, 2, 3))
            Fh[:, H] = 0
            Fh[:, :, H] = 0
            Fh[:, :, :, H] = 0
            G = torch.zeros_like(fc)
            for t in range(T):
                a = torch.fft.irfftn(Fh * At[t], s=(N, N, N), dim=(1, 2, 3), norm="forward")
                b = torch.fft.irfftn(Fh * Bt[t], s=(N, N, N), dim=(1, 2, 3), norm="forward")
                G.addcmul_(a, b)
            Q[s0:s0 + chunk] = G

    run()
    torch.cuda.synchronize(f.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run()
    e1.record()
    torch.cuda.synchronize(f.device)
    err = float(torch.linalg.vector_norm(Q - Q_ref) / torch.linalg.vector_norm(Q_ref))
    return e0.elapsed_time(e1), err


def time_ragged(torch, coll, synth, dev, w, reps=5):
    """The uneven batch of the 256 x 256 regime mask (about 10 K cells, N in {16, 24,
    32, 48}, FP32 anisotropic cells, hard spheres, M = 48, Mr = 16): one ragged
    persistent launch, captured in a CUDA graph and replayed."""
    rb = synth.ragged_batch(L=w["L"])
    plans, groups, cells, flops = [], [], [], 0.0
    for N in synth.RAGGED_N:
        g = rb.groups[N]
        if g.shape[0] == 0:
            continue
        p = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="f32", max_cells=1,
                      device=dev)
        f = torch.from_numpy(g).to(dev)
        plans.append(p)
        groups.append((p.handle, f, torch.empty_like(f)))
        cells.append(g.shape[0])
        flops += algorithmic_flops_per_cell(N, p.n_terms - 1) * g.shape[0]
    del rb
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, cells), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(st):
        coll.coll_eval_ragged(groups, cells, ws, stream=st)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(graph, stream=st):
            coll.coll_eval_ragged(groups, cells, ws, stream=st)
        for _ in range(2):
            graph.replay()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record(st)
        for _ in range(reps):
            graph.replay()
        b.record(st)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / reps
    status = max(p.status() for p in plans)
    for p in plans:
        p.close()
    return {"cells": int(sum(cells)), "cells_per_N": {str(p.N): c for p, c in zip(plans, cells)}, "ms": ms,
            "flops": flops, "status": status}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's value (the job's time); a no-op on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every replica processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


def src_hash(kernel_key: str) -> str:
    """Hash of the sources a kernel is compiled from (a stale ncu traffic figure reads as null)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel_key]:
        h.update(open(os.path.join(ROOT, "paper_2505_03360_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _smi_id(torch, dev, local_rank):
    """nvidia-smi -i selector of the device torch uses (UUID when available)."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local_rank].strip()
    return str(local_rank)


def load_traffic(kernel_key: str):
    """Per-launch DRAM bytes from the committed ncu summary, if taken on the current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel_key)
        if e and e.get("src_hash") == src_hash(kernel_key):
            return e.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


def _oracle_setup(n_cells: int, seed_offset: int = 0):
    """Plan (multipliers) and inputs of an oracle sample: not timed."""
    from oracle.kernel import Params, multipliers
    from paper_2505_03360_gb300 import synth
    w = WORKLOAD
    p = Params(N=w["N"], L=w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"])
    f = synth.bimodal_batch(n_cells, w["N"], w["L"], seed=synth.BASE_SEED + 2 + seed_offset)
    return p, multipliers(p), f


def _oracle_run(p, m, f) -> float:
    """Q and the moments record of every cell of f with the CPU oracle; seconds."""
    from oracle import moments as om
    from oracle.collision import q_fast
    w = WORKLOAD
    t0 = time.perf_counter()
    for c in range(f.shape[0]):
        q_fast(f[c], p, m)
        om.cell_moments(f[c], w["L"], w["eta0"], w["delta0"])
    return time.perf_counter() - t0


def oracle_sample(n_cells: int, seed_offset: int = 0):
    """Time the CPU oracle (as it stands) on n_cells cells of the workload, one core."""
    return _oracle_run(*_oracle_setup(n_cells, seed_offset))


def _oracle_proc(n_cells, seed_offset, barrier, out):
    """One spawned worker of oracle_sample_parallel: plan setup and inputs, then
    a barrier, then the timed oracle work; reports its wall-clock interval."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    p, m, f = _oracle_setup(n_cells, seed_offset)
    _oracle_run(p, m, f[:1])                            # imports and first-call costs
    barrier.wait()
    t0 = time.time()
    dt = _oracle_run(p, m, f)
    out.put((t0, time.time(), dt))


def oracle_sample_parallel(n_per_worker: int, workers: int = 0, seed_offset: int = 0):
    """The CPU oracle (as it stands) on all host cores: one spawned process per core,
    each on its own n_per_worker cells of the workload, started together after their
    setup.  Returns (cells, wall seconds from the first start to the last finish, workers)."""
    import multiprocessing as mp
    workers = workers or (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_proc, args=(n_per_worker, seed_offset + 1000 * i, barrier, out))
             for i in range(workers)]
    for pr in procs:
        pr.start()
    spans = [out.get(timeout=600) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    return n_per_worker * workers, max(b for _, b, _ in spans) - min(a for a, _, _ in spans), workers


def run_reference(args, rank):
    if rank != 0:
        return
    w = WORKLOAD
    per_worker = 4
    for _ in range(args.warmup):
        oracle_sample(1)
    tt, cells, workers = 0.0, 0, 1
    for s in range(args.steps):
        c, wall, workers = oracle_sample_parallel(per_worker, seed_offset=100000 * s)
        tt += wall
        cells += c
    per_step = cells // max(1, args.steps)
    value = cells / tt
    line = {"metric": METRIC, "value": value, "unit": "cell-evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "4096-cell batch, N=32^3, hard spheres (lambda=1), M=48, Mr=16, FP64 + moments/mask; "
                                   "each step a %d-cell sample on the host cores" % per_step,
                       "global_batch": w["cells"], "seq_len": w["N"] ** 3, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "cell-evals/s", "cores": workers, "kind": "oracle",
                             "sample": "%d cells per step (%d per core, one spawned process per core) x %d steps of "
                                       "the 4096-cell workload" % (per_step, per_worker, args.steps)},
            "e2e": {"value": value, "unit": "cell-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_lowrank(torch, coll, synth, dev, w, n=1024):
    """Maxwell molecules (lambda = 0, Mr = 8) on n FP32 N = 32 bimodal cells: the
    full radial sum against the low-rank separable kernel at ranks 6, 5, 4
    (ms per launch; relative L2 of the batch against the full operator)."""
    N = w["N"]
    f = synth.bimodal_batch_device(n, N, w["L"], 21, dtype=torch.float32, device=dev)
    out, ref = {}, None
    for rank in (0, 6, 5, 4):
        plan = coll.Plan(N, w["L"], lam=0.0, M=w["M"], Mtheta=w["Mtheta"], Mr=8, prec="f32", max_cells=n,
                         device=dev, rank=rank)
        Q = torch.empty_like(f)
        plan.eval(f, Q)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            plan.eval(f, Q)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 3
        if ref is None:
            ref = Q.double()
        out["rank%d" % rank if rank else "full"] = {
            "terms": plan.n_terms, "ms_per_launch": ms, "cell_evals_per_s": n / (ms / 1e3),
            "rel_l2_vs_full": float(torch.linalg.vector_norm(Q.double() - ref) / torch.linalg.vector_norm(ref))}
        plan.close()
    return {"workload": "%d FP32 cells, N = 32, lambda = 0, M = 48, Mr = 8 (24 directions x 8 radial nodes), "
                        "bimodal Maxwellians" % n, **out}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2505_03360_gb300 import coll, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.profile_m2d:
        # short capture target: the 2D operator alone on --m2d-cells cells, two launches
        mw = M2D_WORKLOAD
        plan2 = coll.Plan2D(mw["N"], mw["L"], A=mw["A"], prec=args.profile_m2d, device=dev)
        f2 = torch.from_numpy(synth.bimodal_batch_2d(args.m2d_cells, mw["N"], mw["L"])).to(dev).to(plan2.torch_dtype)
        Q2 = torch.empty_like(f2)
        for _ in range(2):
            plan2.eval(f2, Q2)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_m2d": args.profile_m2d, "cells": args.m2d_cells, "status": plan2.status()}))
        plan2.close()
        return
    w = WORKLOAD
    N, n = (args.N if args.profile_only else w["N"]), args.cells
    f_host = synth.bimodal_batch(n, N, w["L"], seed=synth.BASE_SEED + 2 + 1000 * rank)
    f_pin = torch.from_numpy(f_host).pin_memory()
    f = f_pin.to(dev)
    del f_host
    Q = torch.empty_like(f)
    prec_main = args.prec if args.profile_only else "f64"
    if prec_main == "f32":
        f = f.float()
    Q = torch.empty_like(f)
    plan = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec=prec_main,
                     max_cells=n, device=dev)
    if args.profile_only and args.variant is not None:
        coll.coll_plan_set_variant(plan.handle, args.variant)
    ws = plan.reserve(n)
    mom = torch.empty((n, coll.MOMENT_DOUBLES), dtype=torch.float64, device=dev)
    mask = torch.empty((n,), dtype=torch.uint8, device=dev)
    cons = torch.empty((n, 8), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        coll.coll_eval_batch(plan.handle, f, Q, n, ws, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        coll.moments_realizability(f, 0 if f.dtype == torch.float64 else 1, N, w["L"], n, w["eta0"], w["delta0"],
                                   mom, mask, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        # FP64 conservation check of Q (mass, momentum, energy per cell)
        coll.coll_conservation(Q, 0 if Q.dtype == torch.float64 else 1, N, w["L"], n, cons, stream=stream)
        if ev is not None:
            ev[3].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = coll.coll_launch_count()
    with ClockSampler(_smi_id(torch, dev, local_rank)) as clk:
        torch.cuda.synchronize(dev)
        t_start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    launches = coll.coll_launch_count() - launches0
    elapsed = t_start.elapsed_time(t_end) / 1e3
    coll_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    mom_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    cons_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    assert plan.status() == coll.COLL_OK
    if world > 1:
        elapsed = max_over_ranks(elapsed, world, device=dev)
        dist.barrier()

    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "N": N, "prec": prec_main, "cells": n,
                              "ms_per_step": 1e3 * elapsed / args.steps, "collision_ms": coll_ms}), flush=True)
        plan.close()
        return
    # end to end through the C ABI from pinned host buffers: every step uploads its f, evaluates
    # Q and the moments/mask, and downloads Q, the records and the mask.  Two buffer sets and
    # three streams (upload, compute, download) overlap step k+1's upload and step k-1's
    # download with step k's compute.
    # eight steps (fewer if --steps is smaller, at least three): the first upload and the
    # last download are not overlapped, and the host copy bandwidth differs from box to box
    e2e_steps = max(3, min(args.steps, 8))
    fb, Qb = [f, torch.empty_like(f)], [Q, torch.empty_like(Q)]
    momb, maskb = [mom, torch.empty_like(mom)], [mask, torch.empty_like(mask)]
    consb = [cons, torch.empty_like(cons)]
    cons_pin = [torch.empty(cons.shape, dtype=cons.dtype).pin_memory() for _ in range(2)]
    Q_pin = [torch.empty(Q.shape, dtype=Q.dtype).pin_memory() for _ in range(2)]
    mom_pin = [torch.empty(mom.shape, dtype=mom.dtype).pin_memory() for _ in range(2)]
    mask_pin = [torch.empty(mask.shape, dtype=mask.dtype).pin_memory() for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    io = 0 if f.dtype == torch.float64 else 1

    def e2e_run(k_steps):
        ev_comp, ev_out = [None, None], [None, None]
        for k in range(k_steps):
            b = k % 2
            if ev_comp[b] is not None:
                s_in.wait_event(ev_comp[b])            # the previous compute on buffer b has read its f
            with torch.cuda.stream(s_in):
                fb[b].copy_(f_pin, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            stream.wait_event(ev_in)
            if ev_out[b] is not None:
                stream.wait_event(ev_out[b])           # buffer b's previous results are downloaded
            coll.coll_eval_batch(plan.handle, fb[b], Qb[b], n, ws, stream=stream)
            coll.moments_realizability(fb[b], io, N, w["L"], n, w["eta0"], w["delta0"], momb[b], maskb[b],
                                       stream=stream)
            coll.coll_conservation(Qb[b], io, N, w["L"], n, consb[b], stream=stream)
            ev_comp[b] = torch.cuda.Event()
            ev_comp[b].record(stream)
            s_out.wait_event(ev_comp[b])
            with torch.cuda.stream(s_out):
                Q_pin[b].copy_(Qb[b], non_blocking=True)
                mom_pin[b].copy_(momb[b], non_blocking=True)
                mask_pin[b].copy_(maskb[b], non_blocking=True)
                cons_pin[b].copy_(consb[b], non_blocking=True)
            ev_out[b] = torch.cuda.Event()
            ev_out[b].record(s_out)

    e2e_run(2)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    stream.wait_event(e0)
    s_out.wait_event(e0)
    e2e_run(e2e_steps)
    e1.record(s_out)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_s = max_over_ranks(e2e_s, world, device=dev)
    assert bool(torch.equal(Q_pin[(e2e_steps - 1) % 2], Qb[(e2e_steps - 1) % 2].cpu()))
    del fb[1], Qb[1], momb[1], maskb[1], consb[1], Q_pin, mom_pin, mask_pin, cons_pin

    def cons_errors(Qv):
        """Largest relative mass, momentum and energy errors over the batch (coll_conservation)."""
        inv = coll.conservation(Qv, w["L"], stream=stream)
        torch.cuda.synchronize(dev)
        e = coll.conservation_errors(inv)
        return {"mass": float(e[:, 0].max()), "momentum": float(e[:, 1].max()), "energy": float(e[:, 2].max())}

    cons64 = cons_errors(Q)

    # float-pair variant (FP64-class accuracy on the FP32 pipe) on the same cells
    Qx = torch.empty_like(f)
    planx = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="f32x2",
                      max_cells=n, device=dev)
    wsx = planx.reserve(n)
    with torch.cuda.stream(stream):
        for _ in range(2):
            coll.coll_eval_batch(planx.handle, f, Qx, n, wsx, stream=stream)
    torch.cuda.synchronize(dev)
    ax, bx = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ax.record(stream)
    for _ in range(args.steps):
        coll.coll_eval_batch(planx.handle, f, Qx, n, wsx, stream=stream)
    bx.record(stream)
    torch.cuda.synchronize(dev)
    tx = ax.elapsed_time(bx) / 1e3 / args.steps
    errx = float(torch.linalg.vector_norm(Qx - Q) / torch.linalg.vector_norm(Q))
    consx = cons_errors(Qx)
    del Qx

    # FP32 variant on the same cells (reported beside the FP64 line)
    f32 = f.float()
    Q32 = torch.empty_like(f32)
    plan32 = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="f32",
                       max_cells=n, device=dev)
    ws32 = plan32.reserve(n)
    with torch.cuda.stream(stream):
        for _ in range(2):
            coll.coll_eval_batch(plan32.handle, f32, Q32, n, ws32, stream=stream)
    torch.cuda.synchronize(dev)
    a32, b32 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a32.record(stream)
    for _ in range(args.steps):
        coll.coll_eval_batch(plan32.handle, f32, Q32, n, ws32, stream=stream)
    b32.record(stream)
    torch.cuda.synchronize(dev)
    t32 = a32.elapsed_time(b32) / 1e3 / args.steps
    err32 = float(torch.linalg.vector_norm(Q32.double() - Q) / torch.linalg.vector_norm(Q))
    cons32 = cons_errors(Q32)
    del Q32, f32

    # tensor-core DFT-GEMM variant (f16 hi+lo split, FP32 accumulate) on the same FP64 cells
    Qm = torch.empty_like(f)
    planm = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="mixed_f16x2",
                      io_dtype=0, max_cells=n, device=dev)
    wsm = planm.reserve(n)
    with torch.cuda.stream(stream):
        for _ in range(2):
            coll.coll_eval_batch(planm.handle, f, Qm, n, wsm, stream=stream)
    torch.cuda.synchronize(dev)
    am, bm = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    am.record(stream)
    for _ in range(args.steps):
        coll.coll_eval_batch(planm.handle, f, Qm, n, wsm, stream=stream)
    bm.record(stream)
    torch.cuda.synchronize(dev)
    tm = am.elapsed_time(bm) / 1e3 / args.steps
    assert planm.status() == coll.COLL_OK
    cell_err = torch.linalg.vector_norm((Qm - Q).reshape(n, -1), dim=1) / torch.linalg.vector_norm(Q.reshape(n, -1), dim=1)
    errm = float(torch.linalg.vector_norm(Qm - Q) / torch.linalg.vector_norm(Q))
    consm = cons_errors(Qm)
    # bf16 three-part variant on the same cells
    planb = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="mixed_bf16x3",
                      io_dtype=0, max_cells=n, device=dev)
    wsb = planb.reserve(n)
    with torch.cuda.stream(stream):
        coll.coll_eval_batch(planb.handle, f, Qm, n, wsb, stream=stream)
    torch.cuda.synchronize(dev)
    ab, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ab.record(stream)
    for _ in range(args.steps):
        coll.coll_eval_batch(planb.handle, f, Qm, n, wsb, stream=stream)
    bb.record(stream)
    torch.cuda.synchronize(dev)
    tb = ab.elapsed_time(bb) / 1e3 / args.steps
    assert planb.status() == coll.COLL_OK
    cell_errb = torch.linalg.vector_norm((Qm - Q).reshape(n, -1), dim=1) / torch.linalg.vector_norm(Q.reshape(n, -1), dim=1)
    errb = float(torch.linalg.vector_norm(Qm - Q) / torch.linalg.vector_norm(Q))
    consb_ = cons_errors(Qm)
    planb.close()
    # fixed-point-slice tensor-core variant (exact leading products, float-pair intermediates)
    plans = coll.Plan(N, w["L"], lam=w["lam"], M=w["M"], Mtheta=w["Mtheta"], Mr=w["Mr"], prec="mixed_sliced",
                      io_dtype=0, max_cells=n, device=dev)
    wss = plans.reserve(n)
    with torch.cuda.stream(stream):
        coll.coll_eval_batch(plans.handle, f, Qm, n, wss, stream=stream)
    torch.cuda.synchronize(dev)
    as_, bs_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    as_.record(stream)
    for _ in range(args.steps):
        coll.coll_eval_batch(plans.handle, f, Qm, n, wss, stream=stream)
    bs_.record(stream)
    torch.cuda.synchronize(dev)
    ts = as_.elapsed_time(bs_) / 1e3 / args.steps
    assert plans.status() == coll.COLL_OK
    cell_errs = torch.linalg.vector_norm((Qm - Q).reshape(n, -1), dim=1) / torch.linalg.vector_norm(Q.reshape(n, -1), dim=1)
    errs = float(torch.linalg.vector_norm(Qm - Q) / torch.linalg.vector_norm(Q))
    conss = cons_errors(Qm)
    n_terms_s = plans.n_terms
    plans.close()
    del Qm

    if rank != 0:
        return
    value = whole_job_rate(n * args.steps, world, elapsed)
    clocks = clk.summary()
    n_gain = plan.n_terms - 1
    flops = algorithmic_flops_per_cell(N, n_gain) * n
    achieved = flops / (coll_ms / 1e3) / 1e12
    sm_for_peak = 2070.0
    peak = fp64_peak_tflops(sm_for_peak)
    traffic = load_traffic("collision_f64_n32")
    peaks = measured_peaks()
    tc_peak = peaks.get("bf16_tflops")
    mma_flops = mixed_mma_flops_per_cell(N, planm.n_terms) * n
    mom_bytes = f.numel() * 8 + mom.numel() * 8 + mask.numel()
    cons_bytes = Q.numel() * 8 + cons.numel() * 8
    e2e_bytes_in = f.numel() * 8
    e2e_bytes_out = Q.numel() * 8 + mom.numel() * 8 + mask.numel() + cons.numel() * 8
    line = {
        "metric": METRIC, "value": value, "unit": "cell-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4096-cell batch, N=32^3, hard spheres (lambda=1), M=48 (24 hemisphere directions), "
                               "Mr=16, FP64 collision + FP64 moments/realizability mask (eta0=1e-3, delta0=1e-4) + FP64 conservation check of Q",
                   "global_batch": n * world, "seq_len": N ** 3, "parallelism": "replicas x%d" % world,
                   "l2": "inputs larger than L2 (f and Q are 1.07 GB each)"},
        "e2e": {"value": whole_job_rate(n * e2e_steps, world, e2e_s), "unit": "cell-evals/s",
                "steps": e2e_steps, "pipelining": "upload / compute / download on three streams, two buffer sets",
                "h2d_bytes_per_step": e2e_bytes_in,
                "d2h_bytes_per_step": e2e_bytes_out},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "collision_kernel<32,double,double>",
                     "peak_basis": "FP64 pipe, 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived; nominal 1.25 TF)",
                     "flops_per_launch": flops, "ms_per_launch": coll_ms},
        "clocks": clocks,
        "variants": {"f32x2": {"value": n / tx, "unit": "cell-evals/s", "rel_l2_vs_f64": errx,
                               "ms_per_launch": 1e3 * tx, "arithmetic": "float pairs (~48 bits) on the FP32 pipe",
                               "conservation_rel_max": consx},
                     "f32": {"value": n / t32, "unit": "cell-evals/s", "rel_l2_vs_f64": err32,
                             "ms_per_launch": 1e3 * t32, "conservation_rel_max": cons32},
                     "mixed_f16x2": {
                         "value": n / tm, "unit": "cell-evals/s", "rel_l2_vs_f64": errm,
                         "cell_rel_l2_median": float(cell_err.median()), "cell_rel_l2_max": float(cell_err.max()),
                         "ms_per_launch": 1e3 * tm, "speedup_vs_f64": coll_ms / (1e3 * tm),
                         "conservation_rel_max": consm,
                         "arithmetic": "DFT-GEMMs on tcgen05 tensor cores, f16 hi+lo operands, FP32 accumulate",
                         "roofline": {"bound": "tensor", "achieved": mma_flops / tm / 1e12, "peak": tc_peak,
                                      "unit": "TFLOP/s",
                                      "frac": (mma_flops / tm / 1e12 / tc_peak) if tc_peak else None,
                                      "peak_basis": "measured dense bf16 burst (f16 runs at the same dense rate)",
                                      "executed_mma_flops_per_launch": mma_flops,
                                      "traffic": load_traffic("mixed_f16_n32"),
                                      "algorithmic_tflops": flops / tm / 1e12}},
                     "mixed_bf16x3": {
                         "value": n / tb, "unit": "cell-evals/s", "rel_l2_vs_f64": errb,
                         "cell_rel_l2_median": float(cell_errb.median()), "cell_rel_l2_max": float(cell_errb.max()),
                         "ms_per_launch": 1e3 * tb, "speedup_vs_f64": coll_ms / (1e3 * tb),
                         "conservation_rel_max": consb_,
                         "arithmetic": "DFT-GEMMs on tcgen05 tensor cores, bf16 hi+mid+lo operands, FP32 accumulate"},
                     "mixed_sliced": {
                         "value": n / ts, "unit": "cell-evals/s", "rel_l2_vs_f64": errs,
                         "cell_rel_l2_median": float(cell_errs.median()), "cell_rel_l2_max": float(cell_errs.max()),
                         "ms_per_launch": 1e3 * ts, "speedup_vs_f64": coll_ms / (1e3 * ts),
                         "conservation_rel_max": conss,
                         "arithmetic": "DFT-GEMMs on tcgen05 tensor cores, fixed-point f16 slices (three 9-bit "
                                       "integer parts + f16 tail), two leading product levels summed exactly in "
                                       "FP32 tensor memory, float-pair intermediates",
                         "roofline": {"bound": "tensor", "achieved": sliced_mma_flops_per_cell(N, n_terms_s) * n / ts / 1e12,
                                      "peak": tc_peak, "unit": "TFLOP/s",
                                      "frac": (sliced_mma_flops_per_cell(N, n_terms_s) * n / ts / 1e12 / tc_peak)
                                      if tc_peak else None,
                                      "peak_basis": "measured dense bf16 burst (f16 runs at the same dense rate)",
                                      "executed_mma_flops_per_launch": sliced_mma_flops_per_cell(N, n_terms_s) * n,
                                      "traffic": load_traffic("mixed_sliced_n32"),
                                      "algorithmic_tflops": flops / ts / 1e12}}},
        "moments": {"kernel": "moments sums + scalar finish (2 launches)", "ms_per_launch": mom_ms,
                    "achieved_gbs": mom_bytes / (mom_ms / 1e3) / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": (mom_bytes / (mom_ms / 1e3) / 1e9 / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                    "bytes_per_launch": mom_bytes, "bound": "hbm", "traffic": load_traffic("moments_f64")},
        "conservation": {"kernel": "cons_kernel<32, double> (exact fixed-point sums of Q (1, v, |v|^2) per cell)",
                         "ms_per_launch": cons_ms, "achieved_gbs": cons_bytes / (cons_ms / 1e3) / 1e9,
                         "peak_gbs": peaks.get("hbm_gbs"),
                         "frac": (cons_bytes / (cons_ms / 1e3) / 1e9 / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                         "bytes_per_launch": cons_bytes, "bound": "hbm", "traffic": load_traffic("conservation_f64"),
                         "rel_max_fp64": cons64},
    }
    if world > 1:
        # replicas: the single-GPU sub-measurements below (next rows, comparisons, serving,
        # CPU baseline) belong to the 1-GPU run; the other GPUs are not held for them
        print(json.dumps(line), flush=True)
        plan.close()
        plan32.close()
        planx.close()
        planm.close()
        return
    # regime update on the 2D grid (indicators + Algorithm 1): the 256 x 256 spatial grid of
    # the ragged workload, and a 4096 x 4096 grid (inputs > L2) for the throughput and roofline
    t256 = time_regime(torch, coll, synth, dev, 256, 256, 50)
    t4k = time_regime(torch, coll, synth, dev, 4096, 4096, 5)
    c4k = 4096 * 4096
    fp64_tf = REGIME_FP64_OPS_PER_CELL * c4k / (t4k / 1e3) / 1e12
    line["regime"] = {
        "kernel": "regime_kernel (central differences, V_eps^1 eigenvalues, lambda_B, Algorithm 1; FP64)",
        "grid_256": {"ms_per_launch": t256, "cells_per_s": 65536 / (t256 / 1e3)},
        "grid_4096": {"ms_per_launch": t4k, "cells_per_s": c4k / (t4k / 1e3)},
        "roofline": {"bound": "alu", "achieved": fp64_tf, "peak": peak, "unit": "TFLOP/s", "frac": fp64_tf / peak,
                     "peak_basis": "FP64 pipe (as the main line)",
                     "flops_per_cell": REGIME_FP64_OPS_PER_CELL, "bytes_per_cell": REGIME_BYTES_PER_CELL,
                     "hbm_gbs": REGIME_BYTES_PER_CELL * c4k / (t4k / 1e3) / 1e9}}
    # penalised IMEX update (PR(2,2,2) stages, HBM-bound streams) on the same 4096 FP64 cells:
    # the Y2 stage reads f, Y1 and Q(Y1) and writes Y2 (4 x 1.07 GB); then one whole PR(2,2,2)
    # step (moments, 3 stages, 2 collision evaluations with the FP64 plan)
    Y1 = torch.empty_like(f)
    Y2 = torch.empty_like(f)
    dt_, eps_ = 1e-2, 1.0
    coll.coll_imex_stage(coll.IMEX_PR_Y1, f, None, None, None, None, mom, None, 0, N, w["L"], n, dt_, eps_, Y1,
                         stream=stream)
    for _ in range(3):
        coll.coll_imex_stage(coll.IMEX_PR_Y2, f, Y1, Q, None, None, mom, None, 0, N, w["L"], n, dt_, eps_, Y2,
                             stream=stream)
    torch.cuda.synchronize(dev)
    ia, ib = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ia.record(stream)
    for _ in range(10):
        coll.coll_imex_stage(coll.IMEX_PR_Y2, f, Y1, Q, None, None, mom, None, 0, N, w["L"], n, dt_, eps_, Y2,
                             stream=stream)
    ib.record(stream)
    torch.cuda.synchronize(dev)
    t_stage = ia.elapsed_time(ib) / 10
    stage_bytes = 4 * f.numel() * 8
    with torch.cuda.stream(stream):
        coll.pr222_step(plan, f, w["L"], dt_, eps_, out=Y2, stream=stream)
        torch.cuda.synchronize(dev)
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        coll.pr222_step(plan, f, w["L"], dt_, eps_, out=Y2, stream=stream)
        pb.record(stream)
    torch.cuda.synchronize(dev)
    t_pr = pa.elapsed_time(pb)
    del Y1, Y2
    line["imex"] = {
        "kernel": "imex_kernel (penalised IMEX stages, eq. 1002 / PR(2,2,2); FP64)",
        "stage_y2_ms": t_stage, "stage_y2_bytes": stage_bytes,
        "roofline": {"bound": "hbm", "achieved": stage_bytes / (t_stage / 1e3) / 1e9, "peak": peaks.get("hbm_gbs"),
                     "unit": "GB/s",
                     "frac": (stage_bytes / (t_stage / 1e3) / 1e9 / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None},
        "pr222_step_ms": t_pr,
        "pr222_step": "moments + Y1 + Q(Y1) + Y2 + Q(Y2) + final on 4096 N=32 cells, FP64 collision plan"}
    # ES-BGK relaxation step (layer 1) on the same 4096 FP64 cells: reads f and writes f^{n+1}
    for _ in range(3):
        coll.coll_esbgk_step(f, mom, 0, N, w["L"], n, 1e-2, 1.0, -0.5, 1.0, Q, stream=stream)
    torch.cuda.synchronize(dev)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(10):
        coll.coll_esbgk_step(f, mom, 0, N, w["L"], n, 1e-2, 1.0, -0.5, 1.0, Q, stream=stream)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    t_es = ea.elapsed_time(eb) / 10
    es_bytes = 2 * f.numel() * 8
    es_tf = ESBGK_FP64_OPS_PER_VALUE * f.numel() / (t_es / 1e3) / 1e12
    line["esbgk"] = {
        "kernel": "esbgk_kernel (ES-BGK IMEX relaxation step, eq. 1000; FP64, beta = -1/2)",
        "ms_per_launch": t_es, "cell_steps_per_s": n / (t_es / 1e3),
        "roofline": {"bound": "alu", "achieved": es_tf, "peak": peak, "unit": "TFLOP/s", "frac": es_tf / peak,
                     "peak_basis": "FP64 pipe (as the main line)", "flops_per_value": ESBGK_FP64_OPS_PER_VALUE,
                     "hbm_gbs": es_bytes / (t_es / 1e3) / 1e9, "bytes_per_launch": es_bytes}}
    # timed comparison: the same algorithm with cuFFT transforms (not on the product path)
    coll.coll_eval_batch(plan.handle, f, Q, n, ws, stream=stream)
    with torch.cuda.stream(stream):
        t_cufft, err_cufft = time_cufft_same_algorithm(torch, coll, plan.desc, f, Q)
    line["cufft_comparison"] = {
        "what": "the same fast-spectral algorithm, FP64, with cuFFT (torch.fft rfftn / irfftn) in place of the "
                "hand-written transforms; unfused (two C2R 3D transforms and elementwise passes per term); "
                "timed comparison only",
        "ms_per_batch": t_cufft, "cell_evals_per_s": n / (t_cufft / 1e3), "rel_l2_vs_ours": err_cufft,
        "ours_ms_per_batch": coll_ms, "speedup_of_ours": t_cufft / coll_ms}
    # 2D Maxwell molecules (sec. 4.4.1, "The 2d case"): 32768 cells N = 32^2, A = 32 angles
    mw = M2D_WORKLOAD
    m2 = time_m2d(torch, coll, synth, dev)
    m2_flops = m2d_flops_per_cell(mw["N"], mw["A"]) * mw["cells"]
    t64 = m2["f64"][0]
    t32m = m2["f32"][0]
    p32 = fp32_peak_tflops(sm_for_peak)
    line["maxwell2d"] = {
        "kernel": "m2d_kernel<32, T, Tio> (2D Maxwell molecules, one CTA per cell, 8 terms side by side)",
        "workload": "%d cells, N = %d^2, A = %d angles (%d terms with the loss), L = %g, R = 2S, "
                    "S = 2L/(3 + sqrt 2); bimodal 2D Maxwellians" % (mw["cells"], mw["N"], mw["A"], mw["A"] + 1,
                                                                    mw["L"]),
        "f64": {"ms_per_launch": t64, "cell_evals_per_s": mw["cells"] / (t64 / 1e3), "status": m2["f64"][2],
                "roofline": {"bound": "alu", "achieved": m2_flops / (t64 / 1e3) / 1e12, "peak": peak,
                             "unit": "TFLOP/s", "frac": m2_flops / (t64 / 1e3) / 1e12 / peak,
                             "peak_basis": "FP64 pipe (as the main line)", "flops_per_launch": m2_flops,
                             "traffic": load_traffic("m2d_f64_n32")}},
        "f32x2": {"ms_per_launch": m2["f32x2"][0], "cell_evals_per_s": mw["cells"] / (m2["f32x2"][0] / 1e3),
                  "rel_l2_vs_f64": m2["f32x2"][1], "status": m2["f32x2"][2]},
        "f32": {"ms_per_launch": t32m, "cell_evals_per_s": mw["cells"] / (t32m / 1e3), "rel_l2_vs_f64": m2["f32"][1],
                "status": m2["f32"][2],
                "roofline": {"bound": "alu", "achieved": m2_flops / (t32m / 1e3) / 1e12, "peak": p32,
                             "unit": "TFLOP/s", "frac": m2_flops / (t32m / 1e3) / 1e12 / p32,
                             "peak_basis": "FP32 pipe, 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz (derived)",
                             "hbm_gbs": 2 * mw["cells"] * mw["N"] ** 2 * 4 / (t32m / 1e3) / 1e9}}}
    # the uneven batch of the 256 x 256 regime mask: one ragged launch replayed from a CUDA graph
    rg = time_ragged(torch, coll, synth, dev, w)
    rg_tf = rg["flops"] / (rg["ms"] / 1e3) / 1e12
    line["ragged"] = {
        "kernel": "ragged_kernel<float, float, 16, 24, 32, 48> (persistent, cells taken from a device counter, "
                  "costliest cells first), memset + launch captured in a CUDA graph",
        "workload": "256 x 256 spatial grid, ~15 % Boltzmann mask in curved shock bands, N iid over "
                    "{16, 24, 32, 48}, FP32 anisotropic-temperature cells, hard spheres, M = 48, Mr = 16",
        "cells": rg["cells"], "cells_per_N": rg["cells_per_N"], "ms_per_launch": rg["ms"],
        "cell_evals_per_s": rg["cells"] / (rg["ms"] / 1e3), "status": rg["status"],
        "roofline": {"bound": "alu", "achieved": rg_tf, "peak": p32, "unit": "TFLOP/s", "frac": rg_tf / p32,
                     "peak_basis": "FP32 pipe (as the 2D FP32 line)", "flops_per_launch": rg["flops"]}}
    # low-rank radial kernel for Maxwell molecules (plan rank): FP32, N = 32, M = 48, Mr = 8
    line["lowrank"] = time_lowrank(torch, coll, synth, dev, w)
    if args.serve_requests > 0:
        from paper_2505_03360_gb300.service import Service, stream_jobs
        svc = Service(hbm_budget_bytes=120e9, device=str(dev), max_wall_s=args.serve_max_wall)
        svc.warm_plans()
        jobs = stream_jobs(n_requests=args.serve_requests, rate_per_s=200.0, max_cells=args.serve_max_cells)
        _, st = svc.run(jobs, realtime=True)
        svc.close()
        line["serving"] = {
            "workload": "Poisson 200 req/s, first %d requests of the stream, cells floor(exp(U[0, ln %d])), "
                        "N in {16,32,48,64}, lambda in {0,1}, precision in {f32, mixed}, 10 evaluations each "
                        "(f += 1e-2 Q between), HBM budget 120 GB" % (args.serve_requests, args.serve_max_cells + 1),
            "cell_evals_per_s": st["cell_evals_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "requests": st["requests"], "wall_s": st["wall_s"], "peak_hbm_gb": st["peak_hbm_bytes"] / 1e9,
            "max_queue_depth": st["max_queue_depth"], "ragged_launches": st["ragged_launches"],
            "requests_by_compute_type": st["requests_by_compute_type"],
            "conservation_rel_max": st["conservation_rel_max"],
            "mass_rel_max_by_compute_type": st["mass_rel_max_by_compute_type"],
            "precision_classes": "f32: FP32 kernels; mixed: fixed-point-slice tensor cores (<= 1e-6 vs FP64) at "
                                 "N = 16, 32, FP32 kernels at N = 48, 64"}
    if not args.no_cpu_baseline:
        ncell = 48
        tcpu = oracle_sample(ncell)
        pc, pwall, workers = oracle_sample_parallel(16)
        line["cpu_baseline"] = {"value": pc / pwall, "unit": "cell-evals/s", "cores": workers, "kind": "oracle",
                                "sample": "%d cells of the 4096-cell workload (q_fast + moments, FP64 numpy), 16 per "
                                          "core in one spawned process per host core" % pc,
                                "single_core": {"value": ncell / tcpu, "cores": 1,
                                                "sample": "%d cells on one core" % ncell}}
    print(json.dumps(line), flush=True)
    plan.close()
    plan32.close()
    planx.close()
    planm.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=WORKLOAD["cells"],
                    help="cells per rank (default: the 4096-cell workload; smaller only for profiling)")
    ap.add_argument("--profile-only", action="store_true",
                    help="time the main path only (no e2e, no variants): for short profiler captures")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="requests of the serving stream measured beside the main line (0: skip)")
    ap.add_argument("--serve-max-cells", type=int, default=64,
                    help="largest request (cells); the full serving workload is --serve-requests 2000 "
                         "--serve-max-cells 2048 (several minutes)")
    ap.add_argument("--serve-max-wall", type=float, default=1800.0)
    ap.add_argument("--profile-m2d", default=None, choices=["f64", "f32x2", "f32"],
                    help="run only the 2D Maxwell operator (two launches) for profiler captures")
    ap.add_argument("--m2d-cells", type=int, default=M2D_WORKLOAD["cells"])
    ap.add_argument("--prec", default="f64", choices=["f64", "f32x2", "f32", "mixed_f16x2", "mixed_bf16x3",
                                                      "mixed_sliced"],
                    help="compute precision of the main path in --profile-only runs")
    ap.add_argument("--N", type=int, default=WORKLOAD["N"],
                    help="velocity grid N of the main path in --profile-only runs")
    ap.add_argument("--variant", type=int, default=None, choices=[0, 1],
                    help="slab shape of the main path's plan in --profile-only runs (default: the plan's own)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
