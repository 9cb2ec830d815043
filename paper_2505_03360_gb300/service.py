"""Continuous-batching collision-evaluation service over the C ABI.

Requests (cells x N^3, lambda, precision, a number of repeated evaluations)
arrive over time.  Between GPU iterations the loop admits waiting requests in
arrival order while they fit the HBM budget (f, Q and the workspace of the
request's cells) and keeps every admitted request's f resident on the device.  Each
iteration evaluates the active requests oldest first, up to a cost budget per
iteration (at least one request), so that early requests finish early instead
of every request advancing in lockstep: ONE ragged persistent launch per SIMT
compute type over the cells of the selected requests (coll_eval_ragged), one
ragged launch of the fixed-point-slice tensor-core kernel per N over the
selected mixed-precision requests of that N, then f <- f + dt Q (coll_advance).  A request leaves after its last evaluation; its
memory returns to the budget and the next waiting requests are admitted.
Latency is measured from arrival to the completion of the request's last
evaluation.

Precision classes: "f32" runs the FP32 kernels; "mixed" runs the tensor-core
fixed-point-slice path (COLL_MIXED_SLICED, within 1e-6 of FP64 per cell) where
it supports the grid (N = 16, 32) and the FP32 kernels above (N = 48, 64 have no
tensor-core path); every finished request records the compute type it ran in
and the conservation errors of its last Q (coll_conservation: mass, momentum
and energy relative to the |Q|-weighted integrals), so no result leaves without
a stated accuracy.  Each cell's arithmetic does not depend on what else is in
the batch, so a request's result is the same alone and in the mix.
"""
from __future__ import annotations

import collections
import dataclasses
import json
import math
import time

import numpy as np

from . import coll, synth


def torch_event(stream):
    import torch
    e = torch.cuda.Event()
    e.record(stream)
    return e

TENSOR = ("mixed_sliced", "mixed_f16x2", "mixed_bf16x3")     # compute types without ragged launches


def effective_precision(precision: str, N: int) -> str:
    """The compute type a request of class `precision` runs in at grid size N."""
    if precision == "mixed":
        return "mixed_sliced" if N in (16, 32) else "f32"
    return precision


# Maxwell-molecule requests run the low-rank radial kernel (plan rank) at the
# largest rank whose approximation error stays well inside the class's own
# error: 5 of 8 terms per direction for FP32 (8e-5 against the full operator,
# FP32's own level is 5e-5 .. 5e-4), 7 for the sliced path (1e-9 against its
# 1e-6 target).
LAMBDA0_RANK = {"f32": 5, "mixed_sliced": 7}


# relative GPU time per cell-evaluation by compute type (measured at N = 32, 25 terms)
SPEED = {"f32": 1.0, "mixed_sliced": 3.2, "mixed_f16x2": 0.83, "f32x2": 7.6, "f64": 23.0}


def cell_cost(N: int, lam: float, prec: str, M: int = 48, Mr: int = 8) -> float:
    """Relative cost of one cell-evaluation: terms x N^3 log2 N^3 x the compute type's speed."""
    terms = M // 2 + 1 if lam == 1.0 else (M // 2) * (LAMBDA0_RANK.get(prec) or Mr) + 1
    return terms * N ** 3 * math.log2(N ** 3) * SPEED.get(prec, 1.0)


@dataclasses.dataclass
class Job:
    rid: int
    arrival_s: float
    n_cells: int
    N: int
    lam: float
    precision: str
    n_evals: int = 10
    dt: float = 1e-2
    f_host: object = None           # optional numpy/torch host array; else generated on the device
    seed: int = 0
    # runtime
    f: object = None
    Q: object = None
    done: int = 0
    bytes: int = 0
    t_admit: float = None
    t_finish: float = None
    compute: str = None             # the compute type the request ran in
    cons_err: tuple = None          # relative (mass, momentum, energy) errors of the last Q, worst cell


class Service:
    def __init__(self, hbm_budget_bytes: float = 120e9, L: float = synth.DEFAULT_L, M: int = 48, Mtheta: int = 4,
                 device: str = "cuda", iter_budget_cells: float = 2048.0, max_wall_s: float = 600.0):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.budget = int(hbm_budget_bytes)
        self.L, self.M, self.Mtheta = L, M, Mtheta
        self.plans = {}
        self.stream = torch.cuda.Stream(device=self.device)
        # tensor-core launches (one per mixed request, few CTAs each) run concurrently on side streams
        self.side = [torch.cuda.Stream(device=self.device) for _ in range(8)]
        self.ws = None
        self.lane_ws = {}
        self.in_use = 0
        self.peak_in_use = 0
        self.stats = collections.Counter()
        # cost budget of one iteration, in N = 32, lambda = 1, FP32 cell-evaluations
        self.iter_budget = iter_budget_cells * cell_cost(32, 1.0, "f32", M=M)
        self.min_cells = 2 * torch.cuda.get_device_properties(self.device).multi_processor_count
        self.max_wall_s = max_wall_s

    # ---------------------------------------------------------------- plans
    def plan(self, N: int, lam: float, prec: str):
        key = (N, float(lam), prec)
        if key not in self.plans:
            Mr = 16 if lam == 1.0 else 8
            io = 1 if prec in ("f32",) + TENSOR else 0
            rank = 0 if lam == 1.0 else LAMBDA0_RANK.get(prec, 0)
            self.plans[key] = coll.Plan(N, self.L, lam=lam, M=self.M, Mtheta=self.Mtheta, Mr=Mr, prec=prec,
                                        io_dtype=io, max_cells=1, device=self.device, rank=rank)
        return self.plans[key]

    def _mix_plan(self, j, lane):
        """Tensor-core plan for job j and the workspace of side stream `lane`: one
        plan per (N, lambda) serves every lane (a plan is immutable; each
        concurrent launch needs only its own workspace)."""
        p = self.plan(j.N, j.lam, effective_precision(j.precision, j.N))
        need = max(256, coll.coll_workspace_size(p.handle, max(1, j.n_cells)))
        ws = self.lane_ws.get(lane)
        if ws is None or ws.numel() < need:
            self.side[lane].synchronize()            # the old buffer may still be in use on the lane
            ws = self.torch.empty(need, dtype=self.torch.uint8, device=self.device)
            self.lane_ws[lane] = ws
        return p, ws

    def warm_plans(self, Ns=(16, 32, 48, 64), lams=(0.0, 1.0), precisions=("f32", "mixed")):
        """Build every plan the stream can ask for, launch each kernel once on one
        zero cell and run the synthetic request generator once per (N, dtype), so
        that table building, module loading and first-use compilation stay out of
        serving."""
        torch = self.torch
        for N in Ns:
            for lam in lams:
                for p in precisions:
                    prec = effective_precision(p, N)
                    plan = self.plan(N, lam, prec)
                    dt = torch.float64 if prec in ("f32x2", "f64") else torch.float32
                    f = torch.zeros((1, N, N, N), dtype=dt, device=self.device)
                    Q = torch.empty_like(f)
                    if prec in TENSOR and prec != "mixed_sliced":
                        for lane in range(len(self.side)):
                            j = Job(rid=-1, arrival_s=0.0, n_cells=1, N=N, lam=lam, precision=p)
                            pl, ws = self._mix_plan(j, lane)
                            coll.coll_eval_batch(pl.handle, f, Q, 1, ws, stream=self.side[lane])
                    else:
                        groups = [(plan.handle, f, Q)]
                        self._ensure_ws(coll.coll_ragged_workspace_size(groups, [1]))
                        coll.coll_eval_ragged(groups, [1], self.ws, stream=self.stream)
                        coll.coll_advance(f, Q, 0.0, stream=self.stream)
                    # the device-side request generator's own kernels (first use may JIT-compile them)
                    with torch.cuda.stream(self.stream):
                        synth.bimodal_batch_device(1, N, self.L, 0, dtype=dt, device=self.device)
        torch.cuda.synchronize(self.device)

    # -------------------------------------------------------------- memory
    def _job_bytes(self, j: Job) -> int:
        """f and Q of the request plus the workspace its cells need (an upper
        bound: the ragged launch shares one workspace between requests)."""
        prec = effective_precision(j.precision, j.N)
        es = 8 if prec in ("f32x2", "f64") else 4
        ws = coll.coll_workspace_size(self.plan(j.N, j.lam, prec).handle, max(1, j.n_cells))
        return 2 * j.n_cells * j.N ** 3 * es + ws

    def _ensure_ws(self, nbytes: int):
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = self.torch.empty(int(nbytes * 1.25) + 256, dtype=self.torch.uint8, device=self.device)

    def _admit(self, j: Job, now: float):
        torch = self.torch
        prec = effective_precision(j.precision, j.N)
        dt = torch.float64 if prec in ("f32x2", "f64") else torch.float32
        with torch.cuda.stream(self.stream):
            if j.f_host is not None:
                src = torch.as_tensor(j.f_host)
                j.f = src.to(self.device, dt, non_blocking=True)
            else:
                j.f = synth.bimodal_batch_device(j.n_cells, j.N, self.L, j.seed, dtype=dt, device=self.device)
            j.Q = torch.empty_like(j.f)
        j.bytes = self._job_bytes(j)
        self.in_use += j.bytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        j.t_admit = now

    # ------------------------------------------------------------ one step
    def _select(self, active):
        """Oldest requests first, up to the iteration's cost budget, but with at
        least two cells per SM (so that one heavy request does not leave most of
        the GPU idle) and at least one request."""
        chosen, cost, cells = [], 0.0, 0
        for j in sorted(active, key=lambda j: (j.arrival_s, j.rid)):
            c = j.n_cells * cell_cost(j.N, j.lam, effective_precision(j.precision, j.N), M=self.M)
            if chosen and cost + c > self.iter_budget and cells >= self.min_cells:
                continue
            chosen.append(j)
            cost += c
            cells += j.n_cells
        return chosen

    def _iterate(self, active):
        """One evaluation of the selected jobs: one ragged launch per SIMT compute
        type, one ragged launch of the sliced kernel per N for the fixed-point-slice
        jobs, one launch per job for the other tensor-core types, then f += dt Q."""
        chosen = self._select(active)
        by_kind = collections.defaultdict(list)
        for j in chosen:
            prec = effective_precision(j.precision, j.N)
            by_kind[(prec, j.N) if prec == "mixed_sliced" else prec].append(j)
        side_used = []
        for kind, jobs in by_kind.items():
            prec = kind[0] if isinstance(kind, tuple) else kind
            if prec in TENSOR and prec != "mixed_sliced":
                ready = torch_event(self.stream)
                for i, j in enumerate(jobs):
                    st = self.side[i % len(self.side)]
                    st.wait_event(ready)
                    p, ws = self._mix_plan(j, i % len(self.side))
                    coll.coll_eval_batch(p.handle, j.f, j.Q, j.n_cells, ws, stream=st)
                    self.stats["launches"] += 1
                    if st not in side_used:
                        side_used.append(st)
                continue
            for s in range(0, len(jobs), 256):
                chunk = jobs[s:s + 256]
                groups = [(self.plan(j.N, j.lam, prec).handle, j.f, j.Q) for j in chunk]
                cells = [j.n_cells for j in chunk]
                self._ensure_ws(coll.coll_ragged_workspace_size(groups, cells))
                coll.coll_eval_ragged(groups, cells, self.ws, stream=self.stream)
                self.stats["launches"] += 1
        for st in side_used:
            self.stream.wait_event(torch_event(st))
        for j in chosen:
            if j.done + 1 < j.n_evals:
                coll.coll_advance(j.f, j.Q, j.dt, stream=self.stream)
        # requests whose last evaluation this was: conservation check of the last Q
        last = [j for j in chosen if j.done + 1 >= j.n_evals]
        invs = [coll.conservation(j.Q, self.L, stream=self.stream) for j in last]
        self.stream.synchronize()
        for j in chosen:
            j.done += 1
            self.stats["cell_evals"] += j.n_cells
        for j, inv in zip(last, invs):
            e = self.torch.nan_to_num(coll.conservation_errors(inv), nan=0.0).amax(0)
            j.cons_err = tuple(float(x) for x in e.cpu())
            j.compute = effective_precision(j.precision, j.N)

    # ----------------------------------------------------------------- run
    def run(self, jobs, realtime: bool = True, max_wall_s: float = None, keep_outputs: bool = False):
        """Serve jobs (sorted by arrival).  Returns finished jobs and a stats dict.
        realtime=False advances a simulated clock by the measured GPU time
        (deterministic admission order); keep_outputs keeps each finished
        job's final f and last Q on the device."""
        max_wall_s = self.max_wall_s if max_wall_s is None else max_wall_s
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival_s))
        waiting = collections.deque()
        active, finished = [], []
        t0 = time.perf_counter()
        clock = 0.0
        max_q = 0
        while pending or waiting or active:
            now = time.perf_counter() - t0 if realtime else clock
            if now > max_wall_s:
                raise TimeoutError("service exceeded %.0f s" % max_wall_s)
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            # admission: arrival order, skipping requests that do not fit yet
            for j in list(waiting):
                b = self._job_bytes(j)
                if self.in_use + b <= self.budget:
                    waiting.remove(j)
                    self._admit(j, now)
                    active.append(j)
                elif b > self.budget:
                    raise ValueError("request %d needs %d bytes > budget" % (j.rid, b))
            max_q = max(max_q, len(waiting))
            if not active:
                if pending:
                    nxt = pending[0].arrival_s
                    if realtime:
                        time.sleep(max(0.0, min(0.05, nxt - now)))
                    else:
                        clock = nxt
                continue
            t_it = time.perf_counter()
            self._iterate(active)
            if not realtime:
                clock += time.perf_counter() - t_it
            now = time.perf_counter() - t0 if realtime else clock
            still = []
            for j in active:
                if j.done >= j.n_evals:
                    j.t_finish = now
                    self.in_use -= j.bytes
                    if not keep_outputs:
                        j.f = j.Q = None
                    finished.append(j)
                else:
                    still.append(j)
            active = still
        wall = time.perf_counter() - t0 if realtime else clock
        lat = np.array([j.t_finish - j.arrival_s for j in finished])
        cons = np.array([j.cons_err for j in finished if j.cons_err is not None]).reshape(-1, 3)
        by_type = collections.defaultdict(list)
        for j in finished:
            by_type[j.compute].append(j.cons_err[0] if j.cons_err else float("nan"))
        stats = {
            "requests": len(finished),
            "cell_evals": int(self.stats["cell_evals"]),
            "wall_s": wall,
            "cell_evals_per_s": self.stats["cell_evals"] / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "peak_hbm_bytes": int(self.peak_in_use),
            "hbm_budget_bytes": self.budget,
            "max_queue_depth": int(max_q),
            "ragged_launches": int(self.stats["launches"]),
            "requests_by_compute_type": {k: len(v) for k, v in sorted(by_type.items())},
            "conservation_rel_max": ({"mass": float(cons[:, 0].max()), "momentum": float(cons[:, 1].max()),
                                      "energy": float(cons[:, 2].max())} if cons.size else None),
            "mass_rel_max_by_compute_type": {k: float(np.nanmax(v)) for k, v in sorted(by_type.items())},
        }
        return finished, stats

    def close(self):
        self.torch.cuda.synchronize(self.device)
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        self.lane_ws.clear()


def stream_jobs(n_requests=2000, rate_per_s=200.0, seed=synth.BASE_SEED + 5, max_cells=2048,
                Ns=(16, 32, 48, 64), n_evals=10):
    """The serving workload: Poisson arrivals, log-uniform cell counts, mixed N,
    lambda and precision (request_stream recipe), inputs drawn on the device."""
    reqs = synth.request_stream(n_requests, rate_per_s, seed, Ns=Ns, max_cells=max_cells)
    return [Job(r.rid, r.arrival_s, r.n_cells, r.N, r.lam, r.precision, n_evals=n_evals, seed=r.seed) for r in reqs]


def main():
    import argparse
    ap = argparse.ArgumentParser(description="serve a Poisson stream of collision-evaluation requests")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-cells", type=int, default=2048)
    args = ap.parse_args()
    svc = Service(hbm_budget_bytes=args.budget_gb * 1e9)
    svc.warm_plans()
    jobs = stream_jobs(args.requests, args.rate, max_cells=args.max_cells)
    _, stats = svc.run(jobs)
    print(json.dumps(stats))
    svc.close()


if __name__ == "__main__":
    main()
