"""Serving loop: continuous batching of differentiation-matrix assembly jobs on one GPU.

Jobs (a node set plus n, ell, m, delta) arrive over time.  A job is admitted when a slot
(a CUDA stream with a host worker thread) is free and its device memory fits the remaining
HBM budget; jobs that arrive while others run are admitted as slots and memory free up, and
the admitted jobs' kernels overlap on the device.  Each job's persistent traversal grid fills
the GPU, and with several slots its CTAs leave the job's dependency tail once enough others
wait (``rbffd_opts.elastic``), so the next job's kernels take over those SMs; a per-slot
grid cap (``share_gpu``) is the other way to run jobs side by side.  Every step of every job
runs in the library's kernels; this module only schedules.

The per-stencil computations do not depend on what else is running, so a job's matrix is
bit-identical alone and in the mix.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import nodesets as NS


@dataclass
class Job:
    rid: int
    nodes: np.ndarray          # [N][d] float64, host
    n: int
    ell: int
    m: int
    delta: float
    arrival: float = 0.0       # seconds after the trace starts
    mode: int = 0              # RBFFD_STAB_*


@dataclass
class Result:
    rid: int
    rows: int
    t_arrival: float
    t_admit: float
    t_done: float
    row_ptr: np.ndarray = field(repr=False, default=None)
    col: np.ndarray = field(repr=False, default=None)
    val: np.ndarray = field(repr=False, default=None)
    owner: np.ndarray = field(repr=False, default=None)
    stats: dict = field(repr=False, default=None)
    error: str = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def estimate_bytes(N: int, d: int, n: int, delta: float, ell: int = None) -> int:
    """Upper bound of the device bytes a uniform-stencil job holds at once: the plan's stencil
    arrays, the cell-grid scratch of its kNN step, and the traversal and CSR arrays of its
    assembly, with every retention ball bounded by the stencil size (one node at delta = 1),
    plus 1 MB for alignment and small tables.  Plans of K = n + C(ell + d, d) >= 100 unknowns
    refine ill-conditioned solves by default, and their assembly then keeps, per resident CTA,
    the full K x K system, its first solutions and the residual's partial sums: at most 5 times
    the CTA's shared-memory system, so under 200 MB on a 152-SM GB300 (228 KB of shared memory
    per SM); without `ell` that is assumed.  The exact figure is known after the plan (rbffd_stats: plan_bytes
    + assemble_bytes) and never exceeds this."""
    ball = 1 if delta >= 1.0 else n
    plan = N * (d * 8 + n * 4 + 8 + 4 + 4 + 8) + (2 * N + 64) * 12 + N * (8 + 8 * d)
    asm = N * (4 * 6 + 2 + n * 12 + 16) + N * ball * (n * 8 + 9)
    refined = ell is None or n + math.comb(ell + d, d) >= 100
    return int(plan + asm + (1 << 20) + ((200 << 20) if refined else 0))


class Budget:
    """Admission control: slots and device bytes, FIFO.  A reservation is taken before a job
    allocates anything, so the budget holds at allocation time; nothing waits while it holds
    a slot (a reservation that would have to grow beyond the budget fails the job)."""

    def __init__(self, slots: int, budget_bytes: int):
        self.slots = slots
        self.budget = budget_bytes
        self.free_slots = slots
        self.in_use = 0
        self.peak = 0
        self.cv = threading.Condition()

    def admit(self, need: int):
        """Wait for a free slot and `need` bytes (jobs that can never fit raise MemoryError)."""
        if need > self.budget:
            raise MemoryError(f"job needs {need} bytes > budget {self.budget}")
        with self.cv:
            while self.free_slots == 0 or self.in_use + need > self.budget:
                self.cv.wait()
            self.free_slots -= 1
            self.in_use += need
            self.peak = max(self.peak, self.in_use)

    def resize(self, old: int, new: int):
        """Correct a held reservation once the exact size is known.  Shrinking always works;
        growing never waits (the job holds a slot, and two growing jobs could wait on each
        other): it succeeds if the budget has room now, else raises MemoryError and the
        reservation stays `old`."""
        with self.cv:
            if new > old and self.in_use - old + new > self.budget:
                raise MemoryError(f"exact size {new} bytes does not fit the budget "
                                  f"({self.in_use - old} of {self.budget} in use by others)")
            self.in_use += new - old
            self.peak = max(self.peak, self.in_use)
            self.cv.notify_all()

    def release(self, need: int):
        with self.cv:
            self.free_slots += 1
            self.in_use -= need
            self.cv.notify_all()


class Server:
    """Replays a trace of jobs against one GPU with `slots` concurrent streams."""

    def __init__(self, slots: int = 4, budget_bytes: int = 40 << 30, device: int = 0,
                 keep_results: bool = True, share_gpu: bool = False, elastic: int | None = None):
        import torch
        from . import rbffd as R
        self.R = R
        self.torch = torch
        self.slots = slots
        self.device = device
        self.keep = keep_results
        self.budget = Budget(slots, budget_bytes)
        torch.cuda.set_device(device)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        # share_gpu: cap each slot's traversal grid at its share of the GPU
        self.max_ctas = 0 if (slots == 1 or not share_gpu) else max(sms, (sms * 12) // slots)
        # rbffd_opts.elastic for every job (default with several slots: the SM count): traversal
        # CTAs leave a job's dependency tail when that many others wait, so a concurrent job's
        # kernels take their SMs.  Saturated 256-job trace, 4 slots: 3.95 M rows/s with the
        # grid cap, 4.06 M with full grids, 4.12 M with full grids and the elastic tail
        # (1 slot: 3.75 M).
        self.elastic = (sms if elastic is None else elastic) if slots > 1 else 0

    def _run_one(self, job: Job, stream, t0: float, res: Result, reserved: int):
        R = self.R
        p = None
        try:
            with self.torch.cuda.stream(stream):
                p = R.Plan(job.nodes, job.n, job.ell, job.m, job.delta, mode=job.mode,
                           stream=stream, max_ctas=self.max_ctas, elastic=self.elastic)
                st = p.stats()
                exact = st["plan_bytes"] + st["assemble_bytes"]
                self.budget.resize(reserved, exact)  # (raises rather than wait)
                reserved = exact
                p.assemble()
                if self.keep:
                    res.row_ptr, res.col, res.val, res.owner = p.export()
                res.stats = p.stats()
        except Exception as e:  # a failed job is reported, never the process
            res.error = f"{type(e).__name__}: {e}"
        finally:
            if p is not None:
                p.close()
        res.t_done = time.perf_counter() - t0
        return reserved

    def run(self, jobs):
        """Run the trace: job.arrival seconds after the start each job becomes available.
        Returns (results ordered by rid, summary dict)."""
        jobs = sorted(jobs, key=lambda j: (j.arrival, j.rid))
        results = {}
        threads = []
        free = list(range(self.slots))
        free_lock = threading.Lock()
        t0 = time.perf_counter()

        def worker(job, slot, reserved, res):
            try:
                reserved = self._run_one(job, self.streams[slot], t0, res, reserved)
            finally:
                with free_lock:  # hand the stream back before the slot is counted free
                    free.append(slot)
                self.budget.release(reserved)

        for job in jobs:
            now = time.perf_counter() - t0
            if job.arrival > now:
                time.sleep(job.arrival - now)
            N, d = job.nodes.shape
            need = estimate_bytes(N, d, job.n, job.delta, ell=job.ell)
            res = Result(job.rid, N, job.arrival, 0.0, 0.0)
            results[job.rid] = res
            try:
                self.budget.admit(need)  # blocks until a slot and the memory are free
            except MemoryError as e:  # can never fit: reported, the trace goes on
                res.t_admit = res.t_done = time.perf_counter() - t0
                res.error = f"MemoryError: {e}"
                continue
            res.t_admit = time.perf_counter() - t0
            with free_lock:
                slot = free.pop()
            th = threading.Thread(target=worker, args=(job, slot, need, res), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        makespan = time.perf_counter() - t0
        out = [results[k] for k in sorted(results)]
        lat = np.array([r.latency for r in out if r.error is None])
        rows = sum(r.rows for r in out if r.error is None)
        summary = {
            "jobs": len(out), "failed": sum(r.error is not None for r in out),
            "rows": rows, "makespan_s": makespan, "rows_per_s": rows / makespan,
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "peak_reserved_bytes": self.budget.peak, "slots": self.slots,
            "errors": [f"job {r.rid} (N={r.rows}): {r.error}" for r in out if r.error][:5],
        }
        return out, summary


# ------------------------------------------------------------------ the serving workload
def serving_jobs(count: int = 256, seed: int = 5, n_min: int = 1000, n_max: int = 200000):
    """Seeded mix of jobs: d in {2, 3}; N log-uniform in [n_min, n_max]; ell in {2..5};
    delta uniform in [0.2, 1]; n = 2M + 1; m = 5 for ell = 2, else 7.  Node sets are the
    disk / ball recipes (jittered Halton), each with its own seed."""
    u = NS.uniform(seed, count * 4).reshape(count, 4)
    jobs = []
    for i in range(count):
        d = 2 if u[i, 0] < 0.5 else 3
        N = int(round(math.exp(math.log(n_min) + u[i, 1] * (math.log(n_max) - math.log(n_min)))))
        ell = 2 + min(int(u[i, 2] * 4), 3)
        delta = 0.2 + 0.8 * u[i, 3]
        M = math.comb(ell + d, d)
        n = 2 * M + 1
        m = 5 if ell == 2 else 7
        X = NS.disk2d(N, seed=1000 + i) if d == 2 else NS.ball3d(N, seed=1000 + i)
        jobs.append(Job(i, X, n, ell, m, delta))
    return jobs


def poisson_arrivals(jobs, rate: float, seed: int = 9):
    """Assign Poisson arrival times (rate jobs per second) in job order."""
    gaps = -np.log1p(-NS.uniform(seed, len(jobs))) / rate
    t = np.cumsum(gaps)
    for j, a in zip(jobs, t):
        j.arrival = float(a)
    return jobs
