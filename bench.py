"""Benchmark: forming the sparse FP64 Laplacian differentiation matrix with overlapped RBF-FD.

The headline step is the delta sweep of the largest sweep workload: for each delta in
(1.0, 0.4, 0.2), plan the stencils (kNN, retention balls) and assemble L (traversal with
Lebesgue stabilization, one factorization per center, multi-RHS solves, CSR) for N = 100,000
quasi-uniform nodes in the unit ball, PHS r^7, degree-3 polynomials (M = 20), n = 45.
Metric: matrix rows per second.  The same JSON line carries, under "configs", the 2D square
sweep (N = 40,000), the clustered mixed-degree cube (N = 500,000, eager and replayed from a
captured CUDA graph), a batch of four node sets of different dimension and degree (one graph
against one graph per plan) and the serving trace (256 jobs: 1 slot against 4 slots on the
same arrival traces), each with its own roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--headline-only] [--workload NAME | batch | serve]

Under torchrun (N > 1) every rank forms its own copy of the headline workload (independent
replicas: the method has no exchange step on this path) and rank 0 prints one JSON line with
the aggregate rows/s over the max-over-ranks time.  ``--impl reference`` times the CPU oracle
(the plain sequential restatement of the method) on bounded samples instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ball3d_N100000_l3_n45_r7"      # headline: the largest delta-sweep workload
SWEEP_2D = "square2d_N40000_l4_n31_r7"
MIXED = "cube3d_N500000_mixed_l2to5"
METRIC = "diff-matrix rows/s (FP64, delta sweep)"
UNIT = "rows/s"
# The FP64 pipe of a GB300: 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz = 1.259 TFLOP/s;
# the profiling recipe's nominal figure is 1.25 (the measured peaks file has no FP64 entry).
FP64_PEAK_TFLOPS = 1.25
PEAK_DERIVATION = ("nominal GB300 FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.259 "
                   "TFLOP/s, quoted as 1.25 (profiling recipe); MEASURED_PEAKS.json has no "
                   "FP64 entry")
L2_FLUSH_BYTES = 256 << 20
# bounded oracle sample for the CPU baseline and the reference arm: the headline's recipe and
# stencil parameters at a fifth of its size (the oracle's brute-force kNN is quadratic in N)
ORACLE_SAMPLE_N = 20000


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _workload(name=None):
    """(X, workload dict, (bc, normals) or None)."""
    from paper_1606_03135_gb300 import nodesets as NS
    name = name or WORKLOAD
    if name in NS.BC_WORKLOADS:
        w = NS.BC_WORKLOADS[name]
        X, bc, nrm = w["gen"](**w["kw"])
        return X, w, (bc, nrm)
    w = NS.WORKLOADS[name]
    return NS.make(name), w, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(path):
    """sha256 (16 hex digits) of a CUDA source with its comments and blank space removed, so
    that a comment edit does not invalidate counters taken from the same kernel code."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.strip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _traffic_entry(workload):
    """DRAM traffic of the traversal kernel on `workload` from the committed ncu summary, if
    the kernel source is unchanged since it was captured."""
    path = os.path.join(ROOT, "profiles", "traversal_traffic.json")
    src = os.path.join(ROOT, "paper_1606_03135_gb300", "csrc", "assemble.cu")
    try:
        rec = json.load(open(path))
        h = kernel_source_hash(src)
        if rec.get("assemble_cu_code_sha256_16") == h and rec.get("workload") == workload:
            return rec
    except (OSError, ValueError):
        pass
    return None


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest value of x over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cpu():
    """(threads available to this process, CPU model) of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return cores, model or platform.processor() or platform.machine()


def _oracle_sample(seed):
    return __import__("paper_1606_03135_gb300.nodesets", fromlist=["ball3d"]).ball3d(
        ORACLE_SAMPLE_N, seed=seed)


def oracle_sweep(seed):
    """The oracle as it stands on one host core: the headline's delta sweep (kNN + traversal
    + solves + CSR per delta) on a bounded sample of its recipe.  Returns (rows, seconds)."""
    from oracle import oracle as O
    from paper_1606_03135_gb300 import nodesets as NS
    w = NS.WORKLOADS[WORKLOAD]
    X = _oracle_sample(seed)
    t = time.perf_counter()
    for delta in w["deltas"]:
        O.assemble(X, w["n"], w["ell"], w["m"], delta, O.STAB_SEQ)
    return X.shape[0] * len(w["deltas"]), time.perf_counter() - t


def cpu_baseline_entry():
    """The oracle timed on this host: one core, then every core of the process at once (one
    independent sample per core, a spawn pool, so no state of the GPU process is inherited)."""
    from oracle import oracle as O
    O.build()
    cores, model = host_cpu()
    rows1, t1 = oracle_sweep(3)
    import multiprocessing
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(oracle_sweep, [3 + k for k in range(cores)])
        wall = time.perf_counter() - t0
    rows_all = sum(r for r, _ in res)
    sample = (f"the headline's delta sweep (1.0, 0.4, 0.2; n=45, ell=3, r^7) on the unit-ball "
              f"recipe at N={ORACLE_SAMPLE_N} instead of 100,000 (brute-force kNN is quadratic "
              f"in N): one sweep on 1 core in {t1:.1f} s; {cores} sweeps with their own seeds "
              f"on {cores} cores at once in {wall:.1f} s")
    return {"value": rows_all / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample, "single_core_value": rows1 / t1, "cpu_model": model,
            "nproc": os.cpu_count()}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1606_03135_gb300 import nodesets as NS
    O.build()
    w = NS.WORKLOADS[WORKLOAD]
    X = _oracle_sample(3)
    deltas = w["deltas"]

    def step(k):
        t = time.perf_counter()
        O.assemble(X, w["n"], w["ell"], w["m"], deltas[k % len(deltas)], O.STAB_SEQ)
        return time.perf_counter() - t

    for k in range(args.warmup):
        step(k)
    times = [step(k) for k in range(args.steps)]
    total = sum(times)
    value = X.shape[0] * args.steps / total
    cores, model = host_cpu()
    sample = (f"one delta of the sweep per step (1.0, 0.4, 0.2 in turn), the unit-ball recipe at "
              f"N={ORACLE_SAMPLE_N} (n=45, ell=3, r^7; the workload has N=100,000), "
              f"single-threaded plain C oracle (brute-force kNN)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": ORACLE_SAMPLE_N, "d": 3, "n": w["n"],
                   "ell": w["ell"], "m": w["m"], "deltas": list(deltas), "stab": "seq"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu_model": model, "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


PROBE = None  # FP64 pipe rates measured on this GPU before anything is timed (probe.measure)


def roofline_entry(stats, kernel_ms, kernel, share=None, traffic=None, factor_lu=False):
    """FP64 roofline of the local-solve kernels over the launches in `stats` (rbffd_stats
    dicts) taking `kernel_ms` of device time (CUDA events on the launching stream).
    flops_executed: (1/3) K^3 per LDL^T factorization ((2/3) K^3 for LU) + 2 K^2 per solved
    column (every retained node, kept or rejected); flops_survey: the cost model's
    (2/3) K^3 + 2 K^2 p.  The refinement step's work is reported beside, not counted."""
    k3 = sum(s["sum_k3"] for s in stats)
    k2c = sum(s["sum_k2_cols"] for s in stats)
    executed = (2.0 / 3.0 if factor_lu else 1.0 / 3.0) * k3 + 2.0 * k2c
    survey = 2.0 / 3.0 * k3 + 2.0 * k2c
    sec = kernel_ms / 1e3
    achieved = executed / sec / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "flops_executed": executed, "flops_survey": survey,
            "frac_survey": survey / sec / 1e12 / FP64_PEAK_TFLOPS,
            "flops_refine": sum(s["flops_refine"] for s in stats),
            "peak_source": PEAK_DERIVATION, "traffic": traffic, "share_of_step": share,
            "kernel_ms": kernel_ms,
            **({"peak_measured_dfma": PROBE["dfma"]["tflops"],
                "frac_of_measured_dfma": achieved / PROBE["dfma"]["tflops"],
                "dmma_tflops_measured": PROBE["dmma"]["tflops"],
                "peak_probe": "include/fp64_probe.h: independent DFMA chains and FP64 "
                              "mma.sync m8n8k4 tiles on every SM, CUDA events, best of 3"}
               if PROBE else {})}


def run_sweep(args, name, dev, world=1, e2e=True, steps=None, warmup=None):
    """One delta sweep workload: autotuned schedules, `steps` timed steps (L2 flushed
    between them), the end-to-end form with host buffers.  Returns the JSON fields."""
    import torch
    from paper_1606_03135_gb300 import rbffd as R
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    X, w, bcw = _workload(name)
    N, n, ell, m, deltas = X.shape[0], w["n"], w["ell"], w["m"], w["deltas"]
    d = X.shape[1]
    Xd = torch.from_numpy(X).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ts_buf = {delta: torch.empty(N * n, dtype=torch.float64, device=dev) for delta in deltas} \
        if bcw is not None else None
    stream = torch.cuda.current_stream(dev)
    copy_stream = torch.cuda.Stream(dev)
    plan_stream = torch.cuda.Stream(dev)
    # with --concurrent-deltas each delta's assembly runs on its own stream, and CTAs of a
    # traversal's dependency tail leave (rbffd_opts.elastic) so the next delta's kernel fills
    # their SMs
    conc = getattr(args, "concurrent_deltas", False)
    fresh = getattr(args, "fresh_plans", False)  # every delta runs its own kNN
    asm_streams = [torch.cuda.Stream(dev) for _ in deltas] if conc else [stream] * len(deltas)
    elastic = args.elastic if conc else 0
    # Schedule per delta (team size, grid cap, right-hand sides per factorization), chosen by
    # timing the candidates on this node set before anything is timed; the matrix does not
    # depend on it.
    sched = {delta: {} for delta in deltas}
    if not args.no_autotune:
        for delta in deltas:
            sched[delta], _ = R.autotune(Xd, n, ell, m, delta, repeats=3)

    def one_step(detail=None, nodes=None, host_out=False, spans=None, end_event=None):
        # The sweep keeps its plans (and their CSR) on the device until every delta is
        # assembled, so the host plans the next delta while the GPU assembles the current one.
        # Each delta's plan (kNN, retention balls: independent of the other deltas) is built
        # on a side stream, so it runs while the previous delta assembles and the host's wait
        # for its sizing covers only its own stencils; the assemblies run in order on the
        # compute stream.
        # The kNN stencils do not depend on delta (§4.1): the first delta's plan searches them
        # and the others copy them from it (rbffd_plan_delta), recomputing only their balls.
        launches = 0
        d2h = 0
        plans, sts = [], []
        plan_stream.wait_stream(stream)  # (after the step's start event)
        for k, delta in enumerate(deltas):
            kw = dict(sync=False, stream=plan_stream, elastic=elastic, **sched[delta])
            if k == 0 or fresh:
                p = R.Plan(Xd if nodes is None else nodes, n, ell, m, delta, **kw)
            else:
                p = plans[0][1].with_delta(delta, **kw)
            if bcw is not None:  # boundary rows and the time-stepping matrix of §5
                p.set_boundary(*bcw)
            s_k = asm_streams[k]
            if s_k is not stream:
                s_k.wait_stream(stream)
            if spans is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(s_k)
            p.assemble(stream=s_k)
            if bcw is not None:
                p.timestep_matrix(w["timestep_c"], out=ts_buf[delta])
            if spans is not None:
                f = torch.cuda.Event(enable_timing=True)
                f.record(s_k)
                spans.append((e, f))
            plans.append((delta, p))
        for s_k in asm_streams:
            if s_k is not stream:
                stream.wait_stream(s_k)
        if end_event is not None:  # the step's device work ends with the last assembly
            end_event.record(stream)
        if host_out:  # into pinned host buffers allocated once, on a copy stream: one delta's
            for delta, p in plans:  # copies overlap the next deltas' assembly
                row_ptr, col, val, owner = p.export_async(host_out[delta], copy_stream)
                d2h += row_ptr.nbytes + col.nbytes + val.nbytes + owner.nbytes
        for delta, p in plans:
            st = p.stats()  # (waits for the plan's copies too)
            if st["status"] != 0:
                raise RuntimeError(f"delta {delta}: {R.rbffd_strerror(st['status'])}")
            launches += st["n_launches"]
            sts.append(st)
            if detail is not None:
                detail.setdefault(delta, []).append(st)
            p.close()
        return launches, sts, d2h

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    detail = {}
    launches = 0
    all_st = []
    spans = [[] for _ in range(steps)]
    ev_host = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.fill_(float(k))  # evict L2 between timed steps (not inside a step's events)
            ev[k][0].record(stream)
            l, sts, _ = one_step(detail, spans=spans[k], end_event=ev[k][1])
            ev_host[k].record(stream)
            launches += l
            all_st += sts
        barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    # (the host then reads each plan's counters and frees it: up to the event after that)
    host_ms = [e0.elapsed_time(h) for (e0, _), h in zip(ev, ev_host)]
    # device time of the assemblies (traversal + its small init and CSR launches): the union
    # of their intervals, so that assemblies running side by side count once
    asm_union_ms = 0.0
    for k in range(steps):
        iv = sorted((ev[k][0].elapsed_time(a), ev[k][0].elapsed_time(b)) for a, b in spans[k])
        lo, hi = iv[0]
        for a, b in iv[1:]:
            if a > hi:
                asm_union_ms += hi - lo
                lo, hi = a, b
            else:
                hi = max(hi, b)
        asm_union_ms += hi - lo
    total_ms = max_over_ranks(sum(step_ms), dev)
    rows = N * len(deltas) * steps * world
    value = rows / (total_ms / 1e3)

    out = {"value": value, "ms_per_step": total_ms / steps, "steps": steps, "warmup": warmup,
           "ms_per_step_with_host_readout": sum(host_ms) / steps,
           "config": {"workload": name, "N": N, "d": d, "n": n, "ell": ell, "m": m,
                      "deltas": list(deltas), "stab": "seq",
                      **({"boundary": f"{int((bcw[0] > 0).sum())} boundary rows (kind "
                                      f"{int(bcw[0].max())}) + time-stepping matrix c="
                                      f"{w['timestep_c']:.3g}"} if bcw is not None else {}),
                      "l2": "flushed between timed steps (256 MB write)",
                      "plans": ("each delta's own kNN" if fresh else
                                "one kNN per step: the first delta's plan searches the stencils, "
                                "the others copy them and recompute their balls "
                                "(rbffd_plan_delta)") +
                               "; built on a side stream beside the previous delta's assembly "
                               "(per_delta ms_stencils of later deltas include that overlap)",
                      "schedule": ({str(k): v for k, v in sched.items()}
                                   if not args.no_autotune else "library default"),
                      "deltas_concurrent": bool(conc), "elastic": elastic},
           "gpu_launches": launches, "clocks": clk.summary()}

    if e2e:  # end to end through the public API with host buffers: host nodes in, host CSR
        # out, both in pinned memory allocated once (as a caller that streams node sets would)
        e2e_steps = max(1, min(steps, 5))
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        X_pinned = pin(X.shape, torch.float64)
        X_pinned[...] = X
        bufs = {delta: (pin(N + 1, torch.int64), pin(N * n, torch.int32),
                        pin(N * n, torch.float64), pin(N, torch.int32)) for delta in deltas}
        one_step(nodes=X_pinned, host_out=bufs)  # warm-up of the host path
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(e2e_steps):
            _, _, d2h = one_step(nodes=X_pinned, host_out=bufs)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        out["e2e"] = {"value": N * len(deltas) * e2e_steps * world / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": int(X.nbytes * (len(deltas) if fresh else 1)),
                      "d2h_bytes_per_step": int(d2h)}

    # the traversal kernels' device time: their own events when they run one after another,
    # else the union of the assemblies' intervals (which adds the tiny init and CSR launches)
    trav_ms = asm_union_ms if conc else sum(s["ms_traversal"] for s in all_st)
    tr = _traffic_entry(name)
    out["roofline"] = roofline_entry(
        all_st, trav_ms, "k_traversal (FP64 LDL^T factorization + solves, persistent)"
        + ("; time = union of the concurrent assemblies' intervals" if conc else ""),
        share=trav_ms / total_ms * world, traffic=(tr["bytes_per_launch"] if tr else None))
    per_delta = {}
    for delta, sts in detail.items():
        per_delta[str(delta)] = {
            "n_centers": sts[-1]["n_centers"], "sum_cols": sts[-1]["sum_cols"],
            "ms_stencils": statistics.median(s["ms_stencils"] for s in sts),
            "ms_traversal": statistics.median(s["ms_traversal"] for s in sts),
            "ms_finalize": statistics.median(s["ms_finalize"] for s in sts),
            "traversal_tflops_executed": statistics.median(
                (s["sum_k3"] / 3.0 + 2.0 * s["sum_k2_cols"]) / s["ms_traversal"] / 1e9
                for s in sts)}
    out["per_delta"] = per_delta
    from paper_1606_03135_gb300 import model as CM
    M_terms = math.comb(ell + d, d)
    out["speedup_model"] = CM.sweep_report(
        {float(k): {"n_centers": v["n_centers"], "sum_cols": v["sum_cols"],
                    "ms_traversal": v["ms_traversal"]} for k, v in per_delta.items()},
        N, n, M_terms, d)
    return out


def run_mixed_config(args, steps=3, warmup=1):
    """The mixed-degree workload: one plan + assemble per step on the clustered cube with
    per-node degree 2..5 (n = 2M + 1), delta = 0.3, FALLBACK stabilization; then the same
    assembly replayed from one captured CUDA graph."""
    import torch
    from paper_1606_03135_gb300 import nodesets as NS
    from paper_1606_03135_gb300 import rbffd as R
    name = args.workload if args.workload in NS.MIXED_WORKLOADS else MIXED
    w = NS.MIXED_WORKLOADS[name]
    X = w["gen"](**w["kw"])
    n_node, ell_node, m_node = NS.mixed_degree_params(X, w["ells"])
    Xd = torch.from_numpy(X).cuda()
    delta = w["deltas"][0]
    stream = torch.cuda.current_stream()
    # schedule picked by the autotuner on this node set (untimed, like a library's heuristics)
    sched, sched_ms = R.autotune(Xd, n_node, ell_node, m_node, delta, mode=R.STAB_FALLBACK,
                                 repeats=1)

    def step():
        p = R.Plan(Xd, n_node, ell_node, m_node, delta, mode=R.STAB_FALLBACK, **sched)
        p.assemble()
        st = p.stats()
        p.close()
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    sts = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            ev[k][0].record(stream)
            sts.append(step())
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    N = X.shape[0]
    st = sts[-1]
    solve_ms = sum(x["ms_traversal"] + x["ms_fallback"] for x in sts)
    out = {"value": N * steps / (total_ms / 1e3), "unit": UNIT, "steps": steps,
           "warmup": warmup, "ms_per_step": total_ms / steps,
           "config": {"workload": name, "N": N, "d": 3, "ells": list(w["ells"]),
                      "n_max": int(n_node.max()), "delta": delta, "stab": "fallback",
                      "refine": "auto (pivot ratio >= 2^16)"},
           "roofline": roofline_entry(sts, solve_ms, "k_traversal + k_fallback_solve (FP64 "
                                      "LDL^T local solves, refined where ill-conditioned)",
                                      share=solve_ms / total_ms),
           "split_ms": {k: statistics.median(x[k] for x in sts)
                        for k in ("ms_stencils", "ms_traversal", "ms_fallback", "ms_finalize")},
           "stats": {k: st[k] for k in ("n_centers", "n_fallback", "n_rejected", "sum_cols",
                                        "max_ball", "nnz")},
           "clocks": clk.summary()}
    # the assembly as one captured CUDA graph (plan outside the graph), replayed
    with R.Plan(Xd, n_node, ell_node, m_node, delta, mode=R.STAB_FALLBACK, sync=False,
                **sched) as p:
        p.assemble()
        torch.cuda.synchronize()
        g = p.capture_assemble()
        g.replay()
        torch.cuda.synchronize()
        gs = torch.cuda.Stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(gs):
            e0.record(gs)
            for _ in range(steps):
                g.replay()
            e1.record(gs)
        torch.cuda.synchronize()
        rep_ms = e0.elapsed_time(e1) / steps
        gst = p.stats()
        if gst["status"] != 0:
            raise RuntimeError(f"graph replay: {R.rbffd_strerror(gst['status'])}")
    out["schedule"] = {"autotuned": {k: int(v) for k, v in sched.items()},
                       "candidates_ms": {str(dict(k)): round(v, 3) for k, v in sched_ms.items()}}
    out["graph_replay"] = {"ms_per_assembly": rep_ms, "assemble_rows_per_s": N / (rep_ms / 1e3),
                           "eager_assemble_ms": st["ms_traversal"] + st["ms_fallback"]
                           + st["ms_finalize"]}
    return out


def run_batch_config(args, steps=5, warmup=2):
    """Batching across dimensions and degrees: four node sets (2D square, degree 4; 3D ball,
    degree 3; 2D disk, degree 5; 3D ball, degree 2), each planned once, their assemblies
    replayed (a) one after another, each from its own captured graph, on one stream (the
    plain per-config path) and (b) from one graph holding all four on concurrent streams: as
    they are, with the elastic traversal grid (tail CTAs leave for the other plans' kernels),
    and with each grid capped to a share of the GPU.
    Rows/s of each and the GPU-wide FP64 rate of the solve kernels."""
    import torch
    from paper_1606_03135_gb300 import nodesets as NS
    from paper_1606_03135_gb300 import rbffd as R
    setups = [("square2d N=40000, ell=4, n=31, r^7, delta=0.5", NS.square2d(40000, seed=2),
               (31, 4, 7), 0.5),
              ("ball3d N=100000, ell=3, n=45, r^7, delta=0.4", NS.ball3d(100000, seed=3),
               (45, 3, 7), 0.4),
              ("disk2d N=20000, ell=5, n=43, r^7, delta=0.3", NS.disk2d(20000, seed=11),
               (43, 5, 7), 0.3),
              ("ball3d N=20000, ell=2, n=21, r^5, delta=0.5", NS.ball3d(20000, seed=12),
               (21, 2, 5), 0.5)]
    rows = sum(X.shape[0] for _, X, _, _ in setups)

    def make(cap, elastic=0):
        ps = []
        for _, X, params, delta in setups:
            p = R.Plan(torch.from_numpy(X).cuda(), *params, delta, sync=False, max_ctas=cap,
                       elastic=elastic)
            p.assemble()
            ps.append(p)
        torch.cuda.synchronize()
        return ps

    def timed(replay, plans):
        for _ in range(warmup):
            replay()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            replay()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        sts = [p.stats() for p in plans]
        for st in sts:
            if st["status"] != 0:
                raise RuntimeError(f"batch replay: {R.rbffd_strerror(st['status'])}")
        rf = roofline_entry(sts, ms, "local-solve kernels of the four plans, over the replay")
        return {"ms_per_batch": ms, "rows_per_s": rows / (ms / 1e3), "fp64_tflops": rf["achieved"],
                "fp64_frac": rf["frac"], "roofline": rf}

    out = {"config": {"workload": "batch of 4: " + "; ".join(n for n, _, _, _ in setups),
                      "rows_per_batch": rows}}
    plans = make(0)
    graphs = [p.capture_assemble() for p in plans]
    out["plain"] = timed(lambda: [g.replay() for g in graphs], plans)
    for p in plans:
        p.close()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    variants = (("batched", 0, 0), ("batched_elastic", 0, sms), ("batched_shared", 4 * sms, 0))
    for name, cap, elastic in variants:
        plans = make(cap, elastic)
        g = R.capture_assemble_batch(plans)
        out[name] = timed(g.replay, plans)
        out[name]["max_ctas"] = cap
        out[name]["elastic"] = elastic
        for p in plans:
            p.close()
    best = max((v[0] for v in variants), key=lambda k: out[k]["rows_per_s"])
    out["value"] = out[best]["rows_per_s"]
    out["roofline"] = out[best]["roofline"]
    out["unit"] = UNIT
    out["speedup"] = out["value"] / out["plain"]["rows_per_s"]
    return out


def run_serve_config(args):
    """The serving workload: a seeded mix of jobs (2D/3D, N log-uniform in [1k, 200k], ell
    2..5, random delta), replayed on equal terms with 1 slot (one job at a time: the plain
    per-config path) and with `slots` slots (continuous batching): saturated (every job
    available at t = 0) and with the same Poisson arrival trace at 0.5 and 0.9 of the
    1-slot saturated rate.  p50/p99 latency, rows/s and the GPU-wide FP64 rate of each."""
    from paper_1606_03135_gb300 import serve as S
    count = args.jobs
    jobs = S.serving_jobs(count=count)
    warm = S.serving_jobs(count=4, seed=77, n_min=1000, n_max=5000)
    S.Server(slots=1, keep_results=False).run(warm)
    S.Server(slots=args.slots, keep_results=False).run(warm)

    def summarise(results, summ):
        sts = [r.stats for r in results if r.error is None and r.stats]
        solve_ms = sum(s["ms_traversal"] + s["ms_fallback"] for s in sts)
        rf = roofline_entry(sts, summ["makespan_s"] * 1e3, "local-solve kernels of every job, "
                            "over the makespan (GPU-wide FP64 rate)")
        keep = ("jobs", "failed", "rows", "makespan_s", "rows_per_s", "p50_latency_s",
                "p99_latency_s", "peak_reserved_bytes", "slots")
        return {**{k: summ[k] for k in keep}, "fp64_tflops": rf["achieved"],
                "fp64_frac": rf["frac"], "solve_kernel_ms": solve_ms, "roofline": rf}

    out = {"config": {"workload": f"serve{count}: d in {{2,3}}, N log-uniform [1k,200k], "
                                  "ell 2..5, n=2M+1, delta U[0.2,1]", "hbm_budget_gb": 40,
                      "slots": args.slots,
                      "overlap": "full traversal grids; with several slots a job's CTAs leave "
                                 "its dependency tail (elastic = SM count) for the next job"},
           "saturated": {}, "poisson": {}}
    for j in jobs:
        j.arrival = 0.0
    for slots in (1, args.slots):
        res, summ = S.Server(slots=slots, keep_results=False).run(jobs)
        out["saturated"][f"{slots}_slot"] = summarise(res, summ)
    rate1 = count / out["saturated"]["1_slot"]["makespan_s"]
    for load in (0.5, 0.9):
        S.poisson_arrivals(jobs, rate=load * rate1)
        out["poisson"][str(load)] = {}
        for slots in (1, args.slots):
            res, summ = S.Server(slots=slots, keep_results=False).run(jobs)
            out["poisson"][str(load)][f"{slots}_slot"] = summarise(res, summ)
    sat = out["saturated"]
    out["value"] = sat[f"{args.slots}_slot"]["rows_per_s"]
    out["roofline"] = sat[f"{args.slots}_slot"]["roofline"]  # (the served form, saturated)
    out["unit"] = UNIT
    out["speedup_saturated"] = sat[f"{args.slots}_slot"]["rows_per_s"] / sat["1_slot"]["rows_per_s"]
    return out


def run_gpu(args):
    import torch
    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1606_03135_gb300 import rbffd as R
    from paper_1606_03135_gb300 import probe as P
    R.load()
    global PROBE
    PROBE = P.measure(iters=5000, repeats=3)
    name = args.workload or WORKLOAD
    t_start = time.perf_counter()
    h = run_sweep(args, name, dev, world=world)
    line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world,
            "steps": h["steps"], "warmup": h["warmup"], "ms_per_step": h["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {**h["config"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": h["roofline"], "cpu_baseline": None, "e2e": h["e2e"],
            "gpu_launches": h["gpu_launches"], "clocks": h["clocks"],
            "per_delta": h["per_delta"], "speedup_model": h["speedup_model"],
            "fp64_probe": PROBE}
    if rank == 0 and world == 1 and args.workload is None and not args.headline_only:
        cfg = {}
        s2 = run_sweep(args, SWEEP_2D, dev, e2e=True)
        cfg[SWEEP_2D] = {k: s2[k] for k in ("value", "ms_per_step", "steps", "roofline", "e2e",
                                            "per_delta", "gpu_launches", "clocks")}
        cfg[SWEEP_2D]["schedule"] = s2["config"]["schedule"]
        cfg[MIXED] = run_mixed_config(args)
        cfg["batch"] = run_batch_config(args)
        cfg["serve"] = run_serve_config(args)
        line["configs"] = cfg
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry()
    line["bench_wall_s"] = time.perf_counter() - t_start
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="the library's default schedule instead of one tuned per delta "
                         "(rbffd.autotune, before the timed region)")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline sweep (no 2D, mixed or serving configs)")
    ap.add_argument("--workload", default=None,
                    help="one named delta-sweep workload instead of the default set, "
                         f"'{MIXED}', 'batch' or 'serve'")
    ap.add_argument("--concurrent-deltas", action="store_true",
                    help="assemble the deltas of a sweep on concurrent streams with an "
                         "elastic traversal grid (rbffd_opts.elastic)")
    ap.add_argument("--elastic", type=int, default=152,
                    help="waiting CTAs beyond which a traversal CTA leaves (with "
                         "--concurrent-deltas)")
    ap.add_argument("--fresh-plans", action="store_true",
                    help="every delta of a sweep runs its own kNN instead of copying the first "
                         "delta's stencils")
    ap.add_argument("--jobs", type=int, default=256, help="serving trace length")
    ap.add_argument("--slots", type=int, default=4, help="serving slots (streams)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    from paper_1606_03135_gb300 import nodesets as NS
    if args.workload in ("serve", "batch") or args.workload in NS.MIXED_WORKLOADS:
        import torch
        from paper_1606_03135_gb300 import rbffd as R
        R.load()
        torch.cuda.set_device(0)
        out = run_serve_config(args) if args.workload == "serve" else \
            run_batch_config(args) if args.workload == "batch" else \
            run_mixed_config(args, steps=args.steps, warmup=args.warmup)
        print(json.dumps({"metric": "serving rows/s and p50/p99 latency (FP64)"
                          if args.workload == "serve" else METRIC, **out}), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
