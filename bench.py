"""Benchmark: forming the sparse FP64 Laplacian differentiation matrix with overlapped RBF-FD.

One step = the delta sweep of the 2D workload: for each delta in (1.0, 0.5, 0.3), plan the
stencils (kNN, retention balls) and assemble L (traversal with Lebesgue stabilization, one
factorization per center, multi-RHS solves, CSR) for N = 40,000 jittered nodes in the unit
square, PHS r^7, degree-4 polynomials (M = 15), n = 31.  Metric: matrix rows per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank forms its own copy of the workload (independent replicas:
the method has no exchange step on this path) and rank 0 prints one JSON line with the
aggregate rows/s over the max-over-ranks time.  ``--impl reference`` times the CPU oracle
(the plain sequential restatement of the method) instead, one delta of the sweep per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "square2d_N40000_l4_n31_r7"
METRIC = "diff-matrix rows/s (FP64, delta sweep)"
UNIT = "rows/s"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (no FP64 entry in the measured peaks)
L2_FLUSH_BYTES = 256 << 20


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


def _traffic_entry():
    """DRAM traffic of the traversal kernel from the committed ncu summary, if the kernel
    source is unchanged since it was captured."""
    path = os.path.join(ROOT, "profiles", "traversal_traffic.json")
    src = os.path.join(ROOT, "paper_1606_03135_gb300", "csrc", "assemble.cu")
    try:
        rec = json.load(open(path))
        h = kernel_source_hash(src)
        if rec.get("assemble_cu_code_sha256_16") == h:
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


def cpu_oracle_step(X, w, delta, bcw=None):
    """The oracle as it stands, on this host's cores: kNN + traversal + solves + CSR."""
    from oracle import oracle as O
    t = time.perf_counter()
    bc, nrm = bcw if bcw is not None else (None, None)
    O.assemble(X, w["n"], w["ell"], w["m"], delta, O.STAB_SEQ, bc=bc, normals=nrm)
    return time.perf_counter() - t


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    X, w, _ = _workload()
    deltas = w["deltas"]
    for s in range(args.warmup):
        cpu_oracle_step(X, w, deltas[s % len(deltas)])
    times = []
    for s in range(args.steps):
        times.append(cpu_oracle_step(X, w, deltas[s % len(deltas)]))
    total = sum(times)
    rows = X.shape[0] * args.steps
    value = rows / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": X.shape[0], "d": 2, "n": w["n"], "ell": w["ell"],
                   "m": w["m"], "deltas": list(deltas), "stab": "seq"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one delta of the sweep per step, full N=40000 node set, "
                                   "single-threaded plain C oracle (brute-force kNN)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1606_03135_gb300 import rbffd as R
    R.load()
    X, w, bcw = _workload(args.workload)
    N, n, ell, m, deltas = X.shape[0], w["n"], w["ell"], w["m"], w["deltas"]
    d = X.shape[1]
    Xd = torch.from_numpy(X).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ts_buf = {delta: torch.empty(N * n, dtype=torch.float64, device=dev) for delta in deltas} \
        if bcw is not None else None
    stream = torch.cuda.current_stream(dev)
    copy_stream = torch.cuda.Stream(dev)
    plan_stream = torch.cuda.Stream(dev)
    # Schedule per delta (team size, grid cap, right-hand sides per factorization), chosen by
    # timing the candidates on this node set before anything is timed; the matrix does not
    # depend on it.
    sched = {delta: {} for delta in deltas}
    if not args.no_autotune:
        for delta in deltas:
            sched[delta], _ = R.autotune(Xd, n, ell, m, delta, repeats=3)

    def one_step(detail=None, nodes=None, host_out=False):
        # The sweep keeps its plans (and their CSR) on the device until every delta is
        # assembled, so the host plans the next delta while the GPU assembles the current one.
        # Each delta's plan (kNN, retention balls: independent of the other deltas) is built
        # on a side stream, so it runs while the previous delta assembles and the host's wait
        # for its sizing covers only its own stencils; the assemblies run in order on the
        # compute stream.
        launches = 0
        alg = trav_ms = 0.0
        d2h = 0
        plans = []
        plan_stream.wait_stream(stream)  # (after the step's start event)
        for delta in deltas:
            p = R.Plan(Xd if nodes is None else nodes, n, ell, m, delta, sync=False,
                       stream=plan_stream, **sched[delta])
            if bcw is not None:  # boundary rows and the time-stepping matrix of §5
                p.set_boundary(*bcw)
            p.assemble(stream=stream)
            if bcw is not None:
                p.timestep_matrix(w["timestep_c"], out=ts_buf[delta])
            plans.append((delta, p))
        if host_out:  # into pinned host buffers allocated once, on a copy stream: one delta's
            for delta, p in plans:  # copies overlap the next deltas' assembly
                row_ptr, col, val, owner = p.export_async(host_out[delta], copy_stream)
                d2h += row_ptr.nbytes + col.nbytes + val.nbytes + owner.nbytes
        for delta, p in plans:
            st = p.stats()  # (waits for the plan's copies too)
            if st["status"] != 0:
                raise RuntimeError(f"delta {delta}: {R.rbffd_strerror(st['status'])}")
            launches += st["n_launches"]
            alg += st["alg_flops"]
            trav_ms += st["ms_traversal"]
            if detail is not None:
                detail.setdefault(delta, []).append(st)
            p.close()
        return launches, alg, trav_ms, d2h

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    detail = {}
    launches = 0
    alg = trav_ms = 0.0
    barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s in range(args.steps):
            flush.fill_(float(s))  # evict L2 between timed steps (not inside a step's events)
            ev[s][0].record(stream)
            l, a, t, _ = one_step(detail)
            ev[s][1].record(stream)
            launches += l
            alg += a
            trav_ms += t
        barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    rows = N * len(deltas) * args.steps * world
    value = rows / (total_ms / 1e3)

    # end to end through the public API with host buffers: host nodes in, host CSR out, both
    # in pinned memory allocated once (as a caller that streams many node sets would)
    e2e_steps = max(1, min(args.steps, 5))
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    X_pinned = pin(X.shape, torch.float64)
    X_pinned[...] = X
    bufs = {delta: (pin(N + 1, torch.int64), pin(N * n, torch.int32), pin(N * n, torch.float64),
                    pin(N, torch.int32)) for delta in deltas}
    one_step(nodes=X_pinned, host_out=bufs)  # warm-up of the host path
    barrier()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        _, _, _, d2h = one_step(nodes=X_pinned, host_out=bufs)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = N * len(deltas) * e2e_steps * world / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        t_cpu = cpu_oracle_step(X, w, deltas[1], bcw)
        cpu = {"value": N / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full assembly at delta={deltas[1]} (N={N}, kNN + traversal + "
                         f"solves + CSR), single-threaded plain C oracle, {t_cpu:.1f} s"}

    achieved = alg / (trav_ms / 1e3) / 1e12  # TFLOP/s of the traversal kernel
    tr = _traffic_entry()
    roofline = {"bound": "alu", "kernel": "k_traversal (FP64 LDL^T + solves)",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (profiling recipe); "
                               "MEASURED_PEAKS.json has no FP64 entry",
                "traffic": (tr["bytes_per_launch"] if tr else None),
                "share_of_step": trav_ms / total_ms}
    per_delta = {}
    for delta, sts in detail.items():
        per_delta[str(delta)] = {
            "n_centers": sts[-1]["n_centers"], "sum_cols": sts[-1]["sum_cols"],
            "ms_stencils": statistics.median(s["ms_stencils"] for s in sts),
            "ms_traversal": statistics.median(s["ms_traversal"] for s in sts),
            "ms_finalize": statistics.median(s["ms_finalize"] for s in sts),
            "traversal_tflops": statistics.median(s["alg_flops"] / s["ms_traversal"] / 1e9
                                                  for s in sts)}
    from paper_1606_03135_gb300 import model as CM
    M_terms = math.comb(ell + d, d)
    speedup = CM.sweep_report({float(k): {"n_centers": v["n_centers"], "sum_cols": v["sum_cols"],
                                          "ms_traversal": v["ms_traversal"]}
                               for k, v in per_delta.items()}, N, n, M_terms, d)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload or WORKLOAD, "N": N, "d": d, "n": n, "ell": ell, "m": m,
                   "deltas": list(deltas), "stab": "seq",
                   **({"boundary": f"{int((bcw[0] > 0).sum())} boundary rows (kind "
                                   f"{int(bcw[0].max())}) + time-stepping matrix c="
                                   f"{w['timestep_c']:.3g}"} if bcw is not None else {}),
                   "l2": "flushed between timed steps (256 MB write)",
                   "plans": "built on a side stream beside the previous delta's assembly "
                            "(per_delta ms_stencils of later deltas include that overlap)",
                   "schedule": ({str(k): v for k, v in sched.items()} if not args.no_autotune
                                else "library default"),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "speedup_model": speedup,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(X.nbytes * len(deltas)),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches, "clocks": clk.summary(), "per_delta": per_delta,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_mixed(args):
    """The mixed-degree workload: one plan + assemble per step on the clustered cube with
    per-node degree 2..5 (n = 2M + 1), delta = 0.3, FALLBACK stabilization."""
    import torch
    from paper_1606_03135_gb300 import nodesets as NS
    from paper_1606_03135_gb300 import rbffd as R
    R.load()
    torch.cuda.set_device(0)
    name = args.workload
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

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sts = []
    for s_ in range(args.steps):
        ev[s_][0].record(stream)
        sts.append(step())
        ev[s_][1].record(stream)
    torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    N = X.shape[0]
    st = sts[-1]
    trav = sum(x["ms_traversal"] + x["ms_fallback"] for x in sts)
    alg = sum(x["alg_flops"] for x in sts)
    line = {"metric": METRIC, "value": N * args.steps / (total_ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": name, "N": N, "d": 3, "ells": list(w["ells"]),
                       "n_max": int(n_node.max()), "delta": delta, "stab": "fallback"},
            "roofline": {"bound": "alu", "achieved": alg / (trav / 1e3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": alg / (trav / 1e3) / 1e12 / FP64_PEAK_TFLOPS},
            "stats": {k: st[k] for k in ("n_centers", "n_fallback", "n_rejected", "sum_cols",
                                         "max_ball", "nnz", "ms_stencils", "ms_traversal",
                                         "ms_fallback", "ms_finalize")}}
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
            for _ in range(args.steps):
                g.replay()
            e1.record(gs)
        torch.cuda.synchronize()
        rep_ms = e0.elapsed_time(e1) / args.steps
        gst = p.stats()
        if gst["status"] != 0:
            raise RuntimeError(f"graph replay: {R.rbffd_strerror(gst['status'])}")
    line["schedule"] = {"autotuned": {k: int(v) for k, v in sched.items()},
                        "candidates_ms": {str(dict(k)): round(v, 3) for k, v in sched_ms.items()}}
    line["graph_replay"] = {"ms_per_assembly": rep_ms, "assemble_rows_per_s": N / (rep_ms / 1e3),
                            "eager_assemble_ms": st["ms_traversal"] + st["ms_fallback"]
                            + st["ms_finalize"]}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """The serving workload: a seeded mix of jobs (2D/3D, N log-uniform, ell 2..5, random
    delta) replayed with Poisson arrivals at two offered loads of the measured single-stream
    throughput; prints one JSON line with p50/p99 latency and rows/s per load."""
    import torch
    from paper_1606_03135_gb300 import serve as S
    from paper_1606_03135_gb300 import rbffd as R
    R.load()
    torch.cuda.set_device(0)
    count = args.jobs
    jobs = S.serving_jobs(count=count)
    warm = S.serving_jobs(count=4, seed=77, n_min=1000, n_max=5000)
    S.Server(slots=1, keep_results=False).run(warm)
    for j in jobs:
        j.arrival = 0.0
    _, single = S.Server(slots=1, keep_results=False).run(jobs)
    rate1 = count / single["makespan_s"]
    out = {"metric": "serving rows/s and p50/p99 latency (FP64)", "unit": "rows/s",
           "value": None, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"serve{count}: d in {{2,3}}, N log-uniform [1k,200k], "
                                  "ell 2..5, n=2M+1, delta U[0.2,1], Poisson arrivals",
                      "slots": args.slots, "hbm_budget_gb": 40},
           "single_stream": {"rows_per_s": single["rows_per_s"],
                             "makespan_s": single["makespan_s"]},
           "loads": {}}
    for load in (0.5, 0.9):
        S.poisson_arrivals(jobs, rate=load * rate1)
        _, summ = S.Server(slots=args.slots, keep_results=False).run(jobs)
        out["loads"][str(load)] = summ
    out["value"] = out["loads"]["0.9"]["rows_per_s"]
    print(json.dumps(out), flush=True)
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
    ap.add_argument("--workload", default=None,
                    help="another named node-set workload (default: the 2D delta sweep), "
                         "or 'serve' for the serving trace")
    ap.add_argument("--jobs", type=int, default=256, help="serving trace length")
    ap.add_argument("--slots", type=int, default=4, help="serving slots (streams)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload and args.workload.startswith("cube3d_") and "mixed" in args.workload:
        return run_mixed(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
