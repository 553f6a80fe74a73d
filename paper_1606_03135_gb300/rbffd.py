"""Python binding of librbffd.so (include/rbffd.h): argument marshalling only.

Every step of the differentiation-matrix construction runs in the library's CUDA kernels.
The functions below carry the C names; ``Plan`` wraps them for torch users (torch provides
device memory and the current CUDA stream, nothing else).  Importing this module never
falls back to anything: if the shared library cannot be built or loaded, it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, EDUPLICATE, ENOMEM, ESINGULAR, ETIMEOUT, ECUDA, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
STAB_SEQ, STAB_OFF, STAB_FALLBACK = 0, 1, 2
FACTOR_LDLT, FACTOR_LU = 0, 1
LREF_CENTER, LREF_CENTROID = 0, 1  # reference point of the Lebesgue test (rbffd_opts.lebesgue_ref)
REFINE_AUTO, REFINE_ALL, REFINE_NONE = 0, 1, 2  # iterative refinement (rbffd_opts.refine)
REFINE_MIN_K = 100  # RBFFD_REFINE_MIN_K: systems at least this large are refined by default


class rbffd_opts(C.Structure):
    _fields_ = [("stab_mode", C.c_int), ("nodes_on_host", C.c_int), ("timeout_ms", C.c_int),
                ("sync", C.c_int), ("fault_inject", C.c_int), ("factor", C.c_int),
                ("max_ctas", C.c_int), ("team", C.c_int), ("rhs_chunk", C.c_int),
                ("lebesgue_ref", C.c_int), ("refine", C.c_int), ("elastic", C.c_int)]


class rbffd_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class rbffd_stats_t(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_centers", C.c_int64), ("n_fallback", C.c_int64),
                ("n_rejected", C.c_int64), ("sum_cols", C.c_int64), ("max_ball", C.c_int64),
                ("n_singular", C.c_int64), ("status", C.c_int32), ("n", C.c_int32),
                ("M", C.c_int32), ("K", C.c_int32), ("d", C.c_int32), ("alg_flops", C.c_double),
                ("n_launches", C.c_int64), ("ms_stencils", C.c_float),
                ("ms_traversal", C.c_float), ("ms_fallback", C.c_float),
                ("ms_finalize", C.c_float), ("nnz", C.c_int64), ("plan_bytes", C.c_int64),
                ("assemble_bytes", C.c_int64), ("n_boundary", C.c_int64),
                ("n_speculated", C.c_int64), ("n_spec_used", C.c_int64),
                ("rhs_chunk", C.c_int64), ("sum_k3", C.c_double), ("sum_k2_cols", C.c_double),
                ("flops_refine", C.c_double), ("refine_min_K", C.c_int32), ("pad0", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_SIGS = {
    "rbffd_plan": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int,
                             C.c_double, C.POINTER(rbffd_opts), C.c_void_p,
                             C.POINTER(C.c_void_p)]),
    "rbffd_plan_mixed": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_double, C.POINTER(rbffd_opts), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "rbffd_plan_delta": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(rbffd_opts), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "rbffd_assemble": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(rbffd_csr)]),
    "rbffd_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_set_boundary": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_timestep_matrix": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "rbffd_stats": (C.c_int, [C.c_void_p, C.POINTER(rbffd_stats_t)]),
    "rbffd_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_export_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "rbffd_export_stencils": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_export_lambda": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_stencils_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rbffd_destroy": (None, [C.c_void_p]),
    "rbffd_strerror": (C.c_char_p, [C.c_int]),
}


def load() -> C.CDLL:
    """Build (if stale) and load librbffd.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class RbffdError(RuntimeError):
    def __init__(self, code, what):
        msg = load().rbffd_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def _check(rc, what):
    if rc != OK:
        raise RbffdError(rc, what)


def _p(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


# ------------------------------------------------------------------ C names
def rbffd_plan(nodes_ptr, N, d, n, ell, m, delta, opts=None, stream=None):
    out = C.c_void_p()
    rc = load().rbffd_plan(nodes_ptr, N, d, n, ell, m, float(delta),
                           C.byref(opts) if opts is not None else None, stream, C.byref(out))
    return rc, out


def rbffd_plan_mixed(nodes_ptr, N, d, n_node, ell_node, m_node, delta, opts=None, stream=None):
    out = C.c_void_p()
    rc = load().rbffd_plan_mixed(nodes_ptr, N, d, _p(n_node), _p(ell_node), _p(m_node),
                                 float(delta), C.byref(opts) if opts is not None else None,
                                 stream, C.byref(out))
    return rc, out


def rbffd_plan_delta(base, delta, opts=None, stream=None):
    out = C.c_void_p()
    rc = load().rbffd_plan_delta(base, float(delta), C.byref(opts) if opts is not None else None,
                                 stream, C.byref(out))
    return rc, out


def rbffd_assemble(plan, stream=None):
    csr = rbffd_csr()
    rc = load().rbffd_assemble(plan, stream, C.byref(csr))
    return rc, csr


def rbffd_apply(plan, u_ptr, y_ptr, stream=None):
    return load().rbffd_apply(plan, u_ptr, y_ptr, stream)


def rbffd_stats(plan):
    st = rbffd_stats_t()
    rc = load().rbffd_stats(plan, C.byref(st))
    return rc, st


def rbffd_export(plan, row_ptr, col, val, owner):
    return load().rbffd_export(plan, _p(row_ptr), _p(col), _p(val), _p(owner))


def rbffd_export_async(plan, row_ptr, col, val, owner, stream):
    return load().rbffd_export_async(plan, _p(row_ptr), _p(col), _p(val), _p(owner), stream)


def rbffd_export_stencils(plan, nbr, rho2, ball_len):
    return load().rbffd_export_stencils(plan, _p(nbr), _p(rho2), _p(ball_len))


def rbffd_export_lambda(plan, lam_row, is_center):
    return load().rbffd_export_lambda(plan, _p(lam_row), _p(is_center))


def rbffd_stencils_noalloc(nodes, N, d, n, delta, nbr, rho2, ball_len, stream=None):
    """Allocation-free stencil step on caller-owned device buffers (torch tensors)."""
    return load().rbffd_stencils_noalloc(_p(nodes), N, d, n, float(delta), _p(nbr), _p(rho2),
                                         _p(ball_len), stream)


def rbffd_destroy(plan):
    if plan:
        load().rbffd_destroy(plan)


def rbffd_strerror(code):
    return load().rbffd_strerror(code).decode()


# ------------------------------------------------------------------ torch-facing wrapper
def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Plan:
    """Stencils of one node set (``rbffd_plan``); ``assemble()`` forms L on the device.

    nodes: a torch float64 tensor [N, d] on the GPU (or a numpy array on the host, copied by
    the library inside ``rbffd_plan``)."""

    def __init__(self, nodes, n, ell, m, delta, mode=STAB_SEQ, timeout_ms=5000, sync=True,
                 stream=None, fault_inject=0, factor=FACTOR_LDLT, max_ctas=0, team=0,
                 rhs_chunk=0, lebesgue_ref=0, refine=REFINE_AUTO, elastic=0):
        self._plan = None
        self._stream = stream
        if isinstance(nodes, np.ndarray):
            self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
            on_host = 1
        else:
            import torch
            if nodes.dtype != torch.float64 or not nodes.is_cuda:
                raise TypeError("nodes must be a float64 CUDA tensor or a numpy array")
            self._nodes = nodes.contiguous()
            on_host = 0
        self.N, self.d = self._nodes.shape
        self.ell, self.m, self.delta, self.mode = ell, m, delta, mode
        self.sync = bool(sync)
        opts = rbffd_opts(mode, on_host, timeout_ms, 1 if sync else 0, fault_inject, factor,
                          max_ctas, team, rhs_chunk, lebesgue_ref, refine, elastic)
        if np.ndim(n) == 0:  # one stencil size, degree and exponent for every node
            self.n = int(n)
            rc, plan = rbffd_plan(_p(self._nodes), self.N, self.d, n, ell, m, delta, opts,
                                  _stream_handle(stream))
            _check(rc, "rbffd_plan")
        else:                # per-node arrays
            self._node_params = [np.ascontiguousarray(v, dtype=np.int32) for v in (n, ell, m)]
            self.n = int(self._node_params[0].max())
            rc, plan = rbffd_plan_mixed(_p(self._nodes), self.N, self.d, *self._node_params,
                                        delta, opts, _stream_handle(stream))
            _check(rc, "rbffd_plan_mixed")
        self._plan = plan

    def with_delta(self, delta, mode=STAB_SEQ, timeout_ms=5000, sync=True, stream=None,
                   fault_inject=0, factor=FACTOR_LDLT, max_ctas=0, team=0, rhs_chunk=0,
                   lebesgue_ref=0, refine=REFINE_AUTO, elastic=0):
        """A plan for this plan's nodes and stencil parameters at another delta
        (``rbffd_plan_delta``): the kNN stencils are copied from this plan on the device and
        only the retention balls are recomputed; the result equals a new ``Plan`` with these
        arguments.  This plan may be closed once the call returns."""
        q = Plan.__new__(Plan)
        q._plan = None
        q._stream = stream
        q._nodes = self._nodes
        q.N, q.d, q.n, q.ell, q.m = self.N, self.d, self.n, self.ell, self.m
        if hasattr(self, "_node_params"):
            q._node_params = self._node_params
        q.delta, q.mode, q.sync = delta, mode, bool(sync)
        opts = rbffd_opts(mode, 0, timeout_ms, 1 if sync else 0, fault_inject, factor, max_ctas,
                          team, rhs_chunk, lebesgue_ref, refine, elastic)
        rc, plan = rbffd_plan_delta(self._plan, delta, opts, _stream_handle(stream))
        _check(rc, "rbffd_plan_delta")
        q._plan = plan
        return q

    def assemble(self, stream=None):
        """Form L on the device (``rbffd_assemble``).  `stream` (a torch CUDA stream) moves the
        plan to another stream from here on, e.g. assemble on the compute stream while the next
        plan is built on a side stream."""
        if stream is not None:
            self._stream = stream
        rc, csr = rbffd_assemble(self._plan, _stream_handle(self._stream))
        _check(rc, "rbffd_assemble")
        return csr

    def capture_assemble(self, stream=None):
        """Record one rbffd_assemble into a CUDA graph (torch.cuda.CUDAGraph); each replay()
        forms L again on the device with no host work.  The plan must be asynchronous
        (sync=False) and assembled once before capture, so the graph allocates nothing."""
        import torch
        if self.sync:
            raise ValueError("capture needs a plan created with sync=False")
        g = torch.cuda.CUDAGraph()
        s = stream if stream is not None else torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            rc, _ = rbffd_assemble(self._plan, C.c_void_p(s.cuda_stream))
        _check(rc, "rbffd_assemble (capture)")
        self._stream = s
        return g

    def set_boundary(self, bc, normals=None):
        """Boundary nodes (§5): bc [N] uint8 (0 interior, 1 Dirichlet, 2 Neumann), normals
        [N][d] unit outward normals of the Neumann nodes; None removes the boundary."""
        bcv = None if bc is None else np.ascontiguousarray(bc, dtype=np.uint8)
        nrv = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
        if bcv is not None and bcv.shape != (self.N,):
            raise ValueError("bc must have one entry per node")
        if nrv is not None and nrv.shape != (self.N, self.d):
            raise ValueError("normals must be [N][d]")
        _check(load().rbffd_set_boundary(self._plan, _p(bcv), _p(nrv)), "rbffd_set_boundary")

    def timestep_matrix(self, c, out=None):
        """Values of the time-stepping matrix of §5 on L's pattern (interior rows e_i - c L_i,
        boundary rows unchanged) into a device tensor of nnz doubles, returned."""
        import torch
        if out is None:
            out = torch.empty(self.stats()["nnz"], dtype=torch.float64, device="cuda")
        _check(load().rbffd_timestep_matrix(self._plan, float(c), C.c_void_p(out.data_ptr()),
                                            _stream_handle(self._stream)),
               "rbffd_timestep_matrix")
        return out

    def apply(self, u, y):
        _check(rbffd_apply(self._plan, _p(u), _p(y), _stream_handle(self._stream)),
               "rbffd_apply")

    def stats(self) -> dict:
        rc, st = rbffd_stats(self._plan)
        _check(rc, "rbffd_stats")
        return st.as_dict()

    def export(self, out=None):
        """Host copies (row_ptr, col, val, owner) of the CSR and the stencil owning each row.
        `out` may supply the four arrays (e.g. in pinned memory, reused across calls): int64
        [N+1], int32 [>= nnz], float64 [>= nnz], int32 [N]; the views of the filled parts are
        returned."""
        N = self.N
        nnz = self.stats()["nnz"]
        if out is None:
            out = (np.zeros(N + 1, np.int64), np.zeros(nnz, np.int32),
                   np.zeros(nnz, np.float64), np.zeros(N, np.int32))
        row_ptr, col, val, owner = out
        for a, dt, size in ((row_ptr, np.int64, N + 1), (col, np.int32, nnz),
                            (val, np.float64, nnz), (owner, np.int32, N)):
            if a.dtype != dt or not a.flags.c_contiguous or a.size < size:
                raise ValueError("export buffers: wrong dtype, layout or size")
        _check(rbffd_export(self._plan, row_ptr, col, val, owner), "rbffd_export")
        return row_ptr[:N + 1], col[:nnz], val[:nnz], owner[:N]

    def export_async(self, out, stream):
        """export() into caller buffers `out` (pinned host arrays, as for export) enqueued on
        the torch CUDA stream `stream` without waiting; the arrays are filled once the stream
        has reached the copies.  Returns the views of the parts that will be filled."""
        N = self.N
        # per-node stencils: nnz from the counters (rbffd_stats waits for the assembly)
        nnz = self.stats()["nnz"] if hasattr(self, "_node_params") else N * self.n
        row_ptr, col, val, owner = out
        for a, dt, size in ((row_ptr, np.int64, N + 1), (col, np.int32, nnz),
                            (val, np.float64, nnz), (owner, np.int32, N)):
            if a.dtype != dt or not a.flags.c_contiguous or a.size < size:
                raise ValueError("export buffers: wrong dtype, layout or size")
        _check(rbffd_export_async(self._plan, row_ptr, col, val, owner,
                                  _stream_handle(stream)), "rbffd_export_async")
        return row_ptr[:N + 1], col[:nnz], val[:nnz], owner[:N]

    def export_stencils(self):
        N, n = self.N, self.n
        nbr = np.zeros((N, n), np.int32)
        rho2 = np.zeros(N, np.float64)
        bl = np.zeros(N, np.int32)
        _check(rbffd_export_stencils(self._plan, nbr, rho2, bl), "rbffd_export_stencils")
        return nbr, rho2, bl

    def export_lambda(self):
        lam = np.zeros(self.N, np.float64)
        isc = np.zeros(self.N, np.uint8)
        _check(rbffd_export_lambda(self._plan, lam, isc), "rbffd_export_lambda")
        return lam, isc

    def close(self):
        if self._plan:
            rbffd_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def capture_assemble_batch(plans, streams=None):
    """Record one rbffd_assemble of every plan in `plans` into a single CUDA graph
    (torch.cuda.CUDAGraph): each plan on its own stream, forked from the capture stream and
    joined back, so a replay runs the plans' kernels concurrently, whatever their dimension,
    degree or stencil sizes.  Every plan must be asynchronous (sync=False) and assembled once
    before capture (so the graph allocates nothing).  Each plan's later calls (stats, export)
    use its stream from the capture."""
    import torch
    for p in plans:
        if p.sync:
            raise ValueError("capture needs plans created with sync=False")
    g = torch.cuda.CUDAGraph()
    s0 = torch.cuda.Stream()
    ss = list(streams) if streams is not None else [torch.cuda.Stream() for _ in plans]
    s0.wait_stream(torch.cuda.current_stream())
    rcs = []
    with torch.cuda.graph(g, stream=s0):
        for p, s in zip(plans, ss):
            s.wait_stream(s0)
            rcs.append(rbffd_assemble(p._plan, C.c_void_p(s.cuda_stream))[0])
        for s in ss:
            s0.wait_stream(s)
    for rc in rcs:
        _check(rc, "rbffd_assemble (batch capture)")
    for p, s in zip(plans, ss):
        p._stream = s
    return g


# ------------------------------------------------------------------ schedule autotuner
def autotune(nodes, n, ell, m, delta, mode=STAB_SEQ, candidates=None, repeats=2):
    """Pick the traversal schedule for a workload -- warp-per-stencil (32 threads), 64-, 96-, 128-
    or 512-thread tiles per stencil, the persistent-grid cap, and, with 96- or 128-thread tiles,
    fewer right-hand sides per factorization (about 0.3, 0.45 and 0.6 of the largest ball:
    more stencils fit an SM, later columns take extra passes) -- by timing assemblies of each
    candidate on the device (CUDA events, best of `repeats`, after a warm-up assembly).
    Returns (best kwargs for Plan, {candidate: ms}).  Results do not depend on the schedule
    (the same stencils are solved the same way), only the time does."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if candidates is None:
        candidates = [dict(team=t) for t in (32, 64, 96, 128, 256, 512)]
        candidates += [dict(team=0, max_ctas=c) for c in (0, 4 * sms)]
        if np.ndim(n) == 0:
            with Plan(nodes, n, ell, m, delta, mode=mode) as p:
                max_ball = p.stats()["max_ball"]
            chunks = sorted({max(4, round(max_ball * f)) for f in (0.3, 0.45, 0.6)})
            candidates += [dict(team=t, rhs_chunk=c) for t in (96, 128) for c in chunks
                           if c < max_ball]
    timings = {}
    for cand in candidates:
        try:
            with Plan(nodes, n, ell, m, delta, mode=mode, **cand) as p:
                p.assemble()
                best = float("inf")
                for _ in range(repeats):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    p.assemble()
                    e1.record()
                    e1.synchronize()
                    best = min(best, e0.elapsed_time(e1))
        except RbffdError:
            continue
        timings[tuple(sorted(cand.items()))] = best
    key = min(timings, key=timings.get)
    return dict(key), timings
