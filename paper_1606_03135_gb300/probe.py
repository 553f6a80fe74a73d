"""Binding of libfp64probe.so (include/fp64_probe.h): the FP64 pipe throughput probe.

It measures the GPU's FP64 FMA rate (independent DFMA chains) and its FP64 tensor-core rate
(mma.sync m8n8k4 f64 tiles), alone and mixed, with CUDA events: a measured denominator for
the FP64 roofline of the local-solve kernels, and the evidence for keeping those kernels on
the FMA pipe.  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import threading

from . import build as _build

DFMA, DMMA, MIXED = 0, 1, 2

_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _build.build()
            L = C.CDLL(_build.PROBE_LIB)
            L.fp64_probe_run.restype = C.c_int
            L.fp64_probe_run.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(C.c_float)]
            _lib = L
    return _lib


def fp64_probe_run(kind: int, iters: int, stream=None):
    """(rc, TFLOP/s, ms) of one probe launch on the CUDA stream handle `stream` (None: the
    legacy default stream)."""
    tf, ms = C.c_double(0.0), C.c_float(0.0)
    rc = load().fp64_probe_run(kind, iters, stream, C.byref(tf), C.byref(ms))
    return rc, tf.value, ms.value


def measure(iters: int = 20000, repeats: int = 3) -> dict:
    """Best of `repeats` launches of each kind after one warm-up launch: TFLOP/s and ms."""
    out = {}
    for name, kind in (("dfma", DFMA), ("dmma", DMMA), ("mixed", MIXED)):
        rc, _, _ = fp64_probe_run(kind, max(1, iters // 10))
        if rc != 0:
            raise RuntimeError(f"fp64_probe_run({name}) failed: {rc}")
        best = (0.0, 0.0)
        for _ in range(repeats):
            rc, tf, ms = fp64_probe_run(kind, iters)
            if rc != 0:
                raise RuntimeError(f"fp64_probe_run({name}) failed: {rc}")
            best = max(best, (tf, ms))
        out[name] = {"tflops": best[0], "ms": best[1]}
    return out


if __name__ == "__main__":  # python -m paper_1606_03135_gb300.probe [iters]
    import json
    import sys
    print(json.dumps(measure(iters=int(sys.argv[1]) if len(sys.argv) > 1 else 20000, repeats=5)))
