"""The paper's a-priori cost model of the overlapped method (§4.3) and its delta estimate (§4.4).

Reporting helpers only (host arithmetic on the statistics of an assembly); nothing here is on
the path that forms L.

* p = max((1 - delta)^d n, 1): the nodes a retention ball holds on quasi-uniform nodes.
* eta = C gamma p (n + M + 1) / (n + M + gamma p): the predicted speedup over standard
  (delta = 1) augmented RBF-FD, with q = gamma p rows kept per stencil after stabilization and
  C a dimension-dependent constant (0.4 in 2D and 0.38 in 3D in the paper's experiments, §7).
* The same ratio from measured counts: N (n + M + 1) / (N_delta (n + M + q)).
* delta from a wanted retained fraction t: (1 - delta)^d = t, delta = 1 - t^(1/d).  (The
  printed equation carries a stray factor n; with p = t n the n cancels.)
"""
from __future__ import annotations

import math

C_PAPER = {2: 0.4, 3: 0.38}


def p_hat(delta: float, n: int, d: int) -> float:
    """Expected retention-ball size max((1 - delta)^d n, 1)."""
    return max((1.0 - delta) ** d * n, 1.0)


def eta_predicted(delta: float, n: int, M: int, d: int, gamma: float = 1.0,
                  C: float | None = None) -> float:
    """A-priori speedup over delta = 1: C gamma p (n + M + 1) / (n + M + gamma p)."""
    C = C_PAPER[d] if C is None else C
    p = p_hat(delta, n, d)
    return C * gamma * p * (n + M + 1) / (n + M + gamma * p)


def eta_from_counts(N: int, N_delta: int, n: int, M: int, q: float) -> float:
    """The cost ratio C3 / C4 = N (n + M + 1) / (N_delta (n + M + q)) from measured counts
    (N_delta centers, q right-hand sides per center)."""
    return N * (n + M + 1) / (N_delta * (n + M + q))


def delta_from_retention(t: float, d: int) -> float:
    """The overlap parameter that keeps the fraction t of a stencil's nodes: 1 - t^(1/d)."""
    if not (0.0 < t <= 1.0):
        raise ValueError("t must lie in (0, 1]")
    return 1.0 - t ** (1.0 / d)


def sweep_report(rows: dict, N: int, n: int, M: int, d: int) -> dict:
    """Per delta of a sweep: the measured speedup of the traversal over delta = 1, the paper's
    prediction with gamma = 1 and with the measured gamma, and the counted cost ratio.
    `rows` maps delta -> {"n_centers", "sum_cols", "ms_traversal"}."""
    out = {}
    base = rows.get(1.0)
    for delta, r in sorted(rows.items(), reverse=True):
        q = r["sum_cols"] / r["n_centers"]
        gamma = min(1.0, (N / r["n_centers"]) / p_hat(delta, n, d))
        out[str(delta)] = {
            "N_delta": int(r["n_centers"]), "q_solved": q, "rows_per_center": N / r["n_centers"],
            "p_hat": p_hat(delta, n, d), "gamma": gamma,
            "eta_model_gamma1": eta_predicted(delta, n, M, d),
            "eta_model_gamma": eta_predicted(delta, n, M, d, gamma),
            "eta_counts": eta_from_counts(N, r["n_centers"], n, M, q),
            "speedup_measured": (base["ms_traversal"] / r["ms_traversal"]) if base else None,
        }
    return out
