"""High-precision reference weights for tests (mpmath + sympy), independent of the oracle.

The local system of §4.1 is rebuilt from its definitions in the ORIGINAL (unscaled,
uncentered) coordinates with raw monomials, its right-hand sides differentiated by sympy, and
solved by mpmath LU at `dps` significant digits.
"""
import itertools

import numpy as np


def mp_weights(X, idx, ell, m, Y, dps=40, normal=None):
    """Independent high-precision weights from the definitions of §4.1, in the ORIGINAL
    coordinates with raw monomials x^a y^b (z^c); Laplacians by sympy differentiation.  With
    `normal` (a unit vector) the operator is the derivative along it instead (§5, Neumann)."""
    import mpmath as mp
    import sympy as sp
    mp.mp.dps = dps
    d = X.shape[1]
    syms = sp.symbols("x0:%d" % d)
    cs = sp.symbols("c0:%d" % d)
    r = sp.sqrt(sum((s - c) ** 2 for s, c in zip(syms, cs)))
    if normal is None:
        lap = lambda f: sum(sp.diff(f, s, 2) for s in syms)
    else:
        nv = [sp.Float(float(v), 60) for v in normal]
        lap = lambda f: sum(c * sp.diff(f, s) for c, s in zip(nv, syms))
    phi = r ** m
    lphi = sp.simplify(lap(phi))
    f_lphi = sp.lambdify(syms + cs, lphi, "mpmath")
    exps = [a for g in range(ell + 1) for a in itertools.product(range(g + 1), repeat=d)
            if sum(a) == g]
    monos = [sp.Mul(*[s ** a for s, a in zip(syms, al)]) for al in exps]
    f_mono = [sp.lambdify(syms, p, "mpmath") for p in monos]
    f_lmono = [sp.lambdify(syms, lap(p), "mpmath") for p in monos]
    n, M = len(idx), len(monos)
    K = n + M
    P = [[mp.mpf(float(v)) for v in X[i]] for i in idx]
    A = mp.zeros(K, K)
    for a in range(n):
        for b in range(n):
            A[a, b] = mp.sqrt(sum((P[a][t] - P[b][t]) ** 2 for t in range(d))) ** m
        for l in range(M):
            A[a, n + l] = f_mono[l](*P[a])
            A[n + l, a] = A[a, n + l]
    out = []
    for y in Y:
        yy = [mp.mpf(float(v)) for v in y]
        b = mp.zeros(K, 1)
        for a in range(n):
            same = all(yy[t] == P[a][t] for t in range(d))
            b[a] = 0 if same else f_lphi(*(yy + P[a]))
        for l in range(M):
            b[n + l] = f_lmono[l](*yy)
        x = mp.lu_solve(A, b)
        out.append([float(x[j]) for j in range(n)])
    return np.array(out).T




def lapack_weights(X, idx, ell, m, y):
    """Laplacian weights of stencil X[idx] (center idx[0]) at point y from an independent
    FP64 solve: the local system of §4.1 built with numpy in scaled local coordinates and
    solved by LAPACK (numpy.linalg.solve).  Used to measure how far two correct FP64 solvers
    drift apart on an ill-conditioned stencil."""
    d = X.shape[1]
    c = X[idx[0]]
    rho = np.sqrt(((X[idx] - c) ** 2).sum(1).max())
    xi = (X[idx] - c) / rho
    eta = (y - c) / rho
    ex = [a for g in range(ell + 1) for a in itertools.product(range(g + 1), repeat=d)
          if sum(a) == g]
    n, M = len(idx), len(ex)
    K = n + M
    R = np.sqrt(((xi[:, None] - xi[None]) ** 2).sum(-1))
    A = np.zeros((K, K))
    A[:n, :n] = R ** m
    P = np.stack([np.prod(xi ** np.array(e), axis=1) for e in ex], 1)
    A[:n, n:] = P
    A[n:, :n] = P.T
    b = np.zeros(K)
    rr = np.sqrt(((xi - eta) ** 2).sum(-1))
    b[:n] = m * (m + d - 2) * rr ** (m - 2)
    for l, e in enumerate(ex):
        v = 0.0
        for a in range(d):
            if e[a] >= 2:
                ee = list(e)
                ee[a] -= 2
                v += e[a] * (e[a] - 1) * np.prod(eta ** np.array(ee))
        b[n + l] = v
    return np.linalg.solve(A, b)[:n] / rho ** 2
