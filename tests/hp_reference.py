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


# ------------------------------------------------------------------ double-double reference
# A double-double value is a pair (hi, lo) of float64 arrays whose exact sum carries about 106
# significant bits.  The building blocks are the error-free transformations TwoSum (Knuth,
# TAOCP vol. 2, 4.2.2) and TwoProduct with Veltkamp splitting (Dekker, "A floating-point
# technique for extending the available precision", Numer. Math. 18 (1971)); sums, products,
# quotients and square roots of pairs follow Dekker's algorithms.  numpy evaluates every
# operation below in float64 with no contraction, which these algorithms rely on.

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _fast_two_sum(a, b):  # |a| >= |b|
    s = a + b
    return s, b - (s - a)


def _split(a):
    t = 134217729.0 * a  # 2^27 + 1
    hi = t - (t - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def dd_add(x, y):
    s, e = _two_sum(x[0], y[0])
    t, f = _two_sum(x[1], y[1])
    s, e = _fast_two_sum(s, e + t)
    return _fast_two_sum(s, e + f)


def dd_neg(x):
    return -x[0], -x[1]


def dd_sub(x, y):
    return dd_add(x, dd_neg(y))


def dd_mul(x, y):
    p, e = _two_prod(x[0], y[0])
    return _fast_two_sum(p, e + (x[0] * y[1] + x[1] * y[0]))


def dd_div(x, y):
    q1 = x[0] / y[0]
    r = dd_sub(x, dd_mul((q1, np.zeros_like(q1)), y))
    q2 = r[0] / y[0]
    r = dd_sub(r, dd_mul((q2, np.zeros_like(q2)), y))
    q3 = r[0] / y[0]
    s, e = _fast_two_sum(q1, q2)
    return dd_add((s, e), (q3, np.zeros_like(q3)))


def dd_sqrt(x):
    """Square root of x >= 0: the float64 root refined by one Newton step in double-double."""
    h = np.sqrt(x[0])
    safe = np.where(h > 0, h, 1.0)
    r = dd_sub(x, dd_mul((h, np.zeros_like(h)), (h, np.zeros_like(h))))
    corr = r[0] / (2.0 * safe)
    out = _fast_two_sum(h, np.where(h > 0, corr, 0.0))
    return out


def dd(v):
    v = np.asarray(v, dtype=np.float64)
    return v.copy(), np.zeros_like(v)


def dd_solve(A, B):
    """Solve A X = B in double-double by Gaussian elimination with partial pivoting (largest
    |hi| in the column).  A: (hi, lo) K x K, B: (hi, lo) K x q.  Returns X as (hi, lo)."""
    Ah, Al = A[0].copy(), A[1].copy()
    Bh, Bl = B[0].copy(), B[1].copy()
    K = Ah.shape[0]
    for p in range(K):
        piv = p + int(np.argmax(np.abs(Ah[p:, p])))
        if Ah[piv, p] == 0.0:
            raise ZeroDivisionError("singular system")
        if piv != p:
            for M in (Ah, Al, Bh, Bl):
                M[[p, piv]] = M[[piv, p]]
        if p + 1 == K:
            break
        lh, ll = dd_div((Ah[p + 1:, p], Al[p + 1:, p]),
                        (np.full(K - p - 1, Ah[p, p]), np.full(K - p - 1, Al[p, p])))
        l2 = (lh[:, None], ll[:, None])
        t = dd_mul(l2, (Ah[p, None, p + 1:], Al[p, None, p + 1:]))
        Ah[p + 1:, p + 1:], Al[p + 1:, p + 1:] = dd_sub((Ah[p + 1:, p + 1:], Al[p + 1:, p + 1:]), t)
        t = dd_mul(l2, (Bh[p, None, :], Bl[p, None, :]))
        Bh[p + 1:], Bl[p + 1:] = dd_sub((Bh[p + 1:], Bl[p + 1:]), t)
    Xh, Xl = np.zeros_like(Bh), np.zeros_like(Bl)
    for p in range(K - 1, -1, -1):
        q = Bh.shape[1]
        xp = dd_div((Bh[p], Bl[p]), (np.full(q, Ah[p, p]), np.full(q, Al[p, p])))
        Xh[p], Xl[p] = xp
        if p > 0:
            t = dd_mul((Ah[:p, p, None], Al[:p, p, None]), (xp[0][None, :], xp[1][None, :]))
            Bh[:p], Bl[:p] = dd_sub((Bh[:p], Bl[:p]), t)
    return Xh, Xl


def _dd_pow_int(x, e):
    out = dd(np.ones_like(x[0]))
    for _ in range(e):
        out = dd_mul(out, x)
    return out


def dd_weights(X, idx, ell, m, Y):
    """Laplacian weights [n][q] of stencil X[idx] at the points Y [q][d] from the definitions
    of §4.1 in double-double: PHS r^m plus all monomials of total degree <= ell, right-hand
    sides m (m + d - 2) r^(m-2) and the monomials' Laplacians.  The coordinates are shifted
    to x_c = X[idx[0]] (exact in double-double) and divided by a power of two h near the
    stencil width (exact), a change of variables that leaves the weights invariant up to the
    factor 1/h^2.  Independent of the oracle and of the CUDA library."""
    idx = np.asarray(idx)
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    d = X.shape[1]
    n, q = idx.size, Y.shape[0]
    xc = X[idx[0]]
    P = [_two_sum(X[idx, a], -np.full(n, xc[a])) for a in range(d)]   # exact x - x_c
    E = [_two_sum(Y[:, a], -np.full(q, xc[a])) for a in range(d)]
    ext = max(np.abs(X[idx] - xc).max(), 1e-300)
    h = 2.0 ** np.round(np.log2(ext))
    P = [(u / h, v / h) for u, v in P]
    E = [(u / h, v / h) for u, v in E]
    exps = [a for g in range(ell + 1) for a in itertools.product(range(g + 1), repeat=d)
            if sum(a) == g]
    M = len(exps)
    K = n + M

    def r2_between(U, V):  # pairwise squared distances, U: len-a arrays, V: len-b arrays
        s = dd(np.zeros((U[0][0].size, V[0][0].size)))
        for a in range(d):
            dlt = dd_sub((U[a][0][:, None], U[a][1][:, None]), (V[a][0][None, :], V[a][1][None, :]))
            s = dd_add(s, dd_mul(dlt, dlt))
        return s

    def odd_pow(r2, k):  # r^k for odd k from r^2
        r = dd_sqrt(r2)
        return dd_mul(r, _dd_pow_int(r2, (k - 1) // 2))

    def mono(U, al):
        v = dd(np.ones_like(U[0][0]))
        for a in range(d):
            v = dd_mul(v, _dd_pow_int(U[a], al[a]))
        return v

    Ah, Al = np.zeros((K, K)), np.zeros((K, K))
    phi = odd_pow(r2_between(P, P), m)
    Ah[:n, :n], Al[:n, :n] = phi
    for l, al in enumerate(exps):
        v = mono(P, al)
        Ah[:n, n + l], Al[:n, n + l] = v
        Ah[n + l, :n], Al[n + l, :n] = v
    Bh, Bl = np.zeros((K, q)), np.zeros((K, q))
    lphi = odd_pow(r2_between(P, E), m - 2)
    c = float(m * (m + d - 2))
    Bh[:n], Bl[:n] = dd_mul((np.full((n, q), c), np.zeros((n, q))), lphi)
    for l, al in enumerate(exps):
        s = dd(np.zeros(q))
        for a in range(d):
            if al[a] < 2:
                continue
            be = list(al)
            be[a] -= 2
            s = dd_add(s, dd_mul(dd(np.full(q, float(al[a] * (al[a] - 1)))), mono(E, be)))
        Bh[n + l], Bl[n + l] = s
    Wh, Wl = dd_solve((Ah, Al), (Bh, Bl))
    return (Wh[:n] + Wl[:n]) / (h * h)


# ------------------------------------------------------------------ accuracy criterion
def accuracy_failures(e_cand, e_ora, cls, e_cand_w=None):
    """Compare the forward errors of a candidate FP64 solver (e_cand) with the oracle's (e_ora)
    on the same rows (measured against dd_weights), grouped by stencil class `cls`.  The bar a
    correct FP64 solver meets on ill-conditioned stencils, where two such solvers differ by
    about their own errors and a per-row ratio is largely rounding luck (LAPACK against the
    oracle reaches 10x on single rows):
      per row    e_cand <= max(10 e_ora, the oracle's median over the row's class) + 1e-10,
                 and e_cand <= 1e-9 wherever e_ora <= 1e-10;
      per class  median(e_cand) <= 2 median(e_ora) + 1e-12 and max(e_cand) <= 2 max(e_ora) + 1e-10.
    For Lebesgue values (the l1 norm of a row's weights, whose relative error can reach n
    times that of the weights) pass the candidate's weight errors as e_cand_w: a row then also
    passes when its Lebesgue error is at most 4 times its own weight error (the weights being
    held to the bar above), and the 1e-9 rule is not applied.
    Returns a list of failure descriptions (empty = pass)."""
    e_cand, e_ora, cls = np.asarray(e_cand), np.asarray(e_ora), np.asarray(cls)
    out = []
    med = np.array([np.median(e_ora[cls == c]) for c in cls])
    ok = e_cand <= np.maximum(10.0 * e_ora, med) + 1e-10
    if e_cand_w is not None:
        ok |= e_cand <= 4.0 * np.asarray(e_cand_w)
    for k in np.nonzero(~ok)[0]:
        out.append(f"row {k} (class {cls[k]}): {e_cand[k]:.3e} > max(10 x {e_ora[k]:.3e}, "
                   f"{med[k]:.3e}) + 1e-10")
    if e_cand_w is None:
        for k in np.nonzero((e_ora <= 1e-10) & (e_cand > 1e-9))[0]:
            out.append(f"row {k} (class {cls[k]}): {e_cand[k]:.3e} > 1e-9 where the oracle is "
                       f"{e_ora[k]:.3e}")
    for c in np.unique(cls):
        a, b = e_cand[cls == c], e_ora[cls == c]
        if np.median(a) > 2.0 * np.median(b) + 1e-12:
            out.append(f"class {c}: median {np.median(a):.3e} > 2 x {np.median(b):.3e}")
        if a.max() > 2.0 * b.max() + 1e-10:
            out.append(f"class {c}: max {a.max():.3e} > 2 x {b.max():.3e} + 1e-10")
    return out
