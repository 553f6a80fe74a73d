"""Seeded synthetic node sets for the overlapped RBF-FD differentiation-matrix workloads.

This module only *draws inputs*: it holds none of the method's arithmetic (no kNN, no
local systems, no stabilization).  Both the CUDA path and the CPU oracle are fed from it.

Every random number comes from a counter-based splitmix64 stream written out here in
uint64 numpy arithmetic, so a given (recipe, seed) produces bit-identical nodes on any
machine (x86-64 or aarch64) and any numpy version.  The quasi-random parts use the Halton
sequence (radical inverse in bases 2, 3, 5), written out here too.

The paper measures on Distmesh nodes in the unit disk and Gmsh nodes in the unit ball
(§7.1, §7.2); those node files are not available, so these recipes stand in for them:

* ``disk2d``     -- Halton (2,3) points in the unit disk, jittered by 0.1 h.
* ``square2d``   -- 200x200 cell-centred grid in the unit square, jittered by 0.25 h,
                    emitted in a seeded random order (``order="raster"`` keeps row order).
* ``ball3d``     -- Halton (2,3,5) points in the unit ball, jittered by 0.1 h.
* ``cube3d_clustered`` -- 60 % Halton + 40 % Gaussian clusters (sigma 0.04) in the unit
                    cube, about 10x density contrast.

The traversal order of the nodes changes the overlapped method's result (§4.1, the
"never recomputed" rule), so the emitted order is part of each recipe.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based splitmix64: uint64 outputs for counters offset+1 .. offset+count."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def halton(index: np.ndarray, base: int) -> np.ndarray:
    """Radical inverse of the integer ``index`` (>= 1) in ``base``."""
    i = np.asarray(index, dtype=np.int64).copy()
    out = np.zeros(i.shape, dtype=np.float64)
    f = 1.0 / base
    while np.any(i > 0):
        out += f * (i % base)
        i //= base
        f /= base
    return out


def permutation(seed: int, count: int) -> np.ndarray:
    """A seeded random permutation of range(count) (argsort of splitmix64 keys)."""
    keys = splitmix64(seed, count, offset=1 << 40)
    return np.argsort(keys, kind="stable").astype(np.int64)


def _jitter_in(points, h, amp, seed, inside, max_tries=64):
    """Add U(-amp*h, amp*h) per coordinate; re-draw the jitter of points that leave the domain."""
    n, d = points.shape
    out = points.copy()
    todo = np.arange(n)
    offset = 0
    for _ in range(max_tries):
        u = uniform(seed, todo.size * d, offset).reshape(todo.size, d)
        offset += todo.size * d
        cand = points[todo] + (2.0 * u - 1.0) * (amp * h)
        ok = inside(cand)
        out[todo[ok]] = cand[ok]
        todo = todo[~ok]
        if todo.size == 0:
            return out
    out[todo] = points[todo]  # keep the unjittered point (always inside by construction)
    return out


def _halton_in(N, dims, inside):
    """First N Halton points (bases 2,3[,5], indices from 1) mapped to [-1,1]^d and kept if inside."""
    bases = (2, 3, 5)[:dims]
    pts = []
    got = 0
    start = 1
    while got < N:
        chunk = max(2 * (N - got), 1024)
        idx = np.arange(start, start + chunk)
        P = np.stack([2.0 * halton(idx, b) - 1.0 for b in bases], axis=1)
        P = P[inside(P)]
        pts.append(P)
        got += P.shape[0]
        start += chunk
    return np.concatenate(pts, axis=0)[:N]


def disk2d(N: int = 2000, seed: int = 1) -> np.ndarray:
    """Quasi-uniform nodes in the closed unit disk (stand-in for the paper's Distmesh disk)."""
    inside = lambda P: (P[:, 0] * P[:, 0] + P[:, 1] * P[:, 1]) <= 1.0
    P = _halton_in(N, 2, inside)
    h = math.sqrt(math.pi / N)
    return np.ascontiguousarray(_jitter_in(P, h, 0.1, seed, inside))


def square2d(N: int = 40000, seed: int = 2, order: str = "random") -> np.ndarray:
    """Jittered cell-centred grid in the unit square; N must be a perfect square."""
    side = int(round(math.sqrt(N)))
    if side * side != N:
        raise ValueError("square2d needs N = side^2")
    h = 1.0 / side
    g = (np.arange(side, dtype=np.float64) + 0.5) * h
    gy, gx = np.meshgrid(g, g, indexing="ij")
    P = np.stack([gx.ravel(), gy.ravel()], axis=1)
    u = uniform(seed, N * 2).reshape(N, 2)
    P = P + (2.0 * u - 1.0) * (0.25 * h)
    if order == "random":
        P = P[permutation(seed, N)]
    elif order != "raster":
        raise ValueError("order must be 'random' or 'raster'")
    return np.ascontiguousarray(P)


def ball3d(N: int = 100000, seed: int = 3) -> np.ndarray:
    """Quasi-uniform nodes in the closed unit ball (stand-in for the paper's Gmsh ball)."""
    inside = lambda P: (P[:, 0] * P[:, 0] + P[:, 1] * P[:, 1] + P[:, 2] * P[:, 2]) <= 1.0
    P = _halton_in(N, 3, inside)
    h = (4.0 * math.pi / 3.0 / N) ** (1.0 / 3.0)
    return np.ascontiguousarray(_jitter_in(P, h, 0.1, seed, inside))


def cube3d_clustered(N: int = 500000, seed: int = 4, n_clusters: int = 8,
                     sigma: float = 0.04, frac_clustered: float = 0.4) -> np.ndarray:
    """Unit-cube nodes with ~10x density contrast: Halton background plus Gaussian clusters."""
    n_c = int(round(frac_clustered * N))
    n_u = N - n_c
    idx = np.arange(1, n_u + 1)
    U = np.stack([halton(idx, b) for b in (2, 3, 5)], axis=1)
    centers = 0.15 + 0.7 * uniform(seed, n_clusters * 3, offset=1 << 44).reshape(n_clusters, 3)
    C = np.empty((n_c, 3))
    which = (splitmix64(seed, n_c, offset=1 << 45) % np.uint64(n_clusters)).astype(np.int64)
    todo = np.arange(n_c)
    off = 1 << 46
    while todo.size:
        u1 = uniform(seed, todo.size * 3, off).reshape(-1, 3)
        u2 = uniform(seed, todo.size * 3, off + todo.size * 3).reshape(-1, 3)
        off += todo.size * 6
        g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)  # Box-Muller
        cand = centers[which[todo]] + sigma * g
        ok = np.all((cand > 0.0) & (cand < 1.0), axis=1)
        C[todo[ok]] = cand[ok]
        todo = todo[~ok]
    P = np.concatenate([U, C], axis=0)
    P = P[permutation(seed, N)]
    return np.ascontiguousarray(P)


def disk2d_bc(N_int: int = 2000, seed: int = 1, refine: bool = True):
    """Unit disk with boundary nodes for a Neumann problem (the paper's 2D test, §5 and §7.1):
    N_int jittered Halton nodes inside radius 1 - h (h = sqrt(pi / N_int)), N_b = round(2 pi / h)
    nodes evenly spaced on the unit circle (seeded rotation) and, with `refine`, the boundary
    refinement layer of §6: copies of the boundary nodes h/2 inward along the normals.
    Returns (X, bc, normals): bc = 2 (Neumann) on the circle, 0 elsewhere; normals are the
    outward unit normals on the circle, zero elsewhere."""
    h = math.sqrt(math.pi / N_int)
    inside = lambda P: (P[:, 0] * P[:, 0] + P[:, 1] * P[:, 1]) <= (1.0 - h) * (1.0 - h)
    P = _jitter_in(_halton_in(N_int, 2, inside), h, 0.1, seed, inside)
    Nb = int(round(2.0 * math.pi / h))
    th = 2.0 * math.pi * (np.arange(Nb) + uniform(seed, 1, offset=1 << 47)[0]) / Nb
    B = np.stack([np.cos(th), np.sin(th)], axis=1)
    parts = [P] + ([(1.0 - 0.5 * h) * B] if refine else []) + [B]
    X = np.ascontiguousarray(np.concatenate(parts, axis=0))
    bc = np.zeros(X.shape[0], dtype=np.uint8)
    bc[-Nb:] = 2
    normals = np.zeros_like(X)
    normals[-Nb:] = B
    return X, bc, normals


def ball3d_bc(N_int: int = 20000, seed: int = 3):
    """Unit ball with boundary nodes for a Dirichlet problem (the paper's 3D test, §7.2):
    N_int jittered Halton nodes inside radius 1 - h (h = (4 pi / 3 / N_int)^(1/3)) and
    N_b = round(4 pi / h^2) nodes on the unit sphere on a Fibonacci lattice (seeded rotation).
    Returns (X, bc, normals): bc = 1 (Dirichlet) on the sphere; normals = the sphere points."""
    h = (4.0 * math.pi / 3.0 / N_int) ** (1.0 / 3.0)
    r2 = (1.0 - h) * (1.0 - h)
    inside = lambda P: (P[:, 0] * P[:, 0] + P[:, 1] * P[:, 1] + P[:, 2] * P[:, 2]) <= r2
    P = _jitter_in(_halton_in(N_int, 3, inside), h, 0.1, seed, inside)
    Nb = int(round(4.0 * math.pi / (h * h)))
    i = np.arange(Nb, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / Nb
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = i * (math.pi * (3.0 - math.sqrt(5.0))) + 2.0 * math.pi * uniform(seed, 1, offset=1 << 47)[0]
    B = np.stack([rr * np.cos(ph), rr * np.sin(ph), z], axis=1)
    X = np.ascontiguousarray(np.concatenate([P, B], axis=0))
    bc = np.zeros(X.shape[0], dtype=np.uint8)
    bc[-Nb:] = 1
    normals = np.zeros_like(X)
    normals[-Nb:] = B
    return X, bc, normals


def jittered_grid(side: int, d: int, amp: float = 0.2, seed: int = 7,
                  order: str = "random") -> np.ndarray:
    """side^d cell-centred points in [0,1]^d with U(-amp*h, amp*h) jitter (small test sets)."""
    h = 1.0 / side
    g = (np.arange(side, dtype=np.float64) + 0.5) * h
    mesh = np.meshgrid(*([g] * d), indexing="ij")
    P = np.stack([m.ravel() for m in mesh[::-1]], axis=1)
    N = P.shape[0]
    P = P + (2.0 * uniform(seed, N * d).reshape(N, d) - 1.0) * (amp * h)
    if order == "random":
        P = P[permutation(seed, N)]
    return np.ascontiguousarray(P)


def mixed_degree_params(X: np.ndarray, ells=(2, 3, 4, 5)):
    """Per-node stencil parameters for a node set split into len(ells) slabs along x (by the
    first coordinate's range): slab s uses degree ells[s], n = 2 M + 1 with M = C(ell+d, d)
    monomials, and PHS exponent m = 5 for ell = 2, else 7.  Returns int32 arrays (n, ell, m)."""
    N, d = X.shape
    x = X[:, 0]
    lo, hi = float(x.min()), float(x.max())
    slab = np.minimum(((x - lo) / max(hi - lo, 1e-300) * len(ells)).astype(np.int64),
                      len(ells) - 1)
    ell = np.asarray(ells, dtype=np.int32)[slab]
    M = np.array([math.comb(int(l) + d, d) for l in ell], dtype=np.int32)
    n = (2 * M + 1).astype(np.int32)
    m = np.where(ell == 2, 5, 7).astype(np.int32)
    return n, ell, m


#: The workloads, by name: (generator, kwargs, d, n, ell, m, deltas).
WORKLOADS = {
    "disk2d_N2000_l2_n12_r3": dict(gen=disk2d, kw=dict(N=2000, seed=1), d=2, n=12, ell=2, m=3,
                                   deltas=(1.0, 0.5)),
    "square2d_N40000_l4_n31_r7": dict(gen=square2d, kw=dict(N=40000, seed=2), d=2, n=31, ell=4,
                                      m=7, deltas=(1.0, 0.5, 0.3)),
    "ball3d_N100000_l3_n45_r7": dict(gen=ball3d, kw=dict(N=100000, seed=3), d=3, n=45, ell=3,
                                     m=7, deltas=(1.0, 0.4, 0.2)),
    # reduced sizes of the same recipes (small cases for full profiler captures)
    "ball3d_N20000_l3_n45_r7": dict(gen=ball3d, kw=dict(N=20000, seed=3), d=3, n=45, ell=3,
                                    m=7, deltas=(1.0, 0.4, 0.2)),
    "square2d_N10000_l4_n31_r7": dict(gen=square2d, kw=dict(N=10000, seed=2), d=2, n=31, ell=4,
                                      m=7, deltas=(1.0, 0.5, 0.3)),
    # the 2D square in row-major order: the traversal order is part of the input (§4.1), and
    # this one makes long dependency chains
    "square2d_raster_N40000_l4_n31_r7": dict(gen=square2d, kw=dict(N=40000, seed=2,
                                                                   order="raster"),
                                             d=2, n=31, ell=4, m=7, deltas=(1.0, 0.5, 0.3)),
}


#: Mixed-degree workload: clustered unit cube, degree 2..5 by x-slab, FALLBACK stabilization.
MIXED_WORKLOADS = {
    "cube3d_N500000_mixed_l2to5": dict(gen=cube3d_clustered, kw=dict(N=500000, seed=4), d=3,
                                       ells=(2, 3, 4, 5), deltas=(0.3,), mode="fallback"),
    # the same recipe at a size for full ncu captures of its kernels
    "cube3d_N20000_mixed_l2to5": dict(gen=cube3d_clustered, kw=dict(N=20000, seed=4), d=3,
                                      ells=(2, 3, 4, 5), deltas=(0.3,), mode="fallback"),
}


#: Workloads with boundary nodes (§5): generator returns (X, bc, normals).  The time-stepping
#: matrix coefficient c = (12/25) nu dt is the paper's BDF4 with nu = 1, dt = 1e-3 (§7).
BC_WORKLOADS = {
    "disk2d_bc_N40000_l4_n31_r7": dict(gen=disk2d_bc, kw=dict(N_int=40000, seed=1), d=2, n=31,
                                       ell=4, m=7, deltas=(1.0, 0.5, 0.3),
                                       timestep_c=12.0 / 25.0 * 1e-3),
}


def make(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return w["gen"](**w["kw"])
