"""CUDA path vs the CPU oracle, element by element, through the C ABI.

The bar: kNN stencils, stencil widths, retention balls, stencil ownership and the CSR
structure bit-exact; weights within 1e-9 of the row's largest weight (the tolerance the
method's specification states); Lebesgue values within 1e-9 relative.  Structural parity is
asserted where the oracle saw no Lebesgue decision within 1e-9 of a tie.
"""
import math
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


def gpu_run(X, n, ell, m, delta, mode=R.STAB_SEQ, host=False, **kw):
    nodes = X if host else torch.from_numpy(X).cuda()
    with R.Plan(nodes, n, ell, m, delta, mode=mode, **kw) as p:
        p.assemble()
        row_ptr, col, val, owner = p.export()
        nbr, rho2, bl = p.export_stencils()
        lam, isc = p.export_lambda()
        st = p.stats()
    return dict(row_ptr=row_ptr, col=col, val=val, owner=owner, nbr=nbr, rho2=rho2,
                ball_len=bl, lam_row=lam, is_center=isc, stats=st)


def check_rows(g, ref, n, rows=None):
    N = g["row_ptr"].size - 1
    rows = range(N) if rows is None else rows
    worst = 0.0
    for i in rows:
        a = g["val"][i * n:(i + 1) * n]
        b = ref["val"][i * n:(i + 1) * n]
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)  # an all-zero row must match exactly
        worst = max(worst, err)
        assert err <= TOL, f"row {i}: relative weight error {err:.3e}"
    return worst


def compare(X, n, ell, m, delta, mode=R.STAB_SEQ, ref=None, **kw):
    g = gpu_run(X, n, ell, m, delta, mode, **kw)
    if ref is None:
        ref = O.assemble(X, n, ell, m, delta, mode)
    assert np.array_equal(g["nbr"], ref["nbr"])
    assert np.array_equal(g["rho2"], ref["d2"][:, -1])
    assert np.array_equal(g["ball_len"], O.ball_len(ref["d2"], delta))
    if mode != R.STAB_OFF:  # with the test off, no Lebesgue decision shapes the result
        assert ref["stats"]["n_near_tie"] == 0
    assert np.array_equal(g["owner"], ref["owner"])
    assert np.array_equal(g["is_center"], ref["is_center"])
    assert np.array_equal(g["row_ptr"], ref["row_ptr"])
    assert np.array_equal(g["col"], ref["col"])
    check_rows(g, ref, n)
    np.testing.assert_allclose(g["lam_row"], ref["lam_row"], rtol=TOL, atol=0)
    assert g["stats"]["n_centers"] == ref["stats"]["n_centers"]
    assert g["stats"]["n_fallback"] == ref["stats"]["n_fallback"]
    assert g["stats"]["status"] == 0
    return g, ref


# ------------------------------------------------------------------ small workload, all modes
@pytest.mark.parametrize("delta", [1.0, 0.5])
def test_disk2d_N2000_seq(delta):
    X = NS.disk2d(2000, seed=1)
    g, ref = compare(X, 12, 2, 3, delta)
    if delta == 1.0:
        assert g["stats"]["n_centers"] == 2000
    else:
        assert ref["stats"]["n_rejected"] > 0


@pytest.mark.parametrize("mode", [R.STAB_OFF, R.STAB_FALLBACK])
def test_disk2d_N2000_other_modes(mode):
    X = NS.disk2d(2000, seed=1)
    g, ref = compare(X, 12, 2, 3, 0.5, mode)
    if mode == R.STAB_FALLBACK:
        assert ref["stats"]["n_fallback"] > 0


@pytest.mark.parametrize("make,n,ell,m,delta", [
    (lambda: NS.disk2d(2000, seed=1), 12, 2, 3, 0.5),
    (lambda: NS.jittered_grid(9, 3, seed=9), 45, 3, 7, 0.3),
    (lambda: NS.square2d(10000, seed=5), 31, 4, 7, 0.3),
])
def test_lu_factorization_option(make, n, ell, m, delta):
    # the partial-pivot LU (the paper's decomposition) and the default symmetric LDL^T give
    # the same matrix up to rounding
    compare(make(), n, ell, m, delta, factor=R.FACTOR_LU)


@pytest.mark.parametrize("N,n,ell,m,delta", [
    (12, 12, 2, 3, 0.5),     # N == n: every stencil is the whole node set
    (13, 12, 2, 3, 0.3),
    (37, 10, 2, 5, 0.4),     # ragged sizes
    (1, 1, 0, 3, 0.5),       # one node, one-term polynomial
    (1000, 31, 4, 7, 0.3),
    (900, 70, 4, 5, 0.2),    # wide stencils: more than 32 columns per stencil
])
def test_small_and_ragged_2d(N, n, ell, m, delta):
    X = NS.disk2d(N, seed=N)
    compare(X, n, ell, m, delta)


@pytest.mark.parametrize("delta,mode", [(0.6, R.STAB_OFF), (1.0, R.STAB_SEQ)])
def test_n_equals_M(delta, mode):
    # n == M: the weights are those of polynomial interpolation, whose Laplacian is the same
    # at every retained node, so every Lebesgue comparison is an exact tie decided by
    # rounding; only tie-free modes have a unique structure here
    X = NS.disk2d(300, seed=300)
    compare(X, 6, 2, 3, delta, mode)


@pytest.mark.parametrize("side,n,ell,m,delta", [(6, 20, 2, 5, 0.5), (9, 45, 3, 7, 0.3),
                                                (7, 35, 3, 5, 1.0)])
def test_small_3d(side, n, ell, m, delta):
    X = NS.jittered_grid(side, 3, seed=side)
    compare(X, n, ell, m, delta)


def test_raster_order_has_deep_dependency_chains():
    X = NS.square2d(10000, seed=2, order="raster")
    compare(X, 31, 4, 7, 0.5)


@pytest.mark.parametrize("scale,offset", [(1.0, 0.0), (1e-40, 0.0), (1e-20, 5e-20), (1e20, 0.0),
                                          (1e150, 0.0), (1.0, 1e6)])
def test_knn_is_exact_at_any_scale_and_offset(scale, offset):
    """The kNN screens candidates in FP32 before their exact FP64 distances: coordinates that
    are FP32 subnormals (1e-40), beyond FP32's range (1e150) or far from the origin (1e6)
    must still give the oracle's stencils and widths bit for bit."""
    for X0, n in ((NS.disk2d(2000, seed=11), 21), (NS.ball3d(2000, seed=12), 30)):
        X = X0 * scale + offset
        nbr, d2 = O.knn(X, n)
        with R.Plan(torch.from_numpy(X).cuda(), n, 2, 3, 0.5) as p:
            g_nbr, rho2, _ = p.export_stencils()
        assert np.array_equal(g_nbr, nbr), (scale, offset, X.shape[1])
        assert np.array_equal(rho2, d2[:, -1]), (scale, offset, X.shape[1])


def test_lattice_with_exact_distance_ties():
    # exact ties in distance are broken by index on both sides
    P = np.array([[i, j] for i in range(30) for j in range(30)], dtype=np.float64) * 0.125
    P = P[NS.permutation(3, P.shape[0])]
    g = gpu_run(P, 13, 2, 3, 1.0, mode=R.STAB_OFF)
    nbr, d2 = O.knn(P, 13)
    assert np.array_equal(g["nbr"], nbr)


def test_ill_conditioned_stencils_are_as_accurate_as_the_oracle():
    # n = 80, ell = 6: the local systems are ill-conditioned enough that rounding alone moves
    # some weights by about 1e-9 of the row scale on either side.  Both are compared with a
    # 40-digit solve of the same stencils; the GPU must be no less accurate than the oracle.
    from tests.hp_reference import mp_weights
    X = NS.disk2d(777, seed=777)
    n, ell, m, delta = 80, 6, 7, 0.25
    g = gpu_run(X, n, ell, m, delta)
    ref = O.assemble(X, n, ell, m, delta)
    assert np.array_equal(g["owner"], ref["owner"]) and np.array_equal(g["col"], ref["col"])
    errs = []
    for i in (23, 100, 400):
        j = ref["owner"][i]
        idx = ref["nbr"][j]
        w_hp = mp_weights(X, idx, ell, m, X[i:i + 1], dps=40)[:, 0]
        o = np.argsort(idx)
        scale = np.abs(w_hp).max()
        e_gpu = np.abs(g["val"][i * n:(i + 1) * n] - w_hp[o]).max() / scale
        e_ora = np.abs(ref["val"][i * n:(i + 1) * n] - w_hp[o]).max() / scale
        errs.append((e_gpu, e_ora))
        assert e_gpu <= max(1e-9, 4.0 * e_ora), (i, e_gpu, e_ora)
    print("forward errors (gpu, oracle):", errs)


# ------------------------------------------------------------------ full-size 2D workload
@pytest.mark.slow
def test_square2d_N40000_full_oracle_all_deltas():
    """The benchmark's workload in the benchmark's launch configuration: the three plans
    built on a side stream from pinned host nodes, assembled asynchronously in order on the
    compute stream, each CSR copied back on a copy stream (rbffd_export_async)."""
    X = NS.square2d(40000, seed=2)
    nbr, d2 = O.knn(X, 31)
    refs = {}
    for delta in (1.0, 0.5, 0.3):
        ref = O.assemble(X, 31, 4, 7, delta, O.STAB_SEQ, nbr, d2)
        ref["nbr"], ref["d2"] = nbr, d2
        refs[delta] = ref
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    Xp = pin(X.shape, torch.float64)
    Xp[...] = X
    side, copy = torch.cuda.Stream(), torch.cuda.Stream()
    compute = torch.cuda.current_stream()
    side.wait_stream(compute)
    plans, outs = [], {}
    for delta in refs:
        p = R.Plan(Xp, 31, 4, 7, delta, sync=False, stream=side)
        p.assemble(stream=compute)
        plans.append((delta, p))
    N = X.shape[0]
    for delta, p in plans:
        outs[delta] = p.export_async((pin(N + 1, torch.int64), pin(N * 31, torch.int32),
                                      pin(N * 31, torch.float64), pin(N, torch.int32)), copy)
    for delta, p in plans:
        st = p.stats()
        assert st["status"] == 0 and st["n_centers"] == refs[delta]["stats"]["n_centers"]
        row_ptr, col, val, owner = outs[delta]
        ref = refs[delta]
        assert np.array_equal(owner, ref["owner"])
        assert np.array_equal(row_ptr, ref["row_ptr"]) and np.array_equal(col, ref["col"])
        check_rows(dict(row_ptr=row_ptr, val=val), ref, 31)
        nb, rho2, bl = p.export_stencils()
        assert np.array_equal(nb, nbr) and np.array_equal(rho2, d2[:, -1])
        lam, isc = p.export_lambda()
        assert np.array_equal(isc, ref["is_center"])
        np.testing.assert_allclose(lam, ref["lam_row"], rtol=TOL, atol=0)
        p.close()


# ------------------------------------------------------------------ apply, repeatability, API
def test_apply_matches_csr_product():
    X = NS.disk2d(2000, seed=1)
    ref = O.assemble(X, 12, 2, 3, 0.5)
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5) as p:
        p.assemble()
        u = torch.from_numpy(np.cos(2 * X[:, 0]) + X[:, 1] ** 2).cuda()
        y = torch.zeros_like(u)
        p.apply(u, y)
        torch.cuda.synchronize()
    yr = O.csr_matvec(ref["row_ptr"], ref["col"], ref["val"], u.cpu().numpy())
    scale = O.csr_matvec(ref["row_ptr"], ref["col"], np.abs(ref["val"]),
                         np.abs(u.cpu().numpy()))
    assert np.all(np.abs(y.cpu().numpy() - yr) <= TOL * scale)


def test_reassembly_is_bitwise_repeatable_and_host_nodes_work():
    X = NS.square2d(10000, seed=5)
    with R.Plan(torch.from_numpy(X).cuda(), 31, 4, 7, 0.3) as p:
        p.assemble()
        a = p.export()
        p.assemble()
        b = p.export()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    c = gpu_run(X, 31, 4, 7, 0.3, host=True)
    assert np.array_equal(c["val"], a[2]) and np.array_equal(c["owner"], a[3])


def test_errors_are_reported_not_raised_on_device():
    X = NS.disk2d(500, seed=3)
    X[100] = X[17]
    with pytest.raises(R.RbffdError) as e:
        R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5)
    assert e.value.code == R.EDUPLICATE
    X = NS.disk2d(500, seed=3)
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5) as p:
        u = torch.zeros(500, dtype=torch.float64, device="cuda")
        with pytest.raises(R.RbffdError) as e:
            p.apply(u, u.clone())
        assert e.value.code == R.ESTATE


def test_bounded_wait_runs_out_and_context_survives():
    # fault injection on the host side of the kernel: no initial center is seeded, so every
    # worker's bounded wait for work runs out and the kernel returns RBFFD_ETIMEOUT
    X = NS.disk2d(2000, seed=1)
    t0 = time.time()
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5, timeout_ms=300,
                fault_inject=1) as p:
        with pytest.raises(R.RbffdError) as e:
            p.assemble()
        assert e.value.code == R.ETIMEOUT
    assert time.time() - t0 < 30
    compare(X, 12, 2, 3, 0.5)  # the context is still usable


# ------------------------------------------------------------------ 3D workload
@pytest.mark.slow
def test_ball3d_N20000_full_oracle_all_deltas():
    # exact structure in 3D at a size the oracle finishes in seconds
    X = NS.ball3d(20000, seed=3)
    nbr, d2 = O.knn(X, 45)
    for delta in (1.0, 0.4, 0.2):
        ref = O.assemble(X, 45, 3, 7, delta, O.STAB_SEQ, nbr, d2)
        ref["nbr"], ref["d2"] = nbr, d2
        compare(X, 45, 3, 7, delta, ref=ref)


def _lebesgue_accepts(X, nbr_j, ell, m, xi):
    """Oracle's Lebesgue test of stencil nbr_j (center nbr_j[0]) at point xi."""
    W, lam = O.local_weights(X, nbr_j, ell, m, np.stack([X[nbr_j[0]], xi]))
    return lam[1] <= lam[0], abs(lam[0] - lam[1]) / lam[0]


@pytest.mark.slow
@pytest.mark.parametrize("delta", [1.0, 0.4, 0.2])
def test_ball3d_N100000_sampled(delta):
    """Full-size 3D workload, in the launch configuration the benchmark uses.  The oracle
    checks sampled stencils, sampled rows, and the properties that characterise the
    traversal uniquely: a node is a center iff no earlier center keeps it; a kept row
    belongs to the earliest center keeping it."""
    X = NS.ball3d(100000, seed=3)
    n, ell, m = 45, 3, 7
    g = gpu_run(X, n, ell, m, delta)
    N = X.shape[0]
    rng = NS.permutation(17, N)
    # kNN and balls on sampled nodes, by brute force
    for k in rng[:300]:
        diff = X[k][None, :] - X
        s = diff[:, 0] * diff[:, 0]
        s = s + diff[:, 1] * diff[:, 1]
        s = s + diff[:, 2] * diff[:, 2]
        order = np.lexsort((np.arange(N), s))[:n]
        assert np.array_equal(g["nbr"][k], order)
        assert g["rho2"][k] == s[order[-1]]
        f = (1.0 - delta) * (1.0 - delta)
        assert g["ball_len"][k] == int((s[order] <= f * s[order[-1]]).sum())
    nbr, bl, owner, isc = g["nbr"], g["ball_len"], g["owner"], g["is_center"]
    # in-neighbours: earlier nodes whose ball holds k
    ins = [[] for _ in range(N)]
    for j in range(N):
        for t in range(1, bl[j]):
            i = nbr[j, t]
            if i > j:
                ins[i].append(j)
    # every row: owner is a center <= i whose ball holds i
    assert np.all(owner <= np.arange(N))
    assert np.all(isc[owner] == 1)
    near = 0
    for i in rng[:400]:
        o = owner[i]
        assert i == o or i in nbr[o, :bl[o]]
        earlier = sorted(j for j in ins[i] if isc[j] == 1 and j < (o if o != i else i))
        for j in earlier:  # no earlier center keeps i
            acc, margin = _lebesgue_accepts(X, nbr[j], ell, m, X[i])
            if margin <= 1e-9:
                near += 1
                continue
            assert not acc, (i, j)
        if o != i:
            acc, margin = _lebesgue_accepts(X, nbr[o], ell, m, X[i])
            assert acc or margin <= 1e-9
        # the row's weights are the owner stencil's weights at x_i
        W, _ = O.local_weights(X, nbr[o], ell, m, X[i:i + 1])
        order = np.argsort(nbr[o])
        a = g["val"][i * n:(i + 1) * n]
        assert np.array_equal(g["col"][i * n:(i + 1) * n], nbr[o][order])
        assert np.abs(a - W[order, 0]).max() <= TOL * np.abs(W).max()
    assert near == 0
    assert g["stats"]["status"] == 0


# ------------------------------------------------------------------ per-node stencils
def gpu_run_mixed(X, n_node, ell_node, m_node, delta, mode=R.STAB_SEQ, **kw):
    with R.Plan(torch.from_numpy(X).cuda(), n_node, ell_node, m_node, delta, mode=mode,
                **kw) as p:
        p.assemble()
        row_ptr, col, val, owner = p.export()
        nbr, rho2, bl = p.export_stencils()
        lam, isc = p.export_lambda()
        st = p.stats()
    return dict(row_ptr=row_ptr, col=col, val=val, owner=owner, nbr=nbr, rho2=rho2,
                ball_len=bl, lam_row=lam, is_center=isc, stats=st)


def forward_errors(X, g, ref, n_node, ell_node, m_node, rows, rho2):
    """Forward errors of the GPU's and the oracle's rows (and scaled Lebesgue values) against
    a double-double solve of each row's stencil (tests/hp_reference.py), relative to the row's
    largest exact weight.  Rows sharing a stencil share its factorization."""
    from tests.hp_reference import dd_weights
    src = np.where(ref["is_center"] >= 2, np.arange(X.shape[0]), ref["owner"])
    out = {}
    for s_ in np.unique(src[rows]):
        rs = [i for i in rows if src[i] == s_]
        idx = ref["nbr"][s_, :n_node[s_]]
        W = dd_weights(X, idx, int(ell_node[s_]), int(m_node[s_]), X[rs])
        order = np.argsort(idx)
        for k, i in enumerate(rs):
            sl = slice(ref["row_ptr"][i], ref["row_ptr"][i + 1])
            w = W[order, k]
            sc = np.abs(w).max()
            lam = np.abs(w).sum() * rho2[s_]  # the scaled local Lebesgue value of the row
            lg = abs(g["lam_row"][i] - lam) / lam if "lam_row" in g else 0.0
            out[i] = (np.abs(g["val"][sl] - w).max() / sc, np.abs(ref["val"][sl] - w).max() / sc,
                      lg, abs(ref["lam_row"][i] - lam) / lam)
    return out


def check_mixed_rows(X, g, ref, n_node, ell_node, m_node, per_class=25, seed=99, max_bad=None,
                     min_rows=100):
    """Weights of per-node (or ill-conditioned uniform) stencils against the oracle.

    Rows within 1e-9 of the oracle pass as they are.  The degree-4 and degree-5 stencils of
    the clustered cube (K = 106 and 169) reach condition numbers near 3e10, where any FP64
    solver is up to ~3e-7 from the exact weights (the oracle's LU, LAPACK and the library
    alike), so 1e-9 between two FP64 solvers is not attainable there.  Every row above 1e-9
    (with max_bad: that many, the worst first), and a stratified sample of `per_class` rows of
    every degree, is measured against a double-double (~32-digit) solve of its stencil, and
    the GPU's forward errors must meet the bar of tests/hp_reference.accuracy_failures against
    the oracle's (which LAPACK meets too), for the weights and for the Lebesgue values (when g
    has them).  Returns the per-degree summary of the sampled forward errors."""
    from tests.hp_reference import accuracy_failures
    N = X.shape[0]
    rp = ref["row_ptr"]
    errs = np.array([np.abs(g["val"][rp[i]:rp[i + 1]] - ref["val"][rp[i]:rp[i + 1]]).max() /
                     np.abs(ref["val"][rp[i]:rp[i + 1]]).max() for i in range(N)])
    src = np.where(ref["is_center"] >= 2, np.arange(N), ref["owner"])
    cls = ell_node[src]
    perm = NS.permutation(seed, N)
    bad = np.nonzero(errs > TOL)[0]
    if max_bad is not None:
        bad = bad[np.argsort(errs[bad])[::-1][:max_bad]]
    rows = set(bad.tolist())
    for c in np.unique(cls):
        rows.update([int(i) for i in perm if cls[i] == c][:per_class])
    rows = sorted(rows)
    rho2 = ref["d2"][np.arange(N), n_node - 1]
    fe = forward_errors(X, g, ref, n_node, ell_node, m_node, rows, rho2)
    v = np.array([fe[i] for i in rows])
    c_rows = cls[rows]
    fails = accuracy_failures(v[:, 0], v[:, 1], c_rows)
    if "lam_row" in g:
        fails += ["Lebesgue " + f for f in accuracy_failures(v[:, 2], v[:, 3], c_rows, v[:, 0])]
    summary = {}
    for c in np.unique(cls):
        w = v[c_rows == c]
        summary[int(c)] = dict(rows=int(w.shape[0]), above_1e9=int((errs[cls == c] > TOL).sum()),
                               gpu_max=float(w[:, 0].max()), gpu_median=float(np.median(w[:, 0])),
                               oracle_max=float(w[:, 1].max()),
                               oracle_median=float(np.median(w[:, 1])))
    print("forward errors per degree:", summary)
    assert not fails, fails[:10]
    assert len(rows) >= min_rows
    return summary


def assert_stencils_equal(g_nbr, ref_nbr, n_node):
    """Per-node stencils: row k's first n_k entries equal the oracle's kNN order (the GPU
    searches only that many neighbours for node k) and the rest of the row is -1."""
    ref_nbr = np.asarray(ref_nbr)
    g = np.asarray(g_nbr).reshape(ref_nbr.shape)
    inside = np.arange(ref_nbr.shape[1])[None, :] < np.asarray(n_node)[:, None]
    assert np.array_equal(g[inside], ref_nbr[inside])
    assert np.all(g[~inside] == -1)


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_mixed_degrees_3d_match_the_mixed_oracle(mode):
    X = NS.cube3d_clustered(3000, seed=4)
    n_node, ell_node, m_node = NS.mixed_degree_params(X)
    g = gpu_run_mixed(X, n_node, ell_node, m_node, 0.3, mode)
    ref = O.assemble_mixed(X, n_node, ell_node, m_node, 0.3, mode)
    assert ref["stats"]["n_near_tie"] == 0
    assert_stencils_equal(g["nbr"], ref["nbr"], n_node)
    assert np.array_equal(g["owner"], ref["owner"])
    assert np.array_equal(g["is_center"], ref["is_center"])
    assert np.array_equal(g["row_ptr"], ref["row_ptr"])
    assert np.array_equal(g["col"], ref["col"])
    check_mixed_rows(X, g, ref, n_node, ell_node, m_node)
    assert g["stats"]["n_fallback"] == ref["stats"]["n_fallback"]
    assert g["stats"]["nnz"] == ref["row_ptr"][-1]


@pytest.mark.slow
@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_mixed_degrees_3d_N20000_match_the_mixed_oracle(mode):
    """The same at N = 20,000 (the clustered cube's recipe, degree 2..5 by x-slab)."""
    X = NS.cube3d_clustered(20000, seed=4)
    n_node, ell_node, m_node = NS.mixed_degree_params(X)
    g = gpu_run_mixed(X, n_node, ell_node, m_node, 0.3, mode)
    ref = O.assemble_mixed(X, n_node, ell_node, m_node, 0.3, mode)
    assert ref["stats"]["n_near_tie"] == 0
    assert_stencils_equal(g["nbr"], ref["nbr"], n_node)
    for key in ("owner", "is_center", "row_ptr", "col"):
        assert np.array_equal(g[key], ref[key]), key
    check_mixed_rows(X, g, ref, n_node, ell_node, m_node)
    assert g["stats"]["n_fallback"] == ref["stats"]["n_fallback"]
    assert g["stats"]["refine_min_K"] == R.REFINE_MIN_K


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_degree4_3d_plan_with_refinement_matches_the_oracle(mode):
    """A uniform degree-4 3D plan (n = 71, K = 106, delta = 0.4): large-system teams, the
    refinement step and, with a Lebesgue test in force, its selection of the columns that can
    be kept, against the oracle (structure bit-exact, weights and Lebesgue values at the
    double-double bar of check_mixed_rows)."""
    X = NS.ball3d(3000, seed=7)
    N, n, ell, m = X.shape[0], 71, 4, 7
    g = gpu_run(X, n, ell, m, 0.4, mode)
    ref = O.assemble(X, n, ell, m, 0.4, mode)
    assert ref["stats"]["n_near_tie"] == 0
    for key in ("nbr", "owner", "is_center", "row_ptr", "col"):
        assert np.array_equal(g[key], ref[key]), key
    check_rows(g, ref, n)  # (these stencils are well enough conditioned for 1e-9)
    check_mixed_rows(X, g, ref, np.full(N, n), np.full(N, ell), np.full(N, m), per_class=100)
    assert g["stats"]["refine_min_K"] == R.REFINE_MIN_K and g["stats"]["flops_refine"] > 0
    assert g["stats"]["n_fallback"] == ref["stats"]["n_fallback"]
    # the kept-column selection refines fewer columns than refining every solved one
    a = gpu_run(X, n, ell, m, 0.4, mode, refine=R.REFINE_ALL)
    assert g["stats"]["flops_refine"] < a["stats"]["flops_refine"]


def test_refinement_options_on_per_node_stencils():
    """Refinement changes weights only (rounding), never the structure: with every system
    refined, only the ill-conditioned ones (the default) or none, the matrices share their
    structure; the default refines a part of what refining everything does."""
    X = NS.cube3d_clustered(3000, seed=4)
    params = NS.mixed_degree_params(X)
    runs = {r: gpu_run_mixed(X, *params, 0.3, refine=r)
            for r in (R.REFINE_AUTO, R.REFINE_ALL, R.REFINE_NONE)}
    for r, g in runs.items():
        for key in ("owner", "is_center", "row_ptr", "col"):
            assert np.array_equal(g[key], runs[R.REFINE_AUTO][key]), (r, key)
        assert g["stats"]["refine_min_K"] == {R.REFINE_NONE: 0x7fffffff, R.REFINE_ALL: 0,
                                              R.REFINE_AUTO: R.REFINE_MIN_K}[r]
    fr = {r: g["stats"]["flops_refine"] for r, g in runs.items()}
    assert fr[R.REFINE_NONE] == 0 < fr[R.REFINE_AUTO] < fr[R.REFINE_ALL]


def test_mixed_entry_with_uniform_parameters_equals_the_uniform_plan():
    X = NS.disk2d(3000, seed=8)
    N = X.shape[0]
    a = gpu_run(X, 12, 2, 3, 0.5)
    b = gpu_run_mixed(X, np.full(N, 12), np.full(N, 2), np.full(N, 3), 0.5)
    for key in ("row_ptr", "col", "val", "owner", "nbr", "ball_len", "lam_row"):
        assert np.array_equal(a[key], b[key]), key


# ------------------------------------------------------------------ the largest stencils
def test_largest_stencil_size_matches_the_oracle():
    """n = 128 (the limit), K = 134: one 512-thread team per system."""
    X = NS.jittered_grid(40, 2, seed=21)
    g, _ = compare(X, 128, 2, 3, 1.0)
    assert g["stats"]["K"] == 134


def test_balls_too_large_for_one_chunk_match_the_oracle():
    """n = 128, degree 5, r^5 at delta = 0.05: K = 149 and balls of up to ~126 columns, more
    right-hand sides than fit in shared memory beside the system, so later columns are solved
    in chunks with the stored factors."""
    X = NS.jittered_grid(40, 2, seed=21)
    g, _ = compare(X, 128, 5, 5, 0.05)
    assert g["stats"]["K"] == 149 and g["stats"]["max_ball"] > 100


@pytest.mark.parametrize("team", [0, 32, 512])
@pytest.mark.parametrize("chunk", [1, 2, 5])
def test_forced_chunks_are_bitwise_equal_to_one_chunk(team, chunk):
    """Columns solved after the factorization get the same operations as the ones carried
    through it, so any chunk size gives the same bits (2D and 3D, warp and CTA teams)."""
    for X, n, ell, m in ((NS.disk2d(3000, seed=4), 31, 4, 7),
                         (NS.ball3d(3000, seed=5), 45, 3, 7)):
        a = gpu_run(X, n, ell, m, 0.3, team=team)
        b = gpu_run(X, n, ell, m, 0.3, team=team, rhs_chunk=chunk)
        for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
            assert np.array_equal(a[key], b[key]), (key, n)


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_OFF, R.STAB_FALLBACK])
def test_forced_chunks_match_the_oracle(mode):
    g, _ = compare(NS.disk2d(2000, seed=6), 21, 3, 5, 0.3, mode, rhs_chunk=2)
    assert g["stats"]["rhs_chunk"] == 2 and g["stats"]["max_ball"] > 2


def test_forced_chunks_on_per_node_stencils_are_bitwise_equal():
    """Per-node degrees 2..5 (K up to 169) with chunks of 4 columns against one chunk."""
    X = NS.cube3d_clustered(3000, seed=4)
    params = NS.mixed_degree_params(X)
    a = gpu_run_mixed(X, *params, 0.3)
    b = gpu_run_mixed(X, *params, 0.3, rhs_chunk=4)
    assert b["stats"]["rhs_chunk"] == 4 and a["stats"]["max_ball"] > 4
    for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
        assert np.array_equal(a[key], b[key]), key


def test_lu_keeps_every_column_and_refuses_balls_that_do_not_fit():
    """LU stores K (K + q) entries and has no chunked solve: the large-ball case that LDL^T
    solves in chunks is RBFFD_EINVAL with LU."""
    X = torch.from_numpy(NS.jittered_grid(40, 2, seed=21)).cuda()
    with pytest.raises(R.RbffdError) as e:
        R.Plan(X, 128, 5, 5, 0.05, factor=R.FACTOR_LU)
    assert e.value.code == R.EINVAL
    with R.Plan(X, 12, 2, 3, 0.3, factor=R.FACTOR_LU) as p:
        st = p.stats()
        assert st["rhs_chunk"] == st["max_ball"]


def test_systems_too_large_for_shared_memory_are_rejected():
    """3D, n = 128 with degree 7: K = 248, whose packed triangle alone (247 KB) is above the
    227 KB of shared memory a CTA can have; the plan says RBFFD_EINVAL."""
    X = torch.from_numpy(NS.jittered_grid(12, 3, seed=21)).cuda()
    with pytest.raises(R.RbffdError) as e:
        R.Plan(X, 128, 7, 7, 1.0)
    assert e.value.code == R.EINVAL


# ------------------------------------------------------------------ centroid reference (§4.2.1)
@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_OFF, R.STAB_FALLBACK])
@pytest.mark.parametrize("case", ["2d", "3d"])
def test_centroid_reference_matches_the_oracle(mode, case):
    """The Lebesgue test against the stencil node nearest the stencil's centroid: reference
    positions from the per-plan pre-pass, the reference solved as one more column when it is
    not a retained node, the center always kept."""
    if case == "2d":
        X, n, ell, m = NS.disk2d(2000, seed=6), 21, 3, 5
    else:
        X, n, ell, m = NS.ball3d(3000, seed=5), 45, 3, 7
    ref = O.assemble(X, n, ell, m, 0.3, mode, lref=O.LREF_CENTROID)
    compare(X, n, ell, m, 0.3, mode, ref=ref, lebesgue_ref=R.LREF_CENTROID)
    # (solved-column counts may differ: the dataflow can solve a member that a center before
    # it, finishing later, keeps; the oracle solves each center's columns in index order)


@pytest.mark.parametrize("team,chunk", [(0, 1), (0, 2), (32, 0), (512, 3)])
def test_centroid_reference_in_chunks_and_teams_is_bitwise_equal(team, chunk):
    X = NS.disk2d(3000, seed=4)
    a = gpu_run(X, 31, 4, 7, 0.3, lebesgue_ref=R.LREF_CENTROID)
    b = gpu_run(X, 31, 4, 7, 0.3, lebesgue_ref=R.LREF_CENTROID, team=team, rhs_chunk=chunk)
    for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
        assert np.array_equal(a[key], b[key]), key


def test_centroid_reference_on_per_node_stencils_matches_the_mixed_oracle():
    X = NS.cube3d_clustered(3000, seed=4)
    params = NS.mixed_degree_params(X)
    g = gpu_run_mixed(X, *params, 0.3, lebesgue_ref=R.LREF_CENTROID)
    ref = O.assemble_mixed(X, *params, 0.3, lref=O.LREF_CENTROID)
    assert ref["stats"]["n_near_tie"] == 0
    for key in ("owner", "is_center", "row_ptr", "col"):
        assert np.array_equal(g[key], ref[key]), key
    check_mixed_rows(X, g, ref, *params)


def test_centroid_reference_at_the_largest_stencil_size():
    """n = 128: the reference pre-pass walks four lanes' worth of nodes per warp lane."""
    X = NS.jittered_grid(40, 2, seed=21)
    ref = O.assemble(X, 128, 2, 3, 0.5, lref=O.LREF_CENTROID)
    compare(X, 128, 2, 3, 0.5, ref=ref, lebesgue_ref=R.LREF_CENTROID)


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_blocked_triangular_solves_of_large_teams_are_bitwise_equal(mode):
    """256- and 512-thread teams take the triangular solves 32 unknowns at a time with all
    warps (the back substitution always, the forward substitution for chunks after the first);
    every entry gets the same FMAs in the same order as the step-by-step solves of a warp
    team.  (512-thread teams also look one pivot ahead in the factorization.)"""
    for X, n, ell, m in ((NS.disk2d(3000, seed=4), 31, 4, 7),
                         (NS.ball3d(3000, seed=5), 45, 3, 7),
                         (NS.jittered_grid(40, 2, seed=21), 128, 5, 5)):
        a = gpu_run(X, n, ell, m, 0.3, mode, team=32)
        for team, chunk in ((512, 0), (512, 2), (256, 0), (256, 2)):
            b = gpu_run(X, n, ell, m, 0.3, mode, team=team, rhs_chunk=chunk)
            for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
                assert np.array_equal(a[key], b[key]), (key, n, team, chunk)


@pytest.mark.parametrize("team,chunk", [(32, 0), (64, 3), (256, 0), (256, 3), (512, 0), (512, 2)])
def test_refined_schedules_are_bitwise_equal(team, chunk):
    """The refinement step does the same arithmetic on every entry whatever the team size or
    chunk (a warp per column or per residual entry), so refined results agree bit for bit."""
    X = NS.cube3d_clustered(3000, seed=4)
    params = NS.mixed_degree_params(X)
    a = gpu_run_mixed(X, *params, 0.3)
    b = gpu_run_mixed(X, *params, 0.3, team=team, rhs_chunk=chunk)
    for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
        assert np.array_equal(a[key], b[key]), key


def test_teams_without_the_refinement_step_are_refused_for_refined_systems():
    X = torch.from_numpy(NS.cube3d_clustered(3000, seed=4)).cuda()
    params = NS.mixed_degree_params(X.cpu().numpy())
    for team in (96, 128):
        with pytest.raises(R.RbffdError) as e:
            R.Plan(X, *params, 0.3, team=team)
        assert e.value.code == R.EINVAL
        with R.Plan(X, *params, 0.3, team=team, refine=R.REFINE_NONE) as p:
            p.assemble()


@pytest.mark.parametrize("elastic", [1, 8, 152])
def test_elastic_grid_forms_the_same_matrix_alone_and_beside_other_plans(elastic):
    """CTAs that leave the traversal's dependency tail (rbffd_opts.elastic) change who solves a
    center, never its arithmetic: the matrix is bit-identical, for one plan and for three
    deltas assembled at once on their own streams."""
    X = NS.square2d(10000, seed=5)
    Xd = torch.from_numpy(X).cuda()
    ref = {d: gpu_run(X, 31, 4, 7, d) for d in (1.0, 0.5, 0.3)}
    g = gpu_run(X, 31, 4, 7, 0.3, elastic=elastic)
    for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
        assert np.array_equal(g[key], ref[0.3][key]), key
    streams = [torch.cuda.Stream() for _ in ref]
    plans = []
    for s, d in zip(streams, ref):
        p = R.Plan(Xd, 31, 4, 7, d, sync=False, elastic=elastic)
        p.assemble(stream=s)
        plans.append((d, p))
    torch.cuda.synchronize()
    for d, p in plans:
        assert p.stats()["status"] == 0
        got = p.export()
        for a, b in zip(got, (ref[d][k] for k in ("row_ptr", "col", "val", "owner"))):
            assert np.array_equal(a, b), d
        p.close()
