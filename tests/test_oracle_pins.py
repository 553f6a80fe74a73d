"""Pins for the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: printed values of the
paper (§2 degree rule), hand derivations (tests/golden), closed forms (5-point and 7-point
Laplacians, Kronecker property), an independent 40-digit solve built with sympy/mpmath from
the definitions of §4.1, library routines (numpy sorting for kNN), exact invariances, and
convergence of L f to the Laplacian of f.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1606_03135_gb300 import nodesets as NS
from tests.hp_reference import mp_weights as _mp_weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng_points(N, d, seed):
    return NS.uniform(seed, N * d).reshape(N, d)


# ------------------------------------------------------------------ §2 degree rule
def test_degree_rule_matches_paper_examples():
    g = json.load(open(os.path.join(GOLDEN, "degree_rule.json")))
    for c in g["cases"]:
        assert O.degree_for_n(c["n"], c["d"]) == (c["s"], c["M"])


def test_degree_rule_is_largest_fitting_degree():
    for d in (2, 3):
        for n in range(2, 400):
            s, M = O.degree_for_n(n, d)
            assert M == math.comb(s + d, d)
            assert 2 * math.comb(s + d, d) <= n < 2 * math.comb(s + 1 + d, d)


def test_poly_terms_span_all_monomials_in_graded_order():
    for d in (2, 3):
        for ell in range(0, 7):
            e = O.poly_terms(d, ell)
            want = {a for a in itertools.product(range(ell + 1), repeat=d) if sum(a) <= ell}
            assert len(e) == math.comb(ell + d, d) == len(want)
            assert {tuple(r) for r in e} == want
            deg = e.sum(axis=1)
            assert np.all(np.diff(deg) >= 0)


# ------------------------------------------------------------------ kNN (§2, §4.1)
def _knn_numpy(X, n):
    N, d = X.shape
    nbr = np.zeros((N, n), np.int32)
    d2 = np.zeros((N, n))
    for k in range(N):
        diff = X[k][None, :] - X
        s = diff[:, 0] * diff[:, 0]
        s = s + diff[:, 1] * diff[:, 1]
        if d == 3:
            s = s + diff[:, 2] * diff[:, 2]
        order = np.lexsort((np.arange(N), s))[:n]
        nbr[k] = order
        d2[k] = s[order]
    return nbr, d2


@pytest.mark.parametrize("d", [2, 3])
def test_knn_matches_numpy_sort_with_exact_ties(d):
    # an integer lattice has many exactly equal distances: the (d2, index) order decides
    side = 9 if d == 2 else 5
    P = np.array(list(itertools.product(range(side), repeat=d)), dtype=np.float64)
    P = P[NS.permutation(5, P.shape[0])]
    for n in (1, 5, 13, 27):
        nbr, d2 = O.knn(P, n)
        nb2, d22 = _knn_numpy(P, n)
        assert np.array_equal(nbr, nb2)
        assert np.array_equal(d2, d22)
        assert np.all(nbr[:, 0] == np.arange(P.shape[0]))


def test_knn_random_matches_numpy():
    X = _rng_points(700, 2, 11)
    nbr, d2 = O.knn(X, 17)
    nb2, d22 = _knn_numpy(X, 17)
    assert np.array_equal(nbr, nb2) and np.array_equal(d2, d22)


def test_knn_duplicate_is_an_error():
    X = _rng_points(50, 2, 3)
    X[31] = X[7]
    with pytest.raises(O.OracleError) as e:
        O.knn(X, 5)
    assert e.value.code == O.EDUPLICATE


# ------------------------------------------------------------------ retention balls (§4.1)
def test_ball_len_special_cases_and_definition():
    X = NS.disk2d(500, seed=9)
    nbr, d2 = O.knn(X, 12)
    assert np.all(O.ball_len(d2, 1.0) == 1)  # delta = 1: the ball is the center alone
    assert np.all(O.ball_len(d2, 1e-17) == 12)  # (1-delta) rounds to 1: the whole stencil
    for delta in (0.2, 0.5, 0.75):
        f = (1.0 - delta) * (1.0 - delta)
        want = (d2 <= (f * d2[:, -1])[:, None]).sum(axis=1)
        assert np.array_equal(O.ball_len(d2, delta), want)
    with pytest.raises(O.OracleError):
        O.ball_len(d2, 0.0)


# ------------------------------------------------------------------ local system (§4.1)
def test_five_point_laplacian_is_recovered_when_n_equals_M():
    # n = M = 6 (ell = 2): P is square, the weights are those of quadratic interpolation,
    # which on {0, +-h e1, +-h e2, (h,h)} is the 5-point Laplacian.
    for h in (1.0, 0.125, 3e-3):
        X = np.array([[0, 0], [h, 0], [-h, 0], [0, h], [0, -h], [h, h]], dtype=np.float64) + 0.3
        W, _ = O.local_weights(X, np.arange(6), 2, 3, X[:1])
        np.testing.assert_allclose(W[:, 0] * h * h, [-4, 1, 1, 1, 1, 0], atol=1e-11)


def test_seven_point_laplacian_3d_when_n_equals_M():
    h = 0.5
    pts = [[0, 0, 0], [h, 0, 0], [-h, 0, 0], [0, h, 0], [0, -h, 0], [0, 0, h], [0, 0, -h],
           [h, h, 0], [h, 0, h], [0, h, h]]
    X = np.array(pts, dtype=np.float64) - 0.2
    W, _ = O.local_weights(X, np.arange(10), 2, 5, X[:1])
    np.testing.assert_allclose(W[:, 0] * h * h, [-6, 1, 1, 1, 1, 1, 1, 0, 0, 0], atol=1e-11)


@pytest.mark.parametrize("d,n,ell,m,seed", [(2, 8, 1, 3, 1), (2, 10, 2, 5, 2), (3, 12, 1, 3, 3),
                                            (3, 14, 2, 7, 4), (2, 15, 3, 7, 5)])
def test_local_weights_match_independent_40_digit_solve(d, n, ell, m, seed):
    X = 0.05 * _rng_points(n, d, seed) + 0.4
    idx = np.arange(n)
    Y = X[[0, 1, n // 2]]
    W, _ = O.local_weights(X, idx, ell, m, Y)
    Wmp = _mp_weights(X, idx, ell, m, Y)
    for e in range(Y.shape[0]):
        scale = np.abs(Wmp[:, e]).max()
        assert np.abs(W[:, e] - Wmp[:, e]).max() <= 1e-9 * scale


@pytest.mark.parametrize("d,n,ell,m", [(2, 31, 4, 7), (3, 45, 3, 7), (2, 12, 2, 3)])
def test_polynomial_reproduction(d, n, ell, m):
    # the augmented system reproduces every polynomial of degree <= ell exactly (§2, §4.1)
    X = NS.jittered_grid(14 if d == 2 else 7, d, seed=3)
    nbr, _ = O.knn(X, n)
    rng_k = [5, 77, 150]
    for k in rng_k:
        idx = nbr[k]
        Y = X[idx[:6]]
        W, _ = O.local_weights(X, idx, ell, m, Y)
        c = X[k] + 0.01
        for al in itertools.product(range(ell + 1), repeat=d):
            if sum(al) > ell:
                continue
            pv = np.prod((X[idx] - c) ** np.array(al), axis=1)
            for e in range(Y.shape[0]):
                y = Y[e] - c
                lap = 0.0
                for a in range(d):
                    if al[a] >= 2:
                        t = al[a] * (al[a] - 1)
                        for b in range(d):
                            t *= y[b] ** (al[b] - 2 if b == a else al[b])
                        lap += t
                got = W[:, e] @ pv
                scale = np.abs(W[:, e]) @ np.abs(pv) + abs(lap) + 1e-300
                assert abs(got - lap) <= 1e-10 * scale


def test_identity_operator_has_kronecker_property_and_lebesgue_at_least_one():
    # interpolation Lagrange functions (§4.2.1): l_j(x_i) = delta_ij, sum_j l_j = 1,
    # hence Lambda = sum_j |l_j| >= 1 everywhere and == 1 at the nodes.
    X = NS.jittered_grid(12, 2, seed=4)
    nbr, _ = O.knn(X, 21)
    idx = nbr[40]
    W, lam = O.local_weights(X, idx, 3, 5, X[idx], op=O.OP_IDENTITY)
    np.testing.assert_allclose(W, np.eye(21), atol=1e-10)
    np.testing.assert_allclose(lam, 1.0, atol=1e-10)
    lo, hi = X[idx].min(axis=0), X[idx].max(axis=0)
    Y = lo + (hi - lo) * NS.uniform(8, 60).reshape(30, 2)
    W, lam = O.local_weights(X, idx, 3, 5, Y, op=O.OP_IDENTITY)
    np.testing.assert_allclose(W.sum(axis=0), 1.0, atol=1e-10)
    assert np.all(lam >= 1.0 - 1e-10)


def test_laplacian_lebesgue_lower_bound():
    # p(xi) = |xi - xi_R|^2 has Laplacian 2d and is reproduced (ell >= 2), so in scaled
    # units Lambda(x_R) >= 2d / max_j |xi_j - xi_R|^2.
    for d, side, n, ell in ((2, 14, 31, 4), (3, 7, 45, 3)):
        X = NS.jittered_grid(side, d, seed=6)
        nbr, d2 = O.knn(X, n)
        for k in (3, 50, 150):
            idx = nbr[k]
            W, lam = O.local_weights(X, idx, ell, 7, X[idx[:8]])
            rho = math.sqrt(d2[k, -1])
            for e in range(8):
                far = (((X[idx] - X[idx[e]]) / rho) ** 2).sum(axis=1).max()
                assert lam[e] >= 2 * d / far * (1 - 1e-12)


# ------------------------------------------------------------------ traversal (§4.1, §4.2.1)
def test_hand_derived_traversal_line8():
    g = json.load(open(os.path.join(GOLDEN, "line8_off.json")))
    X = np.array([[k, 0.001 * (k % 2)] for k in range(8)], dtype=np.float64)
    r = O.assemble(X, g["n"], g["ell"], g["m"], g["delta"], mode=O.STAB_OFF)
    assert np.array_equal(r["nbr"], np.array(g["nbr"]))
    assert np.array_equal(O.ball_len(r["d2"], g["delta"]), g["ball_len"])
    assert np.array_equal(np.flatnonzero(r["is_center"] == 1), g["centers"])
    assert np.array_equal(r["owner"], g["owner"])


def _acc(X, nbr, bl, j, ell, m):
    idx = nbr[j]
    W, lam = O.local_weights(X, idx, ell, m, X[idx[:bl[j]]])
    return W, lam, lam <= lam[0]


@pytest.mark.parametrize("mode", [O.STAB_SEQ, O.STAB_OFF, O.STAB_FALLBACK])
@pytest.mark.parametrize("delta", [1e-9, 0.25, 0.5, 0.8])
def test_traversal_satisfies_its_unique_characterisation(mode, delta):
    # delta -> 0: every ball is the whole stencil, so a center's retained set is the
    # uncovered part of its stencil (§4.1).
    # The index-order traversal is the unique assignment in which node k is a center iff no
    # earlier center keeps it, and each kept row belongs to the earliest center keeping it.
    X = NS.disk2d(300, seed=21)
    n, ell, m = 12, 2, 3
    r = O.assemble(X, n, ell, m, delta, mode=mode)
    bl = O.ball_len(r["d2"], delta)
    acc = {j: _acc(X, r["nbr"], bl, j, ell, m) for j in np.flatnonzero(r["is_center"] == 1)}
    _check_characterisation(X, r, bl, acc, mode, ell, m)


def _check_characterisation(X, r, bl, acc, mode, ell, m):
    """The index-order traversal's unique assignment, given each center's acceptance flags
    acc[j] = (W, lam, ok) over its ball (computed by the caller)."""
    nbr = r["nbr"]
    N = X.shape[0]
    centers = np.flatnonzero(r["is_center"] == 1)
    keep = lambda j, t: bool(acc[j][2][t]) if mode == O.STAB_SEQ else True
    first = np.full(N, -1)
    for j in centers:  # ascending
        for t in range(bl[j]):
            i = nbr[j, t]
            if i >= j and keep(j, t) and first[i] < 0:
                first[i] = j
    for k in range(N):
        earlier = [j for j in centers if j < k and k in nbr[j, :bl[j]] and
                   keep(j, int(np.flatnonzero(nbr[j, :bl[j]] == k)[0]))]
        assert (r["is_center"][k] == 1) == (len(earlier) == 0)
    n_fb = 0
    for i in range(N):
        j = first[i]
        assert j >= 0
        t = int(np.flatnonzero(nbr[j] == i)[0])
        W, lam, ok = acc[j]
        if mode == O.STAB_FALLBACK and not ok[t]:
            n_fb += 1
            assert r["owner"][i] == i and r["is_center"][i] == 2
            Wf, _ = O.local_weights(X, nbr[i], ell, m, X[i:i + 1])
            src_cols, src_w = nbr[i], Wf[:, 0]
        else:
            assert r["owner"][i] == j
            src_cols, src_w = nbr[j], W[:, t]
        o = np.argsort(src_cols)
        sl = slice(r["row_ptr"][i], r["row_ptr"][i + 1])
        assert np.array_equal(r["col"][sl], src_cols[o])
        assert np.array_equal(r["val"][sl], src_w[o])
    assert r["stats"]["n_fallback"] == n_fb


def _centroid_ref(X, idx):
    """Stencil position of the node nearest the centroid of the stencil (numpy mean), and the
    relative gap to the second nearest, so that a test can rule out a near tie."""
    P = X[idx]
    dd = ((P - P.mean(axis=0)) ** 2).sum(axis=1)
    o = np.argsort(dd, kind="stable")
    return int(o[0]), (dd[o[1]] - dd[o[0]]) / max(dd[o[1]], 1e-300)


@pytest.mark.parametrize("mode", [O.STAB_SEQ, O.STAB_FALLBACK])
@pytest.mark.parametrize("delta", [0.25, 0.5])
def test_centroid_reference_traversal_satisfies_its_characterisation(mode, delta):
    """§4.2.1 with the test's reference point at the stencil node nearest the stencil's
    centroid: a retained node is kept iff its Lebesgue value is <= the value at that node
    (found here with numpy, evaluated as a separate point of the same stencil); the center
    always keeps its own row; the traversal is otherwise the unique index-order assignment."""
    X = NS.disk2d(300, seed=21)
    n, ell, m = 12, 2, 3
    r = O.assemble(X, n, ell, m, delta, mode=mode, lref=O.LREF_CENTROID)
    bl = O.ball_len(r["d2"], delta)
    acc, moved = {}, 0
    for j in np.flatnonzero(r["is_center"] == 1):
        idx = r["nbr"][j]
        tref, gap = _centroid_ref(X, idx)
        assert gap > 1e-9
        moved += tref != 0
        W, lam = O.local_weights(X, idx, ell, m, X[idx[:bl[j]]])
        _, lam_ref = O.local_weights(X, idx, ell, m, X[idx[tref]][None, :])
        ok = lam <= lam_ref[0]
        ok[0] = True
        acc[j] = (W, lam, ok)
    assert moved > 0  # the two readings differ on this node set
    _check_characterisation(X, r, bl, acc, mode, ell, m)
    ref = O.assemble(X, n, ell, m, delta, mode=mode)
    assert not np.array_equal(ref["owner"], r["owner"]) or mode != O.STAB_SEQ


def test_centroid_reference_equals_center_reference_when_centroids_are_centers():
    """Nodes evenly spaced on a circle: every stencil (a node and its nearest neighbours on
    both sides) has its centroid on the center's radius, nearest to the center itself, so the
    centroid reading of the test is the center reading and the matrices agree bit for bit."""
    a = 2 * np.pi * np.arange(64) / 64
    X = np.stack([np.cos(a), np.sin(a)], axis=1)
    r0 = O.assemble(X, 5, 1, 3, 0.4)
    assert all(_centroid_ref(X, r0["nbr"][j])[0] == 0 for j in range(64))
    r1 = O.assemble(X, 5, 1, 3, 0.4, lref=O.LREF_CENTROID)
    for key in ("owner", "is_center", "col", "val", "lam_row"):
        assert np.array_equal(r0[key], r1[key]), key
    assert r0["stats"]["n_decisions"] > 0


def test_delta_one_is_standard_rbffd():
    X = NS.disk2d(400, seed=5)
    r = O.assemble(X, 12, 2, 3, 1.0)
    assert np.all(r["is_center"] == 1) and np.array_equal(r["owner"], np.arange(400))
    assert r["stats"]["n_centers"] == 400 and r["stats"]["n_decisions"] == 0


def test_delta_one_matches_a_separately_coded_standard_rbffd():
    """Every row at delta = 1 is standard RBF-FD: the Laplacian weights of the node's own
    stencil, here from a separate numpy/LAPACK construction of the local system."""
    from tests.hp_reference import lapack_weights
    X = NS.disk2d(400, seed=5)
    n, ell, m = 12, 2, 3
    r = O.assemble(X, n, ell, m, 1.0)
    for i in range(0, 400, 7):
        idx = r["nbr"][i]
        w = lapack_weights(X, idx, ell, m, X[i]).ravel()
        order = np.argsort(idx)
        sl = slice(r["row_ptr"][i], r["row_ptr"][i + 1])
        assert np.abs(r["val"][sl] - w[order]).max() <= 1e-10 * np.abs(w).max()


def test_multi_rhs_columns_equal_single_rhs_solves():
    """The overlapped solve (§4.1): each column of a multi-right-hand-side solve is the
    single-right-hand-side solve at that point, bit for bit (one factorization serves all)."""
    X = NS.disk2d(300, seed=6)
    nbr, _ = O.knn(X, 20)
    idx = nbr[17]
    Y = X[idx[:9]]
    W, lam = O.local_weights(X, idx, 3, 5, Y)
    for e in range(9):
        w1, l1 = O.local_weights(X, idx, 3, 5, Y[e:e + 1])
        assert np.array_equal(W[:, e], w1[:, 0]) and lam[e] == l1[0]


@pytest.mark.parametrize("delta", [1.0, 0.5])
def test_gershgorin_radius_is_the_local_lebesgue_value(delta):
    """§4.2: the Gershgorin radius of row i of L is its local Lebesgue value (in the units of
    L) minus the diagonal magnitude: sum_{j != i} |L_ij| = Lambda_i / rho_owner^2 - |L_ii|."""
    X = NS.disk2d(500, seed=8)
    r = O.assemble(X, 12, 2, 3, delta)
    rho2 = r["d2"][:, -1]
    for i in range(500):
        sl = slice(r["row_ptr"][i], r["row_ptr"][i + 1])
        cols, vals = r["col"][sl], r["val"][sl]
        diag = abs(vals[cols == i][0])
        g = np.abs(vals[cols != i]).sum()
        lam = r["lam_row"][i] / rho2[r["owner"][i]]
        assert abs(g - (lam - diag)) <= 1e-12 * lam


def test_stabilization_is_active_on_small_stencils():
    X = NS.disk2d(2000, seed=1)
    nbr, d2 = O.knn(X, 12)
    seq = O.assemble(X, 12, 2, 3, 0.5, O.STAB_SEQ, nbr, d2)
    off = O.assemble(X, 12, 2, 3, 0.5, O.STAB_OFF, nbr, d2)
    assert seq["stats"]["n_rejected"] > 0
    assert seq["stats"]["n_centers"] > off["stats"]["n_centers"]
    assert off["stats"]["n_centers"] < 2000


def test_power_of_two_scaling_is_exact():
    X = NS.disk2d(500, seed=12)
    a = O.assemble(X, 12, 2, 3, 0.5)
    b = O.assemble(X * 2.0, 12, 2, 3, 0.5)
    assert np.array_equal(a["owner"], b["owner"]) and np.array_equal(a["col"], b["col"])
    assert np.array_equal(a["val"], b["val"] * 4.0)


def test_translation_invariance():
    X = NS.disk2d(500, seed=13)
    a = O.assemble(X, 12, 2, 3, 0.5)
    b = O.assemble(X + np.array([0.375, -0.25]), 12, 2, 3, 0.5)
    assert np.array_equal(a["owner"], b["owner"]) and np.array_equal(a["col"], b["col"])
    for i in range(500):
        sl = slice(i * 12, (i + 1) * 12)
        assert np.abs(a["val"][sl] - b["val"][sl]).max() <= 1e-9 * np.abs(a["val"][sl]).max()


# ------------------------------------------------------------------ accuracy (§7)
def _interior_error(X, r, f, lapf, margin):
    y = O.csr_matvec(r["row_ptr"], r["col"], r["val"], f(X))
    inner = np.all((X > margin) & (X < 1 - margin), axis=1)
    return np.abs(y - lapf(X))[inner].max()


@pytest.mark.parametrize("delta,mode", [(1.0, O.STAB_SEQ), (0.5, O.STAB_SEQ)])
def test_laplacian_converges_2d(delta, mode):
    f = lambda P: np.sin(np.pi * P[:, 0]) * np.cos(np.pi * P[:, 1])
    lapf = lambda P: -2 * np.pi ** 2 * f(P)
    errs = []
    for side in (20, 40):
        X = NS.jittered_grid(side, 2, amp=0.2, seed=31)
        r = O.assemble(X, 31, 4, 7, delta, mode)
        errs.append(_interior_error(X, r, f, lapf, 0.2))
    order = math.log2(errs[0] / errs[1])
    assert order > 2.3, (errs, order)  # ell = 4: expected order about ell - 1 = 3


def test_laplacian_converges_3d():
    f = lambda P: np.sin(np.pi * P[:, 0]) * np.cos(np.pi * P[:, 1]) * np.sin(np.pi * P[:, 2])
    lapf = lambda P: -3 * np.pi ** 2 * f(P)
    errs = []
    for side in (9, 18):
        X = NS.jittered_grid(side, 3, amp=0.2, seed=32)
        r = O.assemble(X, 45, 3, 7, 0.6)
        errs.append(_interior_error(X, r, f, lapf, 0.25))
    order = math.log2(errs[0] / errs[1])
    assert order > 1.5, (errs, order)  # ell = 3: expected order about 2


# ------------------------------------------------------------------ mixed stencils
def test_mixed_oracle_with_uniform_parameters_is_the_uniform_oracle():
    X = NS.disk2d(700, seed=17)
    N = X.shape[0]
    for delta, mode in ((0.5, O.STAB_SEQ), (0.3, O.STAB_FALLBACK), (1.0, O.STAB_SEQ)):
        a = O.assemble(X, 12, 2, 3, delta, mode)
        b = O.assemble_mixed(X, np.full(N, 12), np.full(N, 2), np.full(N, 3), delta, mode)
        for key in ("row_ptr", "col", "val", "owner", "is_center", "lam_row"):
            assert np.array_equal(a[key], b[key]), key


def test_mixed_traversal_satisfies_its_characterisation():
    X = NS.cube3d_clustered(900, seed=4)
    N = X.shape[0]
    ell = np.where(X[:, 0] < 0.5, 2, 3).astype(np.int32)
    n_node = np.array([2 * math.comb(int(l) + 3, 3) + 1 for l in ell], dtype=np.int32)
    m_node = np.where(ell == 2, 5, 7).astype(np.int32)
    delta = 0.4
    r = O.assemble_mixed(X, n_node, ell, m_node, delta)
    nbr, d2 = r["nbr"], r["d2"]
    f = (1 - delta) * (1 - delta)
    bl = [int((d2[k, :n_node[k]] <= f * d2[k, n_node[k] - 1]).sum()) for k in range(N)]
    centers = np.flatnonzero(r["is_center"] == 1)
    acc = {}
    for j in centers:
        idx = nbr[j, :n_node[j]]
        W, lam = O.local_weights(X, idx, int(ell[j]), int(m_node[j]), X[idx[:bl[j]]])
        acc[j] = (W, lam <= lam[0])
    first = np.full(N, -1)
    for j in centers:
        for t in range(bl[j]):
            i = nbr[j, t]
            if i >= j and acc[j][1][t] and first[i] < 0:
                first[i] = j
    for k in range(N):
        earlier = [j for j in centers if j < k and k in nbr[j, :bl[j]]
                   and acc[j][1][int(np.flatnonzero(nbr[j, :bl[j]] == k)[0])]]
        assert (r["is_center"][k] == 1) == (len(earlier) == 0)
    for i in range(N):
        j = first[i]
        assert r["owner"][i] == j
        t = int(np.flatnonzero(nbr[j, :n_node[j]] == i)[0])
        cols = nbr[j, :n_node[j]]
        o = np.argsort(cols)
        sl = slice(r["row_ptr"][i], r["row_ptr"][i + 1])
        assert r["row_ptr"][i + 1] - r["row_ptr"][i] == n_node[j]
        assert np.array_equal(r["col"][sl], cols[o])
        assert np.array_equal(r["val"][sl], acc[j][0][o, t])


# ------------------------------------------------------------------ boundary rows (§5)
def _poly_dn_check(X, idx, ell, m, nrm, d):
    """sum_j w_j p(x_j) = grad p(x_c) . n for every monomial p = (x - x_c)^alpha, |alpha| <= ell
    (exactly: n_a for alpha = e_a, 0 otherwise)."""
    W, lam = O.normal_weights(X, idx, ell, m, nrm)
    Z = X[idx] - X[idx[0]]
    worst = 0.0
    for g in range(ell + 1):
        for al in itertools.product(range(g + 1), repeat=d):
            if sum(al) != g:
                continue
            pv = np.prod(Z ** np.array(al), axis=1)
            exact = nrm[al.index(1)] if g == 1 else 0.0
            scale = np.abs(W * pv).sum() + 1.0
            worst = max(worst, abs((W * pv).sum() - exact) / scale)
    return worst, W, lam


@pytest.mark.parametrize("d,n,ell,m", [(2, 21, 3, 5), (2, 31, 4, 7), (3, 41, 3, 7)])
def test_neumann_weights_reproduce_normal_derivatives_of_polynomials(d, n, ell, m):
    X, bc, nrm = NS.disk2d_bc(500, seed=3) if d == 2 else NS.ball3d_bc(3000, seed=4)
    nbr, _ = O.knn(X, n)
    for i in np.flatnonzero(bc)[:: max(1, int(bc.astype(bool).sum()) // 8)]:
        worst, _, _ = _poly_dn_check(X, nbr[i], ell, m, nrm[i], d)
        assert worst < 1e-9, (i, worst)


@pytest.mark.parametrize("d,n,ell,m", [(2, 12, 2, 3), (3, 20, 2, 5)])
def test_neumann_weights_match_independent_high_precision_solve(d, n, ell, m):
    X, bc, nrm = NS.disk2d_bc(300, seed=5) if d == 2 else NS.ball3d_bc(1500, seed=6)
    nbr, _ = O.knn(X, n)
    for i in np.flatnonzero(bc)[:3]:
        W, _ = O.normal_weights(X, nbr[i], ell, m, nrm[i])
        ref = _mp_weights(X, nbr[i], ell, m, X[i:i + 1], dps=40, normal=nrm[i])[:, 0]
        assert np.abs(W - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("kind", [1, 2])
def test_boundary_rows_and_interior_only_traversal(kind):
    """Boundary nodes (§5): never a center of the overlapped traversal nor a member of a
    retention set; each gets its own-stencil row (identity for Dirichlet, normal derivative
    for Neumann); the interior rows come from interior centers whose balls hold them."""
    X, bc, nrm = NS.disk2d_bc(400, seed=7)
    bc = np.where(bc > 0, kind, 0).astype(np.uint8)
    n, ell, m, delta = 12, 2, 3, 0.5
    r = O.assemble(X, n, ell, m, delta, bc=bc, normals=nrm)
    N = X.shape[0]
    nbr, d2 = r["nbr"], r["d2"]
    bl = O.ball_len(d2, delta)
    b = bc > 0
    assert r["stats"]["n_boundary"] == b.sum()
    assert np.array_equal(r["is_center"][b], np.full(b.sum(), 3))
    assert np.array_equal(r["owner"][b], np.flatnonzero(b))
    assert not np.isin(r["owner"][~b], np.flatnonzero(b)).any()
    assert np.all(np.isin(r["is_center"][~b], [0, 1]))
    for i in np.flatnonzero(~b):
        o = r["owner"][i]
        assert o <= i and i in nbr[o, :bl[o]]
    for i in np.flatnonzero(b):
        sl = slice(r["row_ptr"][i], r["row_ptr"][i + 1])
        order = np.argsort(nbr[i])
        assert np.array_equal(r["col"][sl], nbr[i][order])
        if kind == 1:
            assert np.array_equal(r["val"][sl], (nbr[i][order] == i).astype(float))
        else:
            W, _ = O.normal_weights(X, nbr[i], ell, m, nrm[i])
            assert np.array_equal(r["val"][sl], W[order])
    # without boundary nodes it is the plain construction
    r0 = O.assemble(X, n, ell, m, delta)
    r1 = O.assemble(X, n, ell, m, delta, bc=np.zeros(N, np.uint8))
    for key in ("row_ptr", "col", "val", "owner", "is_center"):
        assert np.array_equal(r0[key], r1[key])


# ------------------------------------------------------------------ cost model (§4.3, §4.4)
def test_cost_model_closed_forms():
    from paper_1606_03135_gb300 import model as Mo
    # p: the ball holds (1 - delta)^d n nodes, at least the center
    assert Mo.p_hat(1.0, 31, 2) == 1.0 and Mo.p_hat(0.5, 40, 2) == 10.0
    assert abs(Mo.p_hat(0.5, 80, 3) - 10.0) < 1e-12
    # delta from the retained fraction inverts p = t n
    for d in (2, 3):
        for t in (0.1, 0.25, 0.5, 1.0):
            delta = Mo.delta_from_retention(t, d)
            assert abs(Mo.p_hat(delta, 1000, d) - max(t * 1000, 1.0)) < 1e-9
    # eta: C at delta = 1 with gamma = 1; the cost ratio of counts reduces to it when
    # N_delta = N / q and q = p
    assert abs(Mo.eta_predicted(1.0, 31, 15, 2) - 0.4) < 1e-15
    n, M, N = 31, 15, 40000
    for delta in (0.5, 0.3):
        p = Mo.p_hat(delta, n, 2)
        assert abs(Mo.eta_from_counts(N, N / p, n, M, p) * 0.4 - Mo.eta_predicted(delta, n, M, 2)) < 1e-12
    # more retained rows per stencil: larger predicted speedup, bounded by C gamma (n + M + 1)
    e = [Mo.eta_predicted(dl, n, M, 2) for dl in (0.9, 0.7, 0.5, 0.3, 0.1)]
    assert all(a < b for a, b in zip(e, e[1:])) and e[-1] < 0.4 * (n + M + 1)
