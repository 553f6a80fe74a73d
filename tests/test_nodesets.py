"""The seeded input recipes (CPU): the counter-based splitmix64 stream against its published
test vectors, Halton radical inverses against closed forms, and each node set against the
recipe it states (domain, count, jitter bound, boundary layout, determinism)."""
import math

import numpy as np

from paper_1606_03135_gb300 import nodesets as NS


def test_splitmix64_matches_published_vectors():
    # the reference splitmix64 seeded with 0 and with 1234567 (state += golden gamma, then
    # the two multiply-xorshift rounds)
    assert [int(v) for v in NS.splitmix64(0, 5)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
        0x1B39896A51A8749B]
    assert [int(v) for v in NS.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]
    # counter-based: an offset continues the same stream
    a = NS.splitmix64(99, 10)
    assert np.array_equal(NS.splitmix64(99, 4, offset=6), a[6:])


def test_uniform_is_on_the_53_bit_grid_in_the_unit_interval():
    u = NS.uniform(5, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 0.01


def test_halton_radical_inverse_closed_forms():
    np.testing.assert_array_equal(NS.halton(np.arange(1, 8), 2),
                                  [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875])
    np.testing.assert_allclose(NS.halton(np.arange(1, 6), 3),
                               [1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9], rtol=1e-15)
    np.testing.assert_allclose(NS.halton(np.array([1, 5, 6]), 5), [0.2, 0.04, 0.24], rtol=1e-15)


def test_permutation_is_a_seeded_permutation():
    p = NS.permutation(3, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000))
    assert np.array_equal(p, NS.permutation(3, 1000))
    assert not np.array_equal(p, NS.permutation(4, 1000))


def test_square2d_is_a_jittered_cell_centred_grid_in_seeded_order():
    N, side = 40000, 200
    h = 1.0 / side
    X = NS.square2d(N, seed=2)
    R = NS.square2d(N, seed=2, order="raster")
    assert X.shape == (N, 2)
    # each raster point within 0.25 h of its own cell centre
    g = (np.arange(side) + 0.5) * h
    cy, cx = np.meshgrid(g, g, indexing="ij")
    centre = np.stack([cx.ravel(), cy.ravel()], axis=1)
    assert np.abs(R - centre).max() <= 0.25 * h * (1 + 1e-12)
    # the random order holds the same points
    assert np.array_equal(np.sort(X, axis=0), np.sort(R, axis=0))
    assert not np.array_equal(X, R)


def test_disk_and_ball_are_inside_their_domains_without_duplicates():
    D = NS.disk2d(3000, seed=1)
    assert D.shape == (3000, 2) and np.all((D ** 2).sum(axis=1) <= 1.0)
    B = NS.ball3d(4000, seed=3)
    assert B.shape == (4000, 3) and np.all((B ** 2).sum(axis=1) <= 1.0)
    for P in (D, B):
        assert np.unique(P, axis=0).shape[0] == P.shape[0]
    assert np.array_equal(NS.disk2d(3000, seed=1), D)
    assert not np.array_equal(NS.disk2d(3000, seed=2), D)


def test_clustered_cube_mixes_background_and_clusters():
    N = 20000
    P = NS.cube3d_clustered(N, seed=4)
    assert P.shape == (N, 3) and P.min() >= 0.0 and P.max() < 1.0
    # density contrast: the densest of 1000 equal cells holds far more than the average
    cells = np.minimum((P * 10).astype(int), 9)
    counts = np.bincount(cells[:, 0] * 100 + cells[:, 1] * 10 + cells[:, 2], minlength=1000)
    assert counts.max() > 8 * counts.mean()


def test_disk_with_neumann_boundary_follows_its_recipe():
    N_int = 2000
    X, bc, nrm = NS.disk2d_bc(N_int, seed=1)
    h = math.sqrt(math.pi / N_int)
    Nb = int(round(2 * math.pi / h))
    r = np.sqrt((X ** 2).sum(axis=1))
    assert (bc == 2).sum() == Nb and set(np.unique(bc)) == {0, 2}
    assert np.abs(r[bc == 2] - 1.0).max() <= 1e-15
    assert np.array_equal(nrm[bc == 2], X[bc == 2]) and not nrm[bc == 0].any()
    interior, layer = X[:N_int], X[N_int:N_int + Nb]
    assert np.all(np.sqrt((interior ** 2).sum(axis=1)) <= 1.0 - h)
    np.testing.assert_allclose(np.sqrt((layer ** 2).sum(axis=1)), 1.0 - 0.5 * h, rtol=1e-14)
    # evenly spaced on the circle
    th = np.sort(np.arctan2(X[bc == 2, 1], X[bc == 2, 0]))
    np.testing.assert_allclose(np.diff(th), 2 * math.pi / Nb, rtol=1e-9)


def test_ball_with_dirichlet_boundary_follows_its_recipe():
    N_int = 4000
    X, bc, nrm = NS.ball3d_bc(N_int, seed=3)
    h = (4 * math.pi / 3 / N_int) ** (1 / 3)
    Nb = int(round(4 * math.pi / h ** 2))
    assert (bc == 1).sum() == Nb
    r = np.sqrt((X ** 2).sum(axis=1))
    assert np.abs(r[bc == 1] - 1.0).max() <= 1e-15
    assert np.all(r[bc == 0] <= 1.0 - h)
    assert np.array_equal(nrm[bc == 1], X[bc == 1])
