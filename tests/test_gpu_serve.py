"""Continuous batching on the GPU: each job's matrix is the same alone and in the mix."""
import numpy as np
import pytest

from paper_1606_03135_gb300 import serve as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    jobs = S.serving_jobs(count=12, seed=11, n_min=2000, n_max=20000)
    for j in jobs:
        j.arrival = 0.0  # all at once: the scheduler must overlap them
    mixed, summ = S.Server(slots=4, budget_bytes=8 << 30).run(jobs)
    assert summ["failed"] == 0, [r.error for r in mixed]
    alone, _ = S.Server(slots=1).run(jobs)
    for a, b in zip(mixed, alone):
        assert a.rid == b.rid
        for x, y in ((a.row_ptr, b.row_ptr), (a.col, b.col), (a.val, b.val),
                     (a.owner, b.owner)):
            assert np.array_equal(x, y)
    assert summ["peak_reserved_bytes"] <= 8 << 30


def test_large_polynomial_degree_in_3d_fits():
    # ell = 5 in 3D: M = 56, n = 113, K = 169 (the packed symmetric layout fits in one CTA)
    from oracle import oracle as O
    from paper_1606_03135_gb300 import nodesets as NS
    from paper_1606_03135_gb300 import rbffd as R
    X = NS.ball3d(1500, seed=7)
    with R.Plan(torch.from_numpy(X).cuda(), 113, 5, 7, 0.4) as p:
        p.assemble()
        row_ptr, col, val, owner = p.export()
    ref = O.assemble(X, 113, 5, 7, 0.4)
    assert np.array_equal(owner, ref["owner"]) and np.array_equal(col, ref["col"])
    n = 113
    for i in range(0, 1500, 7):
        a, b = val[i * n:(i + 1) * n], ref["val"][i * n:(i + 1) * n]
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
