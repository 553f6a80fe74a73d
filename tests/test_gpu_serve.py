"""Continuous batching on the GPU: each served job's matrix is the oracle's, and the same alone
and in the mix."""
import os

import numpy as np
import pytest

from paper_1606_03135_gb300 import serve as S
from tests import oracle_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


def test_served_jobs_match_the_oracle_and_are_the_same_alone_and_in_the_mix():
    from paper_1606_03135_gb300 import rbffd as R
    from tests.test_gpu_parity import check_mixed_rows
    jobs = S.serving_jobs(count=12, seed=11, n_min=2000, n_max=20000)
    with oracle_pool.pool(min(8, os.cpu_count() or 1)) as pool:
        pending = pool.map_async(oracle_pool.assemble_job,
                                 [(j.nodes, j.n, j.ell, j.m, j.delta) for j in jobs])
        for j in jobs:
            j.arrival = 0.0  # all at once: the scheduler must overlap them
        mixed, summ = S.Server(slots=4, budget_bytes=8 << 30).run(jobs)
        assert summ["failed"] == 0, [r.error for r in mixed]
        alone, _ = S.Server(slots=1).run(jobs)
        refs = pending.get(timeout=900)
    assert summ["peak_reserved_bytes"] <= 8 << 30
    for job, a, b, ref in zip(jobs, mixed, alone, refs):
        assert a.rid == b.rid == job.rid
        for x, y in ((a.row_ptr, b.row_ptr), (a.col, b.col), (a.val, b.val),
                     (a.owner, b.owner)):
            assert np.array_equal(x, y)
        # the oracle: structure bit-exact, weights within 1e-9 of the row's largest weight; the
        # ill-conditioned degree-5 (and 3D degree-4) stencils have rows above 1e-9, which are
        # measured against a double-double solve (the bar of check_mixed_rows)
        assert ref["n_near_tie"] == 0
        assert np.array_equal(a.owner, ref["owner"]), job.rid
        assert np.array_equal(a.row_ptr, ref["row_ptr"]) and np.array_equal(a.col, ref["col"])
        N, d = job.nodes.shape
        n = job.n
        errs = np.abs(a.val - ref["val"]).reshape(N, n).max(1) / \
            np.abs(ref["val"]).reshape(N, n).max(1)
        if errs.max() > TOL:
            full = lambda v: np.full(N, v, dtype=np.int32)
            check_mixed_rows(job.nodes, dict(val=a.val), ref, full(n), full(job.ell),
                             full(job.m), per_class=10, max_bad=40, min_rows=10)


def test_estimated_job_memory_bounds_the_exact_size():
    """The admission reservation (taken before a job allocates) is an upper bound of the
    device memory the plan reports, over the serving mix's shapes."""
    from paper_1606_03135_gb300 import rbffd as R
    for job in S.serving_jobs(count=24, seed=13, n_min=1000, n_max=30000):
        N, d = job.nodes.shape
        with R.Plan(job.nodes, job.n, job.ell, job.m, job.delta) as p:
            st = p.stats()
        est = S.estimate_bytes(N, d, job.n, job.delta, ell=job.ell)
        assert est >= st["plan_bytes"] + st["assemble_bytes"], (job.rid, est, st)


def test_large_polynomial_degree_in_3d_fits():
    # ell = 5 in 3D: M = 56, n = 113, K = 169 (the packed symmetric layout fits in one CTA)
    from oracle import oracle as O
    from paper_1606_03135_gb300 import nodesets as NS
    from paper_1606_03135_gb300 import rbffd as R
    from tests.test_gpu_parity import check_mixed_rows
    X = NS.ball3d(1500, seed=7)
    with R.Plan(torch.from_numpy(X).cuda(), 113, 5, 7, 0.4) as p:
        p.assemble()
        row_ptr, col, val, owner = p.export()
    ref = O.assemble(X, 113, 5, 7, 0.4)
    assert np.array_equal(owner, ref["owner"]) and np.array_equal(col, ref["col"])
    full = lambda v: np.full(X.shape[0], v, dtype=np.int32)
    check_mixed_rows(X, dict(val=val), ref, full(113), full(5), full(7), per_class=40,
                     max_bad=60, min_rows=40)
