"""The allocation-free stencil entry point gives what the allocating one gives.

rbffd_stencils_noalloc serves callers that cannot allocate device memory while they run (a
solver that has handed all device memory to its own pool, a loop with a fixed time budget).
It works in one fixed array of the library's device memory that every call reuses, so two
calls in a row with different node sets must each match rbffd_plan's stencils exactly: no
contents of the previous call may leak into the next.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_NODES = 32768  # RBFFD_NOALLOC_MAX_NODES in include/rbffd.h


def _with_plan(X, n, ell, m, delta):
    with R.Plan(torch.from_numpy(X).cuda(), n, ell, m, delta) as p:
        return p.export_stencils()


def _noalloc(X, n, delta):
    N, d = X.shape
    nodes = torch.from_numpy(X).cuda()
    nbr = torch.full((N, n), -7, dtype=torch.int32, device="cuda")
    rho2 = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    bl = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = R.rbffd_stencils_noalloc(nodes, N, d, n, delta, nbr, rho2, bl,
                                  R.C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, nbr.cpu().numpy(), rho2.cpu().numpy(), bl.cpu().numpy()


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    cases = [
        (NS.jittered_grid(32, 3, seed=3), 20, 2, 5, 0.5),    # 32768 nodes: the capacity, 3D
        (NS.jittered_grid(18, 3, seed=11), 45, 3, 7, 0.2),   # 5832 nodes, 3D
        (NS.disk2d(3000, seed=4), 12, 2, 3, 0.5),            # then a smaller 2D set
    ]
    for X, n, ell, m, delta in cases:
        rc, nbr, rho2, bl = _noalloc(X, n, delta)
        assert rc == R.OK, R.rbffd_strerror(rc)
        nbr_p, rho2_p, bl_p = _with_plan(X, n, ell, m, delta)
        assert np.array_equal(nbr, nbr_p)      # integer outputs: bit-exact
        assert np.array_equal(rho2, rho2_p)    # squared distances: bit-exact
        assert np.array_equal(bl, bl_p)


def test_noalloc_rejects_sizes_beyond_its_capacity():
    X = NS.jittered_grid(182, 2, seed=2)  # 33124 > MAX_NODES
    assert X.shape[0] > MAX_NODES
    rc, nbr, _, _ = _noalloc(X, 12, 0.5)
    assert rc == R.EINVAL
    assert np.all(nbr == -7)  # nothing written


def test_a_failing_call_leaves_no_error_for_the_next_one():
    """A call on a node set with two coincident nodes returns RBFFD_EDUPLICATE (as rbffd_plan
    does); the next call on a clean node set returns OK and matches rbffd_plan bit for bit, so
    the error status kept in the shared array does not leak into it."""
    X = NS.disk2d(3000, seed=4)
    bad = X.copy()
    bad[100] = bad[17]
    rc, _, _, _ = _noalloc(bad, 12, 0.5)
    assert rc == R.EDUPLICATE
    rc, nbr, rho2, bl = _noalloc(X, 12, 0.5)
    assert rc == R.OK, R.rbffd_strerror(rc)
    nbr_p, rho2_p, bl_p = _with_plan(X, 12, 2, 3, 0.5)
    assert np.array_equal(nbr, nbr_p) and np.array_equal(rho2, rho2_p) and np.array_equal(bl, bl_p)
