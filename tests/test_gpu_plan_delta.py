"""rbffd_plan_delta: a plan for another delta built from an existing plan's stencils equals a
plan built from scratch, bit for bit (§4.1: the kNN stencils and widths do not depend on
delta; only the retention balls do)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("row_ptr", "col", "val", "owner", "nbr", "rho2", "ball_len", "lam_row", "is_center")


def run(p):
    p.assemble()
    row_ptr, col, val, owner = p.export()
    nbr, rho2, bl = p.export_stencils()
    lam, isc = p.export_lambda()
    st = p.stats()
    return dict(row_ptr=row_ptr, col=col, val=val, owner=owner, nbr=nbr, rho2=rho2, ball_len=bl,
                lam_row=lam, is_center=isc, stats=st)


def same(a, b):
    for key in KEYS:
        assert np.array_equal(a[key], b[key]), key
    for key in ("max_ball", "n_centers", "n_fallback", "nnz"):
        assert a["stats"][key] == b["stats"][key], key


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_plans_for_other_deltas_equal_fresh_plans(case):
    if case == "2d":
        X, n, ell, m = NS.disk2d(3000, seed=4), 31, 4, 7
    else:
        X, n, ell, m = NS.ball3d(3000, seed=5), 45, 3, 7
    Xd = torch.from_numpy(X).cuda()
    with R.Plan(Xd, n, ell, m, 1.0) as base:
        for delta, kw in ((0.5, {}), (0.3, dict(mode=R.STAB_FALLBACK)), (0.2, dict(team=32)),
                          (1.0, {}), (0.5, dict(factor=R.FACTOR_LU)),
                          (0.3, dict(lebesgue_ref=R.LREF_CENTROID))):
            with base.with_delta(delta, **kw) as q:
                a = run(q)
            with R.Plan(Xd, n, ell, m, delta, **kw) as f:
                b = run(f)
            same(a, b)


def test_a_derived_plan_outlives_its_base_and_matches_the_oracle():
    from tests.test_gpu_parity import check_rows
    X = NS.disk2d(2000, seed=6)
    Xd = torch.from_numpy(X).cuda()
    base = R.Plan(Xd, 21, 3, 5, 0.3)
    q = base.with_delta(0.5)
    base.close()
    with q:
        g = run(q)
    ref = O.assemble(X, 21, 3, 5, 0.5)
    assert ref["stats"]["n_near_tie"] == 0
    assert np.array_equal(g["rho2"], ref["d2"][:, -1])
    assert np.array_equal(g["ball_len"], O.ball_len(ref["d2"], 0.5))
    for key in ("nbr", "owner", "is_center", "row_ptr", "col"):
        assert np.array_equal(g[key], ref[key]), key
    check_rows(g, ref, 21)


def test_per_node_plans_for_other_deltas_equal_fresh_plans():
    X = NS.cube3d_clustered(3000, seed=4)
    params = NS.mixed_degree_params(X)
    Xd = torch.from_numpy(X).cuda()
    with R.Plan(Xd, *params, 1.0) as base:
        with base.with_delta(0.3, mode=R.STAB_FALLBACK) as q:
            a = run(q)
    with R.Plan(Xd, *params, 0.3, mode=R.STAB_FALLBACK) as f:
        b = run(f)
    same(a, b)


def test_invalid_arguments_leave_no_plan():
    X = torch.from_numpy(NS.disk2d(2000, seed=6)).cuda()
    with R.Plan(X, 21, 3, 5, 1.0) as base:
        for delta in (0.0, -0.5, 1.5, float("nan")):
            rc, out = R.rbffd_plan_delta(base._plan, delta)
            assert rc == R.EINVAL and not out.value, delta
        bad = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LDLT, 0, 48)  # no such team
        rc, out = R.rbffd_plan_delta(base._plan, 0.5, bad)
        assert rc == R.EINVAL and not out.value
        with pytest.raises(R.RbffdError):
            base.with_delta(2.0)
        # the base plan is untouched and still assembles
        base.assemble()
        assert base.stats()["status"] == 0


def test_a_base_built_from_host_nodes_gives_the_same_derived_plans():
    X = NS.disk2d(3000, seed=4)
    with R.Plan(X, 31, 4, 7, 1.0) as base:  # nodes copied from host memory
        with base.with_delta(0.4) as q:
            a = run(q)
    with R.Plan(torch.from_numpy(X).cuda(), 31, 4, 7, 0.4) as f:
        b = run(f)
    same(a, b)
