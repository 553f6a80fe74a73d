"""Boundary rows (§5) on the GPU against the oracle: the overlapped traversal over the
interior only, own-stencil rows for the boundary nodes (identity for Dirichlet, normal
derivative for Neumann), and the time-stepping matrix on L's pattern."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R
from tests.test_gpu_parity import check_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


def run_bc(X, bc, nrm, n, ell, m, delta, mode=R.STAB_SEQ, **kw):
    with R.Plan(torch.from_numpy(X).cuda(), n, ell, m, delta, mode=mode, **kw) as p:
        p.set_boundary(bc, nrm)
        p.assemble()
        row_ptr, col, val, owner = p.export()
        lam, isc = p.export_lambda()
        st = p.stats()
    return dict(row_ptr=row_ptr, col=col, val=val, owner=owner, lam_row=lam, is_center=isc,
                stats=st)


def compare_bc(X, bc, nrm, n, ell, m, delta, mode=R.STAB_SEQ, **kw):
    g = run_bc(X, bc, nrm, n, ell, m, delta, mode, **kw)
    ref = O.assemble(X, n, ell, m, delta, mode, bc=bc, normals=nrm,
                     lref=kw.get("lebesgue_ref", O.LREF_CENTER))
    assert ref["stats"]["n_near_tie"] == 0
    assert np.array_equal(g["owner"], ref["owner"])
    assert np.array_equal(g["is_center"], ref["is_center"])
    assert np.array_equal(g["row_ptr"], ref["row_ptr"])
    assert np.array_equal(g["col"], ref["col"])
    check_rows(g, ref, n)
    np.testing.assert_allclose(g["lam_row"], ref["lam_row"], rtol=TOL, atol=0)
    assert g["stats"]["n_boundary"] == ref["stats"]["n_boundary"] == int((bc > 0).sum())
    assert g["stats"]["n_centers"] == ref["stats"]["n_centers"]
    assert g["stats"]["status"] == 0
    return g, ref


@pytest.mark.parametrize("n,ell,m,delta", [(12, 2, 3, 1.0), (12, 2, 3, 0.5), (31, 4, 7, 0.5)])
def test_neumann_disk_matches_the_oracle(n, ell, m, delta):
    X, bc, nrm = NS.disk2d_bc(3000, seed=1)
    g, ref = compare_bc(X, bc, nrm, n, ell, m, delta)
    assert (g["is_center"] == 3).sum() == (bc > 0).sum()


def test_dirichlet_ball_matches_the_oracle():
    X, bc, nrm = NS.ball3d_bc(4000, seed=3)
    g, _ = compare_bc(X, bc, nrm, 20, 2, 5, 0.3)
    b = np.flatnonzero(bc)
    for i in b[:50]:
        sl = slice(g["row_ptr"][i], g["row_ptr"][i + 1])
        assert np.array_equal(g["val"][sl], (g["col"][sl] == i).astype(float))


def test_boundary_with_fallback_mode():
    X, bc, nrm = NS.disk2d_bc(2000, seed=4)
    compare_bc(X, bc, nrm, 12, 2, 3, 0.3, mode=R.STAB_FALLBACK)


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_boundary_with_right_hand_sides_in_chunks(mode):
    """Chunks of 3 columns: the oracle's rows, and the same bits as one chunk."""
    X, bc, nrm = NS.disk2d_bc(2000, seed=4)
    g, _ = compare_bc(X, bc, nrm, 21, 3, 5, 0.3, mode=mode, rhs_chunk=3)
    assert g["stats"]["rhs_chunk"] == 3
    h = run_bc(X, bc, nrm, 21, 3, 5, 0.3, mode)
    assert np.array_equal(g["val"], h["val"]) and np.array_equal(g["lam_row"], h["lam_row"])


def test_timestep_matrix_and_clearing_the_boundary():
    X, bc, nrm = NS.disk2d_bc(2000, seed=2)
    c = 12.0 / 25.0 * 1.0 * 1e-3  # BDF4, nu = 1, dt = 1e-3
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5) as p:
        p.set_boundary(bc, nrm)
        p.assemble()
        row_ptr, col, val, _ = p.export()
        A = p.timestep_matrix(c).cpu().numpy()
        rows = np.repeat(np.arange(X.shape[0]), np.diff(row_ptr))
        interior = bc[rows] == 0
        cv = c * val
        want = np.where(interior, np.where(col == rows, 1.0 - cv, -cv), val)
        assert np.array_equal(A, want)
        # removing the boundary gives the plain matrix again
        p.set_boundary(None)
        p.assemble()
        plain = p.export()
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5) as q:
        q.assemble()
        for a, b in zip(plain, q.export()):
            assert np.array_equal(a, b)


def test_boundary_argument_errors():
    X, bc, nrm = NS.disk2d_bc(500, seed=2)
    with R.Plan(torch.from_numpy(X).cuda(), 12, 2, 3, 0.5) as p:
        bad = bc.copy()
        bad[0] = 5
        with pytest.raises(R.RbffdError):
            p.set_boundary(bad, nrm)
        with pytest.raises(R.RbffdError):
            p.set_boundary(bc, None)  # Neumann nodes need normals
        with pytest.raises(R.RbffdError):
            p.timestep_matrix(0.1, out=torch.empty(10, dtype=torch.float64, device="cuda"))


def test_boundary_with_the_centroid_reference():
    """Stencils next to the boundary have their centroids shifted inwards: the reference node
    is often not the center, and may be a boundary node (solved as a reference only)."""
    X, bc, nrm = NS.disk2d_bc(2000, seed=4)
    compare_bc(X, bc, nrm, 21, 3, 5, 0.3, lebesgue_ref=R.LREF_CENTROID)
