"""rbffd_assemble captured in a CUDA graph: a replay forms the same matrix with no host work."""
import ctypes

import numpy as np
import pytest

from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _memset_device(ptr, nbytes):
    cu = ctypes.CDLL("libcuda.so.1")
    cu.cuMemsetD8_v2.argtypes = [ctypes.c_uint64, ctypes.c_ubyte, ctypes.c_size_t]
    assert cu.cuMemsetD8_v2(ptr, 0, nbytes) == 0


@pytest.mark.parametrize("mode", [R.STAB_SEQ, R.STAB_FALLBACK])
def test_graph_replay_reforms_the_matrix(mode):
    X = NS.square2d(10000, seed=5)
    with R.Plan(torch.from_numpy(X).cuda(), 31, 4, 7, 0.3, mode=mode, sync=False) as p:
        csr = p.assemble()
        torch.cuda.synchronize()
        ref = p.export()
        st0 = p.stats()
        g = p.capture_assemble()
        for _ in range(2):
            torch.cuda.synchronize()
            _memset_device(csr.val, csr.nnz * 8)    # wipe the matrix the graph must rebuild
            _memset_device(csr.col, csr.nnz * 4)
            g.replay()
            torch.cuda.synchronize()
            got = p.export()
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
            st = p.stats()
            assert st["status"] == 0 and st["n_centers"] == st0["n_centers"]


def test_graph_replay_of_a_mixed_degree_plan_with_fallback():
    """Per-node stencils in FALLBACK mode: the traversal and the per-class fallback launches
    replay from one graph and rebuild the same matrix."""
    X = NS.cube3d_clustered(3000, seed=4)
    nn, ee, mm = NS.mixed_degree_params(X)
    with R.Plan(torch.from_numpy(X).cuda(), nn, ee, mm, 0.3, mode=R.STAB_FALLBACK,
                sync=False) as p:
        csr = p.assemble()
        torch.cuda.synchronize()
        ref = p.export()
        g = p.capture_assemble()
        torch.cuda.synchronize()
        _memset_device(csr.val, int(ref[0][-1]) * 8)
        g.replay()
        torch.cuda.synchronize()
        got = p.export()
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
        assert p.stats()["status"] == 0


def test_one_graph_assembles_plans_of_different_dimension_and_degree():
    """A 2D plan, a 3D plan, a per-node mixed-degree plan with fallback and a degree-5 2D plan
    captured together into one CUDA graph (each on its own stream: their kernels run side by
    side); every replay rebuilds each plan's matrix bit for bit as assembled alone."""
    setups = [
        (NS.square2d(10000, seed=5), (31, 4, 7), 0.3, R.STAB_SEQ),
        (NS.ball3d(10000, seed=3), (45, 3, 7), 0.4, R.STAB_SEQ),
        (NS.cube3d_clustered(3000, seed=4), None, 0.3, R.STAB_FALLBACK),
        (NS.disk2d(4000, seed=9), (43, 5, 7), 0.5, R.STAB_SEQ),
    ]
    solo, plans, csrs = [], [], []
    for X, params, delta, mode in setups:
        params = params if params is not None else NS.mixed_degree_params(X)
        Xd = torch.from_numpy(X).cuda()
        with R.Plan(Xd, *params, delta, mode=mode) as p:
            p.assemble()
            solo.append(p.export())
        p = R.Plan(Xd, *params, delta, mode=mode, sync=False, max_ctas=300)
        csrs.append(p.assemble())
        plans.append(p)
    torch.cuda.synchronize()
    g = R.capture_assemble_batch(plans)
    for _ in range(2):
        torch.cuda.synchronize()
        for p, csr, ref in zip(plans, csrs, solo):
            _memset_device(csr.val, int(ref[0][-1]) * 8)
        g.replay()
        torch.cuda.synchronize()
        for p, ref in zip(plans, solo):
            got = p.export()
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
            assert p.stats()["status"] == 0
    for p in plans:
        p.close()
