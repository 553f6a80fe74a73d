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
