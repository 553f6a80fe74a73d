"""Asynchronous export (rbffd_export_async): the same bytes as the synchronous export, copied on
another stream after the plan's assembly."""
import numpy as np
import pytest

from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pinned(N, nnz):
    pin = lambda size, dt: torch.empty(size, dtype=dt, pin_memory=True).numpy()
    return (pin(N + 1, torch.int64), pin(nnz, torch.int32), pin(nnz, torch.float64),
            pin(N, torch.int32))


def test_export_async_equals_export_for_several_plans():
    X = torch.from_numpy(NS.disk2d(3000, seed=4)).cuda()
    copy = torch.cuda.Stream()
    plans = [R.Plan(X, 31, 4, 7, delta, sync=False) for delta in (1.0, 0.5, 0.3)]
    for p in plans:
        p.assemble()
    outs = [_pinned(p.N, p.N * p.n) for p in plans]
    views = [p.export_async(o, copy) for p, o in zip(plans, outs)]  # before any wait
    for p, v in zip(plans, views):
        st = p.stats()  # waits for the plan's assembly and its copies
        assert st["status"] == 0
        ref = p.export()
        for a, b in zip(v, ref):
            assert np.array_equal(a, b)
        p.close()


def test_export_async_on_per_node_stencils_needs_the_counters():
    X = NS.cube3d_clustered(2000, seed=4)
    params = NS.mixed_degree_params(X, ells=(2, 3))
    with R.Plan(torch.from_numpy(X).cuda(), *params, 0.3, sync=False) as p:
        p.assemble()
        h = R._stream_handle(None)
        assert R.rbffd_export_async(p._plan, None, None, None, None, h) == R.ESTATE
        nnz = p.stats()["nnz"]
        out = _pinned(p.N, nnz)
        v = p.export_async(out, torch.cuda.current_stream())
        torch.cuda.current_stream().synchronize()
        for a, b in zip(v, p.export()):
            assert np.array_equal(a, b)


def test_export_async_argument_errors():
    assert R.rbffd_export_async(None, None, None, None, None, None) == R.EINVAL
    X = torch.from_numpy(NS.disk2d(500, seed=1)).cuda()
    with R.Plan(X, 12, 2, 3, 0.5) as p:
        assert R.rbffd_export_async(p._plan, None, None, None, None, None) == R.ESTATE
