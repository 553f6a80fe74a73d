"""The schedule autotuner: every candidate schedule forms the same matrix; the pick is one of
the timed candidates."""
import numpy as np
import pytest

from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_picks_a_timed_schedule_and_schedules_agree():
    X = torch.from_numpy(NS.square2d(10000, seed=5)).cuda()
    best, timings = R.autotune(X, 31, 4, 7, 0.5)
    assert tuple(sorted(best.items())) in timings and len(timings) >= 3
    mats = []
    for cand in ({}, best, dict(team=512, max_ctas=300)):
        with R.Plan(X, 31, 4, 7, 0.5, **cand) as p:
            p.assemble()
            mats.append(p.export())
    for other in mats[1:]:
        for a, b in zip(mats[0], other):
            assert np.array_equal(a, b)
