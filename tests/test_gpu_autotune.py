"""Stencil schedules: warp-per-stencil (32 threads) and 64-, 96-, 128- and 512-thread teams all
reproduce the oracle, including balls with more solved columns than a team has threads, and
the autotuner's pick is one of the timed schedules."""
import numpy as np
import pytest

from paper_1606_03135_gb300 import nodesets as NS
from paper_1606_03135_gb300 import rbffd as R
from tests.test_gpu_parity import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("team", [32, 64, 96, 128, 512])
def test_team_size_2d_matches_the_oracle(team):
    X = NS.square2d(10000, seed=2)
    compare(X, 31, 4, 7, 0.5, team=team)


@pytest.mark.parametrize("team", [32, 64, 96, 512])
def test_team_size_with_more_columns_than_threads(team):
    # n = 80 at delta = 0.05: retention balls of ~70 members, more than 32 or 64 threads
    X = NS.jittered_grid(40, 2, seed=11)
    g, ref = compare(X, 80, 2, 3, 0.05, team=team)
    assert g["stats"]["max_ball"] > 64


@pytest.mark.parametrize("team", [32, 64, 96])
def test_team_size_3d_matches_the_oracle(team):
    X = NS.jittered_grid(9, 3, seed=9)
    compare(X, 45, 3, 7, 0.3, team=team)


def test_autotune_picks_a_timed_schedule_and_schedules_agree():
    X = torch.from_numpy(NS.square2d(10000, seed=5)).cuda()
    best, timings = R.autotune(X, 31, 4, 7, 0.5)
    assert tuple(sorted(best.items())) in timings and len(timings) >= 4
    mats = []
    for cand in ({}, best, dict(team=32), dict(team=512, max_ctas=300)):
        with R.Plan(X, 31, 4, 7, 0.5, **cand) as p:
            p.assemble()
            mats.append(p.export())
    for other in mats[1:]:
        for a, b in zip(mats[0], other):
            assert np.array_equal(a, b)
