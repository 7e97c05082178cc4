"""Host-side bookkeeping of bench.py that needs no GPU."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _p(ndim):
    return types.SimpleNamespace(ndim=ndim)


def _i(ms, team):
    return types.SimpleNamespace(ms=ms, team_size=team)


def test_solve_ms_shared_launch():
    # a team launch: every pair reports the launch's time once
    assert bench.solve_ms([_p(1)] * 3, [_i(5.0, 76), _i(5.0, 76), _i(5.0, 76)]) == 5.0
    # a grid launch (2D and 3D report team size 0 but share one launch)
    assert bench.solve_ms([_p(2), _p(3)], [_i(7.5, 0), _i(7.5, 0)]) == 7.5


def test_solve_ms_streamed_pairs_share_their_solve():
    # 1D pairs streamed through device memory (team size 0) share the launches
    # of one streamed solve, which report its time
    assert bench.solve_ms([_p(1)] * 4, [_i(9.0, 0)] * 4) == 9.0
    # a mixed call: the team launch, then the streamed pairs
    assert bench.solve_ms([_p(1), _p(1), _p(1)], [_i(4.0, 8), _i(4.0, 8), _i(6.0, 0)]) == 10.0


def test_workload_table_is_consistent():
    for k, W in bench.WORKLOADS.items():
        assert k in bench.GENERATORS
        assert W["variant"] in ("log", "plain", "paper") and W["precision"] in ("fp32", "fp64")
        assert W["bytes_per_nit"] in (28.0, 56.0)


def test_cpu_sample_uses_every_core():
    # one pair per host thread on every core, never more threads than pairs
    W2 = bench.WORKLOADS[2]
    assert bench.cpu_sample_threads(W2, 16) == 16
    assert bench.cpu_sample_threads(W2, 500) == W2["pairs"]
    assert bench.cpu_sample_threads(bench.WORKLOADS[1], 16) == 1
