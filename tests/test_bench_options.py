"""Host logic of bench.py's block-shape step and sweep-point selection (no
GPU): the autotuner's record, the fixed shapes, and the --sweep-points
parser."""
import sys

import pytest

import bench


class _FakeBatch:
    """Records the calls bench makes on a TacBatch."""

    def __init__(self, tuned=256, ms=(3.0, 4.0)):
        self.calls = []
        self._tuned, self._ms = tuned, ms

    def autotune_block_shape(self, poses, reps=1):
        self.calls.append(("autotune", reps))
        return self._tuned, list(self._ms)

    def set_block_shape(self, threads):
        self.calls.append(("set", threads))


def test_auto_runs_the_library_tuner_once_and_reports_both_times():
    b = _FakeBatch(tuned=512, ms=(2.7, 2.3))
    rec = bench.choose_block_shape(b, poses_next=None, mode="auto")
    assert b.calls == [("autotune", 1)]
    assert rec["threads"] == 512
    assert rec["tuning_ms"] == {"256": 2.7, "512": 2.3}
    assert "tac_autotune_block_shape" in rec["chosen_by"]


@pytest.mark.parametrize("mode", ["256", "512"])
def test_fixed_shape_is_set_without_tuning(mode):
    b = _FakeBatch()
    rec = bench.choose_block_shape(b, poses_next=None, mode=mode)
    assert b.calls == [("set", int(mode))]
    assert rec == {"threads": int(mode), "chosen_by": "--block-shape"}


def test_defaults_and_sweep_points(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.steps, a.warmup, a.envs, a.block_shape, a.sweep_points) == (20, 5, 4096, "auto", "")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--sweep", "--sweep-points", "64x50000,1024x2000"])
    a = bench.parse()
    pts = bench.sweep_points(a)
    assert pts == ((64, 50000), (1024, 2000))
    assert set(pts) <= set(bench.SWEEP_POINTS)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--sweep"])
    assert bench.sweep_points(bench.parse()) == bench.SWEEP_POINTS
