"""Host-side pieces of the benchmark: the operator's algorithmic bytes per unit,
the traffic figure's scope, and the oracle windows."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2101_12408_gb300 import scenes  # noqa: E402


class _FakeCtx:
    """Counts as a context reports them: one scene, particles with phases, samples, grid masses."""

    def __init__(self, phases, n_surface, masses):
        self.scenes = [None]
        self.np = [len(phases)]
        self.ns = [n_surface]
        self._phases = np.asarray(phases, np.uint8)
        self._masses = np.asarray(masses, float)

    def get_particles(self, k):
        return {"phase": self._phases}

    def get_grid(self, k, field):
        return self._masses


def test_algorithmic_bytes_per_unit():
    # 3 liquid particles (4 values), 2 solid (48), 5 samples (48), 4 active nodes of 6 (6 values)
    ctx = _FakeCtx([0, 0, 0, 1, 1], 5, [1.0, 2.0, 0.0, 3.0, 4.0, 0.0])
    b, counts = bench.algorithmic_bytes(ctx, 4)
    assert counts == dict(liquid=3, solid=2, surface=5, active_nodes=4)
    assert b == 4 * (3 * 4 + 2 * 48 + 5 * 48 + 4 * 6)
    b8, _ = bench.algorithmic_bytes(ctx, 8)
    assert b8 == 2 * b


def test_traffic_is_reported_only_for_the_captured_workload():
    assert bench.measured_traffic("film", 40) is None
    assert bench.measured_traffic("incline", 20) is None
    v = bench.measured_traffic("incline", 40)
    # reported only while the operator's source regions hash to the recorded value
    match = bench.NCU_TRAFFIC["source_sha256"] == bench.operator_source_hash()
    assert v == (bench.NCU_TRAFFIC["bytes_per_apply"] if match else None)


def test_oracle_windows_hold_whole_cells_of_the_workload():
    sc = scenes.droplet()
    wins = bench.sample_windows(sc, 2)
    assert len(wins) == 2
    for w in wins:
        assert w.dx == sc.dx
        assert 0 < w.n_particles < sc.n_particles
