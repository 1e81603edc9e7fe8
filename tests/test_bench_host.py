"""Host-side helpers of the benchmark (no GPU): the summary of timed windows, the parsing
of a NUMA node's CPU list, and the time step of the plane-wave workload (the sampled speed
times 1.1, below the field's analytic bound)."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_0905_3409_gb300 import inputs  # noqa: E402


def test_window_summary():
    s = bench.window_summary([2.0, 1.0, 4.0, 3.0])
    assert s == {"count": 4, "median_ms": 2.5, "min_ms": 1.0, "max_ms": 4.0, "timed_s": 0.01}


def test_node_cpus_parses_sysfs_lists(tmp_path, monkeypatch):
    import builtins
    real_open = builtins.open

    def fake_open(path, *a, **k):
        if str(path).startswith("/sys/devices/system/node/node7/cpulist"):
            p = tmp_path / "cpulist"
            p.write_text("0-3,8,10-11\n")
            return real_open(p, *a, **k)
        return real_open(path, *a, **k)

    monkeypatch.setattr(builtins, "open", fake_open)
    assert bench.node_cpus(7) == {0, 1, 2, 3, 8, 10, 11}
    assert bench.node_cpus(99999) is None


def test_waves_workload_time_step():
    wl = bench.WORKLOADS["waves2048"]
    modes = bench.wl_modes(wl)
    assert modes.shape == (256, 6)
    dt = bench.wl_dt(wl)
    h = 1.0 / (wl["n"][0] - 1)
    vs = inputs.wave_speed_sampled(modes)
    assert dt == pytest.approx(h / vs)
    # the sampled speed is a real maximum of the field (here at a few points and times)
    rng = np.random.default_rng(2)
    for _ in range(4):
        x, y, t = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50), rng.uniform(0, 1)
        u, v = inputs.wave_velocity(modes, x, y, t)
        assert max(np.max(np.abs(u)), np.max(np.abs(v))) <= vs
    assert vs <= 1.1 * inputs.wave_speed_bound(modes)


def test_wave_modes_statistics():
    m = inputs.wave_modes(4096, seed=1)
    k = np.hypot(m[:, 1], m[:, 2])
    assert k.min() >= math.pi and k.max() <= 4 * math.pi
    assert abs(np.std(m[:, 0]) * math.sqrt(4096) - 0.4) < 0.03
    assert set(np.unique(m[:, 4])) <= {1.0, 2.0}
