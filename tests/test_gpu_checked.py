"""The checked build (libgals_checked.so, compiled with -DGALS_CHECKED: the step kernels
test every data-dependent index against its buffer and report a violation through the
grid's error word, which fails the call with the source line) on small odd grids,
tile-edge sizes, large CFL, both layouts, approach B, the persistent 2D time loop, the
batched mode and the banded host step.  No index may leave its buffer, and the results must be those of the normal
build bit for bit.  The checked library runs in a child process (GALS_LIB), the normal one
in the test's own."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0905_3409_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

ROT = dict(kind="rotation", omega=2 * math.pi, center=(0.5, 0.5, 0.5))
CASES = [
    # (n, velocity, cells per step, layout, cross)
    ((5, 7), dict(kind="vortex2d", T=8.0), 0.9, "full", "central"),
    ((130, 67), ROT, 2.5, "full", "central"),
    ((131, 29), dict(kind="vortex2d", T=8.0), 0.9, "compact", "central"),
    ((61, 47), dict(kind="vortex2d", T=8.0), 1.5, "full", "cell"),
    ((9, 5, 4), dict(kind="deform3d", T=3.0), 0.9, "full", "central"),
    ((21, 18, 17), dict(kind="deform3d", T=3.0), 2.0, "full", "central"),
    ((19, 17, 16), dict(kind="deform3d", T=3.0), 0.9, "compact", "central"),
    ((13, 11, 9), dict(kind="deform3d", T=3.0), 0.9, "full", "cell"),
]


def run_cases():
    """All cases through whichever library gals loads; returns named arrays."""
    from paper_0905_3409_gb300 import gals as G
    out = {}
    for c, (n, vel, cells, layout, cross) in enumerate(CASES):
        st = (inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3) if len(n) == 2 else
              inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.3)).astype(np.float32)
        g = G.Grid(n, layout=layout, cross=cross)
        g.set_state(st, t0=0.2, recon=True)
        g.step(G.Velocity(**vel), cells / (max(n) - 1), 3)
        out[f"case{c}"] = g.read_state()
        out[f"diag{c}"] = np.array([v for v in g.diagnostics(q=2).values()], dtype=np.float64)
        g.close()
    # the persistent 2D time loop (feet 2.5 cells away: gathers from global memory too)
    for c, (n, vel, cells) in enumerate((((130, 67), ROT, 2.5), ((300, 45), dict(kind="vortex2d", T=8.0), 0.9))):
        st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3).astype(np.float32)
        g = G.Grid(n)
        g.set_time_loop("persistent")
        g.set_state(st, t0=0.2, recon=True)
        g.step(G.Velocity(**vel), cells / (max(n) - 1), 4)
        out[f"persist{c}"] = g.read_state()
        g.close()
    sizes = [(4, 4), (5, 4), (130, 17), (6, 129)]
    probs = inputs.batch_problems(len(sizes), seed=3)
    b = G.Batch(sizes)
    vels, dts = [], []
    for p, ((nx, ny), pr) in enumerate(zip(sizes, probs)):
        b.set_state(p, inputs.ellipse_sdf((nx, ny), pr.center, pr.a, pr.b, pr.angle, iters=60).astype(np.float32),
                    recon=True)
        vels.append(G.Velocity("fourier2d", modes=pr.modes))
        dts.append(1.0 / (max(nx, ny) - 1) / inputs.fourier_speed_bound(pr.modes))
    b.step(vels, dts, 2)
    for p in range(len(sizes)):
        out[f"batch{p}"] = b.read_state(p)
    b.close()
    b = G.Batch(sizes)  # the persistent multi-step loop
    b.set_tuning(0, 0, "persistent")
    for p, ((nx, ny), pr) in enumerate(zip(sizes, probs)):
        b.set_state(p, inputs.ellipse_sdf((nx, ny), pr.center, pr.a, pr.b, pr.angle, iters=60).astype(np.float32),
                    recon=True)
    b.step(vels, dts, 3)
    for p in range(len(sizes)):
        out[f"batchp{p}"] = b.read_state(p)
    b.close()
    for c, (n, vel, cells) in enumerate((((150, 200), dict(kind="vortex2d", T=8.0), 0.8),
                                         ((24, 20, 37), dict(kind="deform3d", T=3.0), 0.4))):
        st = (inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3) if len(n) == 2 else
              inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.3)).astype(np.float32)
        g = G.Grid(n)
        g.set_state(st, recon=True)
        full = g.read_state()
        res = np.empty_like(full)
        g.step_host(G.Velocity(**vel), cells / (max(n) - 1), 0.3, full, res)
        out[f"host{c}"] = res
        g.close()
    return out


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def test_checked_build_no_violation_and_same_results(G, tmp_path):
    from paper_0905_3409_gb300 import build
    checked = build.build_checked()
    dst = str(tmp_path / "checked.npz")
    env = dict(os.environ, GALS_LIB=checked)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), dst], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = np.load(dst)
    ref = run_cases()
    assert sorted(got.files) == sorted(ref)
    for k in ref:
        assert np.array_equal(got[k], ref[k], equal_nan=True), k


if __name__ == "__main__":
    from paper_0905_3409_gb300 import gals as _G
    assert _G.LIB_PATH.endswith("libgals_checked.so"), _G.LIB_PATH
    np.savez(sys.argv[1], **run_cases())
