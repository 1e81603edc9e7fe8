"""Batched 2D mode: every problem of a batch evolves bit for bit as the same problem on
its own grid (the per-tile code is shared), for every launch shape and time loop (one
launch per step, or all steps in one persistent launch) the autotuner can pick; one
problem is also checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


SIZES = [(130, 97), (64, 64), (257, 200), (37, 41), (128, 129), (300, 17)]
# the smallest problems the ABI takes, and problems one or two tiles narrow in either axis
TINY = [(4, 4), (5, 4), (4, 5), (6, 1030), (1030, 6), (129, 4), (4, 129)]


def _problems(sizes=SIZES):
    probs = inputs.batch_problems(len(sizes), seed=7)
    states, vels, dts = [], [], []
    for (nx, ny), p in zip(sizes, probs):
        st = inputs.ellipse_sdf((nx, ny), p.center, p.a, p.b, p.angle, iters=60)
        states.append(st.astype(np.float32))
        vels.append(p.modes)
        h = 1.0 / (max(nx, ny) - 1)
        dts.append(h / inputs.fourier_speed_bound(p.modes))
    return sizes, states, vels, dts


@pytest.mark.parametrize("layout", ["full", "compact"])
@pytest.mark.parametrize("sizes", [SIZES, TINY], ids=["mixed", "tiny"])
def test_batch_equals_single_grids(G, layout, sizes):
    sizes, states, modes, dts = _problems(sizes)
    vels = [G.Velocity("fourier2d", modes=m) for m in modes]
    singles = []
    for n, st, v, dt in zip(sizes, states, vels, dts):
        g = G.Grid(n, layout=layout)
        g.set_state(st, t0=0.25, recon=True)
        g.step(v, dt, 3)
        singles.append(g.read_state())
        g.close()
    for variant, blocks, loop in ((0, 0, "launches"), (1, 0, "launches"), (1, 152, "launches"),
                                  (0, 304, "launches"), (0, 0, "persistent"), (1, 0, "persistent")):
        b = G.Batch(sizes, layout=layout)
        for p, st in enumerate(states):
            b.set_state(p, st, t0=0.25, recon=True)
        b.set_tuning(variant, blocks, loop)
        b.step(vels, dts, 2)
        b.step(vels, dts, 1)
        for p in range(len(sizes)):
            assert np.array_equal(b.read_state(p), singles[p]), (variant, blocks, loop, p)
        b.close()


def test_batch_autotune_leaves_state(G):
    sizes, states, modes, dts = _problems()
    vels = [G.Velocity("fourier2d", modes=m) for m in modes]
    b = G.Batch(sizes)
    for p, st in enumerate(states):
        b.set_state(p, st, recon=True)
    before = [b.read_state(p) for p in range(len(sizes))]
    t = b.autotune(vels, dts, trial_steps=2)
    assert t["variant"] in (0, 1) and t["blocks"] >= 0 and t["ms_per_step"] > 0
    assert t["loop"] in ("launches", "persistent")
    for p in range(len(sizes)):
        assert np.array_equal(b.read_state(p), before[p])
    assert b.nodes == sum(nx * ny for nx, ny in sizes)


def test_batch_problem_against_oracle(G):
    sizes, states, modes, dts = _problems()
    vels = [G.Velocity("fourier2d", modes=m) for m in modes]
    b = G.Batch(sizes)
    for p, st in enumerate(states):
        b.set_state(p, st, recon=True)
    p = 2
    before = b.read_state(p).astype(np.float64)
    b.step(vels, dts, 1)
    after = b.read_state(p).astype(np.float64)
    og = oracle.grid(sizes[p])
    ref = oracle.step(og, oracle.velocity("fourier2d", modes=modes[p]), before, 0.0, dts[p])
    assert np.max(np.abs(after[0] - ref[0])) <= 1e-5
    assert np.max(np.abs(after[1:3] - ref[1:3])) <= 1e-4


def test_batch_errors(G):
    b = G.Batch([(16, 16), (20, 12)])
    st = inputs.circle_sdf((16, 16), r=0.3, center=(0.5, 0.5)).astype(np.float32)
    b.set_state(0, st)
    v = [G.Velocity("rotation", omega=1.0, center=(0.5, 0.5, 0.0))] * 2
    with pytest.raises(G.GalsError) as e:
        b.step(v, [0.01, 0.01], 1)
    assert e.value.status == G.ERR_STATE
    b.set_state(1, inputs.circle_sdf((20, 12), r=0.3, center=(0.5, 0.5)).astype(np.float32))
    with pytest.raises(G.GalsError) as e:
        b.step([v[0], G.Velocity("vortex2d", T=8.0)], [0.01, 0.01], 1)
    assert e.value.status == G.ERR_ARG
    with pytest.raises(G.GalsError) as e:
        b.step([G.Velocity("rotation", trace="euler")] * 2, [0.01, 0.01], 1)
    assert e.value.status == G.ERR_UNSUPPORTED
    with pytest.raises(G.GalsError):
        b.set_state(2, st)
