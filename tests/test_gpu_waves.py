"""The plane-wave field (WAVES2D, a costly velocity: one sine and cosine per mode per
evaluation): GPU steps against the FP64 oracle per step (every trace, a ragged grid, a
time-periodic field, and a step call whose graph is replayed), and the surrogate's RK4
training targets for this field against the oracle's flow map."""
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


@pytest.mark.parametrize("trace", ["rk3", "euler", "heun_psi"])
def test_waves_step_against_oracle(G, trace):
    modes = inputs.wave_modes(48, seed=21)
    n = (157, 131)
    h = 1.0 / (n[0] - 1)
    dt = h / inputs.wave_speed_sampled(modes)
    st = inputs.circle_sdf(n, center=(0.5, 0.5), r=0.25).astype(np.float32)
    vel = G.Velocity("waves2d", modes=modes, trace=trace)
    ov = oracle.velocity("waves2d", modes=modes)
    og = oracle.grid(n)
    worst = [0.0, 0.0]
    # three steps, each against one oracle step from the GPU's state before it
    g2 = G.Grid(n)
    g2.set_state(st, t0=0.37, recon=True)
    for _ in range(3):
        before = g2.read_state().astype(np.float64)
        t = g2.time
        g2.step(vel, dt, 1)
        after = g2.read_state()
        ref = oracle.step(og, ov, before, t, dt, trace_scheme=trace)
        worst[0] = max(worst[0], float(np.max(np.abs(after[0] - ref[0]))))
        worst[1] = max(worst[1], float(np.max(np.abs(after[1:3] - ref[1:3]))))
    assert worst[0] <= 1e-5 and worst[1] <= 1e-4, worst
    # a 3-step call equals three 1-step calls bit for bit
    g3 = G.Grid(n)
    g3.set_state(st, t0=0.37, recon=True)
    g3.step(vel, dt, 3)
    assert np.array_equal(g3.read_state(), g2.read_state())
    for x in (g2, g3):
        x.close()


def test_waves_field_refused_where_not_built(G):
    modes = inputs.wave_modes(8, seed=2)
    g = G.Grid((20, 20, 20))
    g.set_state(inputs.sphere_sdf((20, 20, 20)).astype(np.float32), recon=True)
    with pytest.raises(G.GalsError) as e:
        g.step(G.Velocity("waves2d", modes=modes), 0.01, 1)
    assert e.value.status == G.ERR_UNSUPPORTED
    with pytest.raises(G.GalsError):  # more modes than the table holds
        g2 = G.Grid((20, 20))
        g2.set_state(inputs.circle_sdf((20, 20)).astype(np.float32), recon=True)
        g2.step(G.Velocity("waves2d", modes=inputs.wave_modes(G.MAX_WAVES + 1, seed=3)), 0.01, 1)


def test_waves_training_targets_match_oracle(G):
    modes = inputs.wave_modes(64, seed=23)
    n = 257
    h = 1.0 / (n - 1)
    dt = h / inputs.wave_speed_sampled(modes)
    S = G.Surrogate(seed=3)
    rng = np.random.default_rng(5)
    P = np.stack([rng.uniform(0, 1, 200), rng.uniform(0, 1, 200), rng.uniform(0, 1, 200)], 1)
    T = S.targets(G.Velocity("waves2d", modes=modes), dt, h, P, substeps=32)
    ov = oracle.velocity("waves2d", modes=modes)
    for p, t in zip(P, T):
        foot, J = oracle.flowmap_rk4(ov, 2, p[:2], p[2], dt, 32)
        ref = np.array([(foot[0] - p[0]) / h, (foot[1] - p[1]) / h, (J[0, 0] - 1) / dt, J[0, 1] / dt,
                        J[1, 0] / dt, (J[1, 1] - 1) / dt])
        assert np.max(np.abs(t - ref)) <= 1e-3 * max(1.0, np.max(np.abs(ref))), (t, ref)
