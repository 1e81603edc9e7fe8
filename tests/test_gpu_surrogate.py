"""Learned flow-map surrogate: the GPU's RK4 targets, tensor-core forward pass and
training gradients against the FP64 oracle; training lowers the loss; the surrogate step
with every tile falling back equals the exact RK3 step to parity tolerance; the step the
network drives equals the oracle step fed the network's map; the residual-check counters;
and the learned against the plain RK3 trace at equal interface error."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [3, 128, 128, 128, 128, 6]


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


@pytest.fixture(scope="module")
def field():
    modes = inputs.fourier_modes(16, seed=9053409, periodic=True)
    n = 257
    h = 1.0 / (n - 1)
    dt = h / inputs.fourier_speed_bound(modes)
    return modes, n, h, dt


def test_rk4_targets_match_oracle(G, field):
    modes, n, h, dt = field
    S = G.Surrogate(seed=3)
    rng = np.random.default_rng(0)
    P = np.stack([rng.uniform(0, 1, 200), rng.uniform(0, 1, 200), rng.uniform(0, 1, 200)], 1)
    T = S.targets(G.Velocity("fourier2d", modes=modes), dt, h, P, substeps=32)
    ov = oracle.velocity("fourier2d", modes=modes)
    for p, t in zip(P, T):
        foot, J = oracle.flowmap_rk4(ov, 2, p[:2], p[2], dt, 32)
        ref = np.array([(foot[0] - p[0]) / h, (foot[1] - p[1]) / h, (J[0, 0] - 1) / dt, J[0, 1] / dt,
                        J[1, 0] / dt, (J[1, 1] - 1) / dt])
        assert np.max(np.abs(t - ref)) <= 1e-3 * max(1.0, np.max(np.abs(ref))), (t, ref)


def test_forward_matches_oracle(G):
    S = G.Surrogate(seed=11)
    params, scales = S.get_params()
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (1000, 3)).astype(np.float32)
    Y = S.forward(X)
    Yref = oracle.mlp_forward(SIZES, params.astype(np.float64), X.astype(np.float64))
    err = np.max(np.abs(Y - Yref)) / max(1.0, np.max(np.abs(Yref)))
    assert err <= 2e-2, err  # 16-bit operands, hardware tanh in SiLU


def test_forward_device_matches_host_forward(G):
    """The device-pointer entry runs the same kernel: bit-identical outputs, including a
    ragged last tile."""
    import torch
    S = G.Surrogate(seed=11)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (1000, 3)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full((1000, 6), float("nan"), device="cuda")
    torch.cuda.synchronize()
    S.forward_device(Xd.data_ptr(), 1000, Yd.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(Yd.cpu().numpy(), S.forward(X))
    with pytest.raises(G.GalsError):
        S.forward_device(Xd.data_ptr(), 0, Yd.data_ptr())


def test_gradient_matches_oracle(G):
    """Backward kernels (BF16 operands, FP32 accumulation) against the FP64 chain rule,
    tensor by tensor, relative to each tensor's norm."""
    S = G.Surrogate(seed=5)
    params, _ = S.get_params()
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (4096, 3)).astype(np.float32)
    T = rng.normal(0, 1, (4096, 6)).astype(np.float32)
    loss, grad = S.gradient(X, T)
    lref, gref = oracle.mlp_backward(SIZES, params.astype(np.float64), X.astype(np.float64),
                                     T.astype(np.float64))
    assert loss == pytest.approx(lref, rel=1e-2)
    off = 0
    for l in range(5):
        ni, no = SIZES[l], SIZES[l + 1]
        for size in (ni * no, no):
            a, b = grad[off:off + size], gref[off:off + size]
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert rel <= 1e-2, (l, size, rel)
            off += size
    assert off == G.MLP_PARAMS


def test_training_lowers_loss_and_fallback(G, field):
    modes, n, h, dt = field
    vel = G.Velocity("fourier2d", modes=modes)
    S = G.Surrogate(seed=7)
    rep = S.train(vel, dt, h, steps=300, batch=8192, lr=2e-3, lr_min=1e-4)
    assert rep["final_loss"] < 0.25 * rep["initial_loss"], rep
    # every tile falls back (zero tolerance): the step equals the exact RK3 step
    S.set_check(tol_x=0.0, tol_J=0.0, samples=4)
    st = inputs.ellipse_sdf((n, n), (0.5, 0.5), 0.2, 0.1, 0.3, iters=60).astype(np.float32)
    g = G.Grid((n, n))
    g.set_state(st, t0=0.3, recon=True)
    before = g.read_state().astype(np.float64)
    S.stats(reset=True)
    g.step(G.Velocity("fourier2d", modes=modes, trace="surrogate", surrogate=S), dt, 1)
    after = g.read_state().astype(np.float64)
    tiles, falls = S.stats()
    assert tiles == ((n + 127) // 128) * n and falls == tiles
    ref = oracle.step(oracle.grid((n, n)), oracle.velocity("fourier2d", modes=modes), before, 0.3, dt)
    assert np.max(np.abs(after[0] - ref[0])) <= 1e-5
    assert np.max(np.abs(after[1:3] - ref[1:3])) <= 1e-4
    # loose tolerance: no fallback, the learned trace drives the step
    S.set_check(tol_x=1e9, tol_J=1e9, samples=1)
    S.stats(reset=True)
    g.set_state(st, t0=0.3, recon=True)
    g.step(G.Velocity("fourier2d", modes=modes, trace="surrogate", surrogate=S), dt, 3)
    tiles, falls = S.stats()
    assert falls == 0 and tiles == 3 * ((n + 127) // 128) * n
    assert np.isfinite(g.read_state()).all()
    # a field other than the trained one is refused
    with pytest.raises(G.GalsError):
        g.step(G.Velocity("fourier2d", modes=modes * 1.01, trace="surrogate", surrogate=S), dt, 1)


@pytest.mark.parametrize("kind", ["fourier2d", "waves2d"])
def test_learned_step_matches_oracle_given_map(G, field, kind):
    """One step driven by the network alone (residual check off, no fallback) on a
    ragged grid (257 x 130 nodes, h = 1/256 on [0,1] x [0, 129/256]: a partial last
    tile in x and in y) against the oracle step fed the same backward map.  The map is
    rebuilt on the host from the network's normalised outputs y at the nodes' inputs
    (2x - 1, 2y - 1, 2 (t mod 1) - 1), by the documented rule: foot - x = (y0 s0 h,
    y1 s1 h), J = I + dt [[y2 s2, y3 s3], [y4 s4, y5 s5]] (s: the output scales), in FP64.
    The outputs come from the tensor-core forward pass (the tile code the step runs),
    which is itself held to the FP64 oracle network below; the oracle then does the
    Hermite stage and psi+ = J^T grad H (Sec. 4 step 2, eq. superconsistency).  A wrong
    scale, h or dt factor, a transposed J or a shifted input fails the per-step
    tolerances."""
    modes, n, h, dt = field
    if kind == "waves2d":  # the costly field: 96 plane waves
        modes = inputs.wave_modes(96, seed=31)
        dt = h / inputs.wave_speed_sampled(modes)
    vel = G.Velocity(kind, modes=modes)
    S = G.Surrogate(seed=17)
    S.train(vel, dt, h, steps=300, batch=8192, lr=2e-3, lr_min=1e-4)
    S.set_check(tol_x=1e9, tol_J=1e9, samples=1)
    shape = (257, 130)
    hi = (1.0, (shape[1] - 1) * h)
    t0 = 0.3
    st = inputs.circle_sdf(shape, center=(0.45, 0.27), r=0.15, lo=(0.0, 0.0), hi=hi).astype(np.float32)
    g = G.Grid(shape, lo=(0.0, 0.0), hi=hi)
    g.set_state(st, t0=t0, recon=True)
    before = g.read_state().astype(np.float64)
    S.stats(reset=True)
    g.step(G.Velocity(kind, modes=modes, trace="surrogate", surrogate=S), dt, 1)
    after = g.read_state().astype(np.float64)
    tiles, falls = S.stats()
    assert falls == 0 and tiles == ((shape[0] + 127) // 128) * shape[1]

    # the network's inputs at every node, in the kernel's FP32 arithmetic
    i = np.arange(shape[0], dtype=np.float32)
    j = np.arange(shape[1], dtype=np.float32)
    hf = np.float32(h)
    xs, ys = np.meshgrid(i * hf, j * hf)  # (ny, nx), x fastest
    phase = np.float32(t0 - math.floor(t0))
    X = np.stack([np.float32(2) * xs - np.float32(1), np.float32(2) * ys - np.float32(1),
                  np.full_like(xs, np.float32(2) * phase - np.float32(1))], -1).reshape(-1, 3)
    Y = S.forward(X).astype(np.float64)
    params, scales = S.get_params()
    s = scales.astype(np.float64)
    Y = Y.reshape(shape[1], shape[0], 6)
    disp = np.stack([Y[..., 0] * s[0] * h, Y[..., 1] * s[1] * h])
    jac = np.array([[1.0 + dt * Y[..., 2] * s[2], dt * Y[..., 3] * s[3]],
                    [dt * Y[..., 4] * s[4], 1.0 + dt * Y[..., 5] * s[5]]])
    assert np.max(np.abs(disp)) > 0.2 * h  # the network moves the feet
    ref = oracle.step_given(oracle.grid(shape, lo=(0.0, 0.0), hi=hi), before, disp, jac)
    dphi = np.max(np.abs(after[0] - ref[0]))
    dpsi = np.max(np.abs(after[1:3] - ref[1:3]))
    assert dphi <= 1e-5 and dpsi <= 1e-4, (dphi, dpsi)
    # mixed derivatives: the oracle's approach-A rebuild of the GPU's own gradients
    rec = oracle.recon_cross(oracle.grid(shape, lo=(0.0, 0.0), hi=hi), after)
    scale = max(1.0, np.max(np.abs(after[1:3])))
    assert np.max(np.abs(after[3] - rec[3])) <= 2e-6 * scale / h + 1e-6 * scale / h
    # the network's outputs at these inputs against the FP64 oracle network: BF16 operands
    # and activations (unit roundoff 2^-9 per rounding, several roundings per product, five
    # layers, cancellation in trained sums) and the FP16 tanh: about 1 % in norm measured
    Yref = oracle.mlp_forward(SIZES, params.astype(np.float64), X.astype(np.float64))
    Yg = Y.reshape(-1, 6)
    assert np.linalg.norm(Yg - Yref) <= 2e-2 * np.linalg.norm(Yref)
    assert np.max(np.abs(Yg - Yref)) <= 6e-2 * max(1.0, np.max(np.abs(Yref)))


@pytest.mark.parametrize("kind", ["fourier2d", "waves2d"])
def test_learned_vs_plain_at_equal_error(G, field, kind):
    """What the learned trace gains over the plain RK3 trace at equal interface error, on the
    16-mode Fourier field and on the costly 128-plane-wave field (every plain evaluation
    costs one sine and cosine per wave; the network's cost does not depend on the field).
    Both advance the same initial interface to the same end time; each run's error is the
    symmetric difference of its interface from a 4x finer-in-time RK3 run.  The learned trace
    runs at the step it was trained for; the plain trace also takes steps c times longer
    (the scheme is stable at any CFL number), and the cheapest plain run whose error is at
    most 1.1x the learned run's is its equal-error counterpart.

    Outcome asserted (measured on a GB300 at 2048^2 and here): the plain trace wins at equal
    error, by a wide margin -- its error at 8x longer steps is still below the learned
    trace's, and its time to the end time is several times shorter -- although on the
    costly field one network evaluation per node is cheaper than one RK3 step."""
    modes, n, h, dt = field
    if kind == "waves2d":
        modes = inputs.wave_modes(128, seed=41)
        dt = h / inputs.wave_speed_sampled(modes)
    steps = 200
    vel = G.Velocity(kind, modes=modes)
    S = G.Surrogate(seed=9)
    S.train(vel, dt, h, steps=800, batch=16384, lr=2e-3, lr_min=1e-5)
    S.set_check(tol_x=0.05, tol_J=0.05, samples=4)
    st = inputs.circle_sdf((n, n), center=(0.5, 0.6), r=0.2).astype(np.float32)

    def run(v, step, nsteps):
        g = G.Grid((n, n))
        g.set_state(st, t0=0.0, recon=True)
        g.step(v, step, nsteps)  # captures the graph
        g.set_state(st, t0=0.0, recon=True)
        g.synchronize()
        t0 = time.perf_counter()
        g.step(v, step, nsteps)
        g.synchronize()
        return g, time.perf_counter() - t0

    fine, _ = run(vel, dt / 4, 4 * steps)
    learned, t_learned = run(G.Velocity(kind, modes=modes, trace="surrogate", surrogate=S), dt, steps)
    e_learned = learned.diagnostics(q=4, reference=fine)["measure_symdiff"]
    plain = []
    for c in (1, 2, 4, 5, 8, 10, 20, 25, 40, 50):
        g, t = run(vel, c * dt, steps // c)
        plain.append((c, t, g.diagnostics(q=4, reference=fine)["measure_symdiff"]))
        g.close()
    print(f"{kind}: learned {t_learned * 1e3:.1f} ms, interface error {e_learned:.3e}; plain RK3 "
          + ", ".join(f"x{c}: {t * 1e3:.1f} ms err {e:.3e}" for c, t, e in plain))
    assert math.isfinite(e_learned) and e_learned > 0
    ok = [(t, c) for c, t, e in plain if e <= 1.1 * e_learned]
    assert ok, "no plain run reached the learned trace's error"
    t_best, c_best = min(ok)
    assert c_best >= 8 and t_best < 0.5 * t_learned, (c_best, t_best, t_learned)
    for g in (fine, learned):
        g.close()


def test_save_load_roundtrip(G, field, tmp_path):
    """A saved surrogate loads into a fresh handle with the same parameters, scales,
    residual check and bound field: its forward pass and a learned step are bit-identical;
    a file that is not a surrogate is refused."""
    modes, n, h, dt = field
    vel = G.Velocity("fourier2d", modes=modes)
    S = G.Surrogate(seed=13)
    S.train(vel, dt, h, steps=40, batch=4096, lr=2e-3, lr_min=1e-4)
    S.set_check(tol_x=0.07, tol_J=0.06, samples=3)
    path = tmp_path / "mlp.bin"
    S.save(path)
    T = G.Surrogate(seed=99)
    T.load(path)
    p1, s1 = S.get_params()
    p2, s2 = T.get_params()
    assert np.array_equal(p1, p2) and np.array_equal(s1, s2)
    X = np.random.default_rng(6).uniform(-1, 1, (500, 3)).astype(np.float32)
    assert np.array_equal(S.forward(X), T.forward(X))
    st = inputs.ellipse_sdf((n, n), (0.5, 0.5), 0.2, 0.1, 0.3, iters=60).astype(np.float32)
    outs = []
    for sur in (S, T):
        g = G.Grid((n, n))
        g.set_state(st, t0=0.2, recon=True)
        sur.stats(reset=True)
        g.step(G.Velocity("fourier2d", modes=modes, trace="surrogate", surrogate=sur), dt, 2)
        outs.append((g.read_state(), sur.stats()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a surrogate")
    with pytest.raises(G.GalsError):
        T.load(bad)
