"""Pins of the oracle's velocity fields and backward traces (Sec. 4, Sec. 5.1
examples) against closed forms, finite differences and convergence orders."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

FIELDS = [
    ("vortex2d", 2, dict(T=8.0)),
    ("deform3d", 3, dict(T=3.0)),
    ("pseudo1d", 2, {}),
    ("rotation", 2, dict(omega=2 * math.pi, center=(0.5, 0.5))),
    ("fourier2d", 2, dict(modes=inputs.fourier_modes(16, seed=7, periodic=True))),
    ("waves2d", 2, dict(modes=inputs.wave_modes(32, seed=7))),
]


@pytest.mark.parametrize("kind,dim,kw", FIELDS)
def test_jacobian_matches_finite_differences(kind, dim, kw):
    """Dv (written by hand) equals a central difference of v: a wrong sign or a
    dropped factor in any entry fails."""
    vel = oracle.velocity(kind, **kw)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for _ in range(10):
        x = rng.uniform(0.05, 0.95, dim)
        t = rng.uniform(0, 2)
        v, D = oracle.vel_eval(vel, dim, x, t)
        for j in range(dim):
            e = np.zeros(dim)
            e[j] = eps
            vp, _ = oracle.vel_eval(vel, dim, x + e, t)
            vm, _ = oracle.vel_eval(vel, dim, x - e, t)
            assert np.allclose(D[:, j], (vp - vm) / (2 * eps), atol=1e-7 * max(1, np.abs(D).max()))


@pytest.mark.parametrize("kind,dim,kw", [f for f in FIELDS if f[0] != "pseudo1d"])
def test_divergence_free(kind, dim, kw):
    vel = oracle.velocity(kind, **kw)
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.uniform(0, 1, dim)
        _, D = oracle.vel_eval(vel, dim, x, rng.uniform(0, 3))
        assert abs(np.trace(D)) < 1e-12


def test_vortex_stream_function_values():
    # v = (-Psi_y, Psi_x), Psi = (1/pi) cos(pi t/T) sin^2(pi x) sin^2(pi y) (Sec. 6.1.2)
    vel = oracle.velocity("vortex2d", T=2.0)
    x, y, t = 0.3, 0.6, 0.4
    eps = 1e-6
    Psi = lambda X, Y: (1 / math.pi) * math.cos(math.pi * t / 2.0) * math.sin(math.pi * X) ** 2 * math.sin(math.pi * Y) ** 2
    v, _ = oracle.vel_eval(vel, 2, (x, y), t)
    u_ref = -(Psi(x, y + eps) - Psi(x, y - eps)) / (2 * eps)
    w_ref = (Psi(x + eps, y) - Psi(x - eps, y)) / (2 * eps)
    assert v == pytest.approx([u_ref, w_ref], abs=1e-8)


@pytest.mark.parametrize("scheme", ["euler", "rk3"])
def test_constant_velocity_trace_exact(scheme):
    vel = oracle.velocity("const", c=(0.3, -0.2, 0.7))
    for dim in (1, 2, 3):
        x = np.array([0.4, 0.5, 0.6])[:dim]
        foot, J = oracle.trace(scheme, vel, dim, x, 0.3, 0.01)
        assert np.allclose(foot, x - 0.01 * np.array([0.3, -0.2, 0.7])[:dim], atol=1e-15)
        assert np.allclose(J, np.eye(dim), atol=0)


def test_euler_jacobian_is_I_minus_dt_Dv():
    # Ex. (superconsistent forward Euler): grad foot = I - dt grad v(x, t+dt)
    vel = oracle.velocity("vortex2d", T=8.0)
    x, t, dt = np.array([0.3, 0.7]), 1.1, 0.05
    foot, J = oracle.trace("euler", vel, 2, x, t, dt)
    v, D = oracle.vel_eval(vel, 2, x, t + dt)
    assert np.allclose(foot, x - dt * v, atol=1e-15)
    assert np.allclose(J, np.eye(2) - dt * D, atol=1e-15)


def _rotation_exact(x, c, omega, dt):
    # backward rigid rotation by -omega dt about c
    a = -omega * dt
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    return c + R @ (x - c), R


def test_rotation_rk3_fourth_order_per_step():
    """Sec. 4: one RK3 step must be 4th-order accurate for the foot; rotation has a
    closed-form flow, so halving dt divides the error by ~16."""
    omega, c = 2 * math.pi, np.array([0.5, 0.5])
    vel = oracle.velocity("rotation", omega=omega, center=c)
    x = np.array([0.8, 0.3])
    errs, jerrs = [], []
    for dt in (0.02, 0.01, 0.005):
        foot, J = oracle.trace("rk3", vel, 2, x, 0.0, dt)
        ex, R = _rotation_exact(x, c, omega, dt)
        errs.append(np.max(np.abs(foot - ex)))
        jerrs.append(np.max(np.abs(J - R)))
    for e, f in zip(errs, errs[1:]):
        assert 14.0 < e / f < 18.0
    for e, f in zip(jerrs, jerrs[1:]):
        assert 14.0 < e / f < 18.0


def _pseudo1d_exact(x, dt):
    """Closed-form backward flow of eq. velocity_1: with d = (sqrt2, sqrtpi)/sqrt(2+pi)
    and s = d.x, ds/dt = e^s, so s(t) = -ln(e^{-s} + dt); the transverse coordinate
    is fixed.  J = I + d d^T (ds_foot/ds - 1)."""
    d = np.array([math.sqrt(2), math.sqrt(math.pi)]) / math.sqrt(2 + math.pi)
    s = d @ x
    sf = -math.log(math.exp(-s) + dt)
    dsf = math.exp(-s) / (math.exp(-s) + dt)
    return x + (sf - s) * d, np.eye(2) + np.outer(d, d) * (dsf - 1)


def test_pseudo1d_rk3_fourth_order_per_step():
    vel = oracle.velocity("pseudo1d")
    x = np.array([0.6, 0.4])
    errs, jerrs = [], []
    for dt in (0.04, 0.02, 0.01):
        foot, J = oracle.trace("rk3", vel, 2, x, 0.0, dt)
        ex, Jex = _pseudo1d_exact(x, dt)
        errs.append(np.max(np.abs(foot - ex)))
        jerrs.append(np.max(np.abs(J - Jex)))
    for e, f in zip(errs, errs[1:]):
        assert 13.0 < e / f < 19.0
    for e, f in zip(jerrs, jerrs[1:]):
        assert 13.0 < e / f < 19.0


@pytest.mark.parametrize("kind,dim,kw", FIELDS)
def test_rk3_jacobian_is_derivative_of_foot_map(kind, dim, kw):
    """Superconsistency needs J = d foot / d x of the *approximate* map (Sec. 5.1)."""
    vel = oracle.velocity(kind, **kw)
    rng = np.random.default_rng(11)
    eps = 1e-6
    for _ in range(5):
        x = rng.uniform(0.1, 0.9, dim)
        t, dt = rng.uniform(0, 2), 0.03
        foot, J = oracle.trace("rk3", vel, dim, x, t, dt)
        for j in range(dim):
            e = np.zeros(dim)
            e[j] = eps
            fp, _ = oracle.trace("rk3", vel, dim, x + e, t, dt)
            fm, _ = oracle.trace("rk3", vel, dim, x - e, t, dt)
            assert np.allclose(J[:, j], (fp - fm) / (2 * eps), atol=1e-8)


def test_rk4_flowmap_rotation_and_richardson():
    omega, c = 2 * math.pi, np.array([0.5, 0.5])
    vel = oracle.velocity("rotation", omega=omega, center=c)
    x = np.array([0.8, 0.3])
    foot, J = oracle.flowmap_rk4(vel, 2, x, 0.0, 0.05, 32)
    ex, R = _rotation_exact(x, c, omega, 0.05)
    assert np.max(np.abs(foot - ex)) < 1e-10 and np.max(np.abs(J - R)) < 1e-10
    vel = oracle.velocity("fourier2d", modes=inputs.fourier_modes(16, seed=9, periodic=True))
    # Richardson: against a 512-sub-step reference, 8 -> 16 sub-steps divides the
    # error by ~2^4 (classical RK4 is 4th order globally); 16 -> 32 sub-steps
    x0 = np.array([0.3, 0.6])
    fr, Jr = oracle.flowmap_rk4(vel, 2, x0, 0.2, 0.05, 512)
    f8, J8 = oracle.flowmap_rk4(vel, 2, x0, 0.2, 0.05, 16)
    f16, J16 = oracle.flowmap_rk4(vel, 2, x0, 0.2, 0.05, 32)
    r = np.max(np.abs(f8 - fr)) / np.max(np.abs(f16 - fr))
    rj = np.max(np.abs(J8 - Jr)) / np.max(np.abs(J16 - Jr))
    assert 12.0 < r < 20.0 and 12.0 < rj < 20.0


def _golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        return json.load(f)


def test_deform3d_values_at_exact_points():
    """LeVeque's field of Sec. 6.2.4 at points where every sine is exact (values worked
    out by hand from the printed formulas, stored with their derivation): a global sign
    flip, a swapped component, the garbled sin(2 pi x y) reading or a wrong modulation
    fails."""
    gold = _golden()["deform3d_point_values"]
    vel = oracle.velocity("deform3d", T=gold["T"])
    for pt in gold["points"]:
        v, D = oracle.vel_eval(vel, 3, pt["x"], pt["t"])
        assert np.allclose(v, pt["v"], atol=1e-14), (pt["x"], v)
        assert np.allclose(D, np.array(pt["Dv"]), atol=1e-13), (pt["x"], D)


def _fourier_psi(modes, x, y, t):
    """Stream function of the Fourier fields, written out again from its definition:
    Psi = sum_m a_m sin(k_m pi x) sin(l_m pi y) cos(2 pi n_m t + chi_m)."""
    return sum(a * math.sin(k * math.pi * x) * math.sin(l * math.pi * y)
               * math.cos(2 * math.pi * n * t + chi) for a, k, l, n, chi in modes)


def test_fourier_velocity_is_rotated_stream_function_gradient():
    """v = (-dPsi/dy, dPsi/dx) by central differences of an independently written Psi:
    the field running the wrong way round, or a mode's k and l exchanged, fails."""
    modes = inputs.fourier_modes(16, seed=5, periodic=True)
    vel = oracle.velocity("fourier2d", modes=modes)
    rng = np.random.default_rng(8)
    eps = 1e-6
    for _ in range(12):
        x, y, t = rng.uniform(0.02, 0.98), rng.uniform(0.02, 0.98), rng.uniform(0, 1)
        v, _ = oracle.vel_eval(vel, 2, (x, y), t)
        u_ref = -(_fourier_psi(modes, x, y + eps, t) - _fourier_psi(modes, x, y - eps, t)) / (2 * eps)
        w_ref = (_fourier_psi(modes, x + eps, y, t) - _fourier_psi(modes, x - eps, y, t)) / (2 * eps)
        assert v == pytest.approx([u_ref, w_ref], abs=1e-7)


def test_fourier_single_mode_hand_values():
    """One mode Psi = sin(pi x) sin(2 pi y) (a = 1, k = 1, l = 2, steady): at (1/4, 1/8)
    u = -Psi_y = -2 pi sin(pi/4) cos(pi/4) = -pi, v = Psi_x = pi cos(pi/4) sin(pi/4) = pi/2,
    du/dx = -2 pi^2 cos(pi/4)^2 = -pi^2, du/dy = 4 pi^2 sin(pi/4)^2 = 2 pi^2,
    dv/dx = -pi^2 sin(pi/4)^2 = -pi^2/2, dv/dy = pi^2."""
    vel = oracle.velocity("fourier2d", modes=np.array([[1.0, 1.0, 2.0, 0.0, 0.0]]))
    v, D = oracle.vel_eval(vel, 2, (0.25, 0.125), 0.37)
    p2 = math.pi ** 2
    assert v == pytest.approx([-math.pi, math.pi / 2], abs=1e-14)
    assert np.allclose(D, [[-p2, 2 * p2], [-p2 / 2, p2]], atol=1e-13)


def test_waves_single_mode_hand_values():
    """One plane wave Psi = sin(pi x + 2 pi y) cos(2 pi t) (a = 1, k = (pi, 2 pi)):
    at (1/4, 1/8) the phase is pi/2, so u = v = 0 and du/dx = kx ky = 2 pi^2,
    du/dy = ky^2 = 4 pi^2, dv/dx = -kx^2 = -pi^2, dv/dy = -2 pi^2, times cos(2 pi t);
    at the origin the phase is 0: u = -ky = -2 pi, v = kx = pi, Dv = 0."""
    vel = oracle.velocity("waves2d", modes=np.array([[1.0, math.pi, 2 * math.pi, 0.0, 1.0, 0.0]]))
    p2 = math.pi ** 2
    v, D = oracle.vel_eval(vel, 2, (0.25, 0.125), 0.125)
    c = math.cos(math.pi / 4)
    assert v == pytest.approx([0.0, 0.0], abs=1e-14)
    assert np.allclose(D, c * np.array([[2 * p2, 4 * p2], [-p2, -2 * p2]]), atol=1e-12)
    v, D = oracle.vel_eval(vel, 2, (0.0, 0.0), 0.0)
    assert v == pytest.approx([-2 * math.pi, math.pi], abs=1e-14)
    assert np.allclose(D, 0.0, atol=1e-12)


def test_waves_velocity_is_rotated_stream_function_gradient():
    """v = (-dPsi/dy, dPsi/dx) by central differences of Psi written out again, and Dv
    against central differences of v, for 64 random plane waves; trace(Dv) = 0."""
    modes = inputs.wave_modes(64, seed=12)
    vel = oracle.velocity("waves2d", modes=modes)

    def psi(x, y, t):
        return sum(a * math.sin(kx * x + ky * y + ph) * math.cos(2 * math.pi * n * t + chi)
                   for a, kx, ky, ph, n, chi in modes)

    rng = np.random.default_rng(13)
    eps = 1e-6
    for _ in range(8):
        x, y, t = rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(0, 1)
        v, D = oracle.vel_eval(vel, 2, (x, y), t)
        u_ref = -(psi(x, y + eps, t) - psi(x, y - eps, t)) / (2 * eps)
        w_ref = (psi(x + eps, y, t) - psi(x - eps, y, t)) / (2 * eps)
        assert v == pytest.approx([u_ref, w_ref], abs=2e-7)
        for j in range(2):
            e = np.zeros(2)
            e[j] = eps
            vp, _ = oracle.vel_eval(vel, 2, np.array([x, y]) + e, t)
            vm, _ = oracle.vel_eval(vel, 2, np.array([x, y]) - e, t)
            assert np.allclose(D[:, j], (vp - vm) / (2 * eps), atol=1e-6 * max(1, np.abs(D).max()))
        assert abs(np.trace(D)) < 1e-12
    # the sampled speed used for the CFL rule lies below the library's analytic bound
    assert inputs.wave_speed_sampled(modes) <= 1.1 * inputs.wave_speed_bound(modes)
