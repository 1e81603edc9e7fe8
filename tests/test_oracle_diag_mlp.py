"""Pins of the oracle's diagnostics (area/volume by sub-sampling, interface
error, e_max of eq. maximum_norm) and of its FP64 MLP (finite differences, Adam)."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs


def test_half_plane_area_exact():
    """Hermite reproduces linear phi exactly, so {H<0} of phi = x - 0.3 is the
    half plane; with q cell-centred samples the count is exact."""
    n, q = (17, 11), 8
    g = oracle.grid(n)
    st = inputs.linear2d(n, a=(1.0, 0.0), c=-0.3)
    hx = 1.0 / (n[0] - 1)
    xs = (np.arange((n[0] - 1) * q) + 0.5) * hx / q
    expected = np.count_nonzero(xs < 0.3) * (hx / q) * 1.0
    assert oracle.measure_negative(g, st, q) == pytest.approx(expected, abs=1e-14)


def test_circle_area_and_sphere_volume():
    n = 129
    g = oracle.grid((n, n))
    st = oracle.recon_cross(g, inputs.circle_sdf((n, n), r=0.15))
    area = oracle.measure_negative(g, st, 8)
    assert area == pytest.approx(math.pi * 0.15 ** 2, rel=2e-3)
    n3 = 49
    g3 = oracle.grid((n3,) * 3)
    st3 = oracle.recon_cross(g3, inputs.sphere_sdf((n3,) * 3, r=0.25, center=(0.5, 0.5, 0.5)))
    vol = oracle.measure_negative(g3, st3, 4)
    assert vol == pytest.approx(4 / 3 * math.pi * 0.25 ** 3, rel=5e-3)


def test_symdiff_half_planes():
    n, q = (21, 9), 10
    g = oracle.grid(n)
    a = inputs.linear2d(n, a=(1.0, 0.0), c=-0.3)
    b = inputs.linear2d(n, a=(1.0, 0.0), c=-0.35)
    d, amb = oracle.symdiff(g, a, b, q)
    assert d == pytest.approx(0.05, abs=1.0 / ((n[0] - 1) * q))
    same, _ = oracle.symdiff(g, a, a, q)
    assert same == 0.0


def test_emax_definition():
    a = np.array([0.0, 1.0, -2.0])
    b = np.array([0.5, 1.0, 1.0])
    assert oracle.emax(a, b) == 3.0


def _fd_grad(sizes, params, X, T, idx, eps=1e-6):
    out = []
    for i in idx:
        p1 = params.copy(); p1[i] += eps
        p2 = params.copy(); p2[i] -= eps
        l1, _ = oracle.mlp_backward(sizes, p1, X, T)
        l2, _ = oracle.mlp_backward(sizes, p2, X, T)
        out.append((l1 - l2) / (2 * eps))
    return np.array(out)


def test_mlp_gradient_finite_differences():
    sizes = [3, 16, 16, 6]
    rng = np.random.default_rng(0)
    params = rng.normal(0, 0.5, oracle.mlp_param_count(sizes))
    X = rng.uniform(-1, 1, (32, 3))
    T = rng.normal(size=(32, 6))
    loss, grad = oracle.mlp_backward(sizes, params, X, T)
    Y = oracle.mlp_forward(sizes, params, X)
    assert loss == pytest.approx(np.mean((Y - T) ** 2), rel=1e-14)
    idx = rng.choice(params.size, 40, replace=False)
    fd = _fd_grad(sizes, params, X, T, idx)
    assert np.allclose(grad[idx], fd, rtol=1e-6, atol=1e-9)


def test_mlp_forward_silu_closed_form():
    # one hidden unit: y = w2 * silu(w1 x + b1) + b2
    sizes = [1, 1, 1]
    params = np.array([0.7, -0.2, 1.3, 0.4])
    x = np.array([[0.9]])
    z = 0.7 * 0.9 - 0.2
    y = 1.3 * z / (1 + math.exp(-z)) + 0.4
    assert oracle.mlp_forward(sizes, params, x)[0, 0] == pytest.approx(y, abs=1e-15)


def test_adam_first_step_is_signed_lr():
    # first Adam step: mhat = g, vhat = g^2, so p -= lr g/(|g| + eps)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    oracle.adam_update(p, g, m, v, 0.01, 0.9, 0.999, 1e-12, 1)
    assert np.allclose(p, [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], atol=1e-9)
