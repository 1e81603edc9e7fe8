"""Pins of the oracle's Hermite interpolant (Sec. 2.3) against facts the paper and
plain mathematics fix: basis identities, partition of unity, exact reproduction
of p-cubic polynomials (Theorem in Sec. 2.3), the 1D midpoint value of eq.
Hermite_cubic_1D and the subgrid drop/jet/film data of Sec. 3.1."""
import itertools

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle


def test_basis_identities():
    # f(0)=1, f(1)=0, f'(0)=f'(1)=0, g(0)=g(1)=0, g'(0)=1, g'(1)=0 (eq. 1-cubic_basis_functions)
    w0, dw0 = oracle.basis1d(0.0)
    w1, dw1 = oracle.basis1d(1.0)
    # index v*2+a: (v=0,a=0) f(x), (0,1) g(x), (1,0) f(1-x), (1,1) -g(1-x)
    # value/derivative at the vertex they belong to is 1 for exactly one type
    assert np.allclose(w0, [1, 0, 0, 0]) and np.allclose(dw0, [0, 1, 0, 0])
    assert np.allclose(w1, [0, 0, 1, 0]) and np.allclose(dw1, [0, 0, 0, 1])
    xs = np.linspace(0, 1, 11)
    for x in xs:
        w, dw = oracle.basis1d(x)
        f = 1 - 3 * x * x + 2 * x ** 3
        g = x * (1 - x) ** 2
        assert np.allclose(w, [f, g, 1 - 3 * (1 - x) ** 2 + 2 * (1 - x) ** 3, -(1 - x) * x * x])
        # partition of unity of the value basis
        assert abs(w[0] + w[2] - 1.0) < 1e-15


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_partition_of_unity(dim):
    np_ = 2 ** dim
    data = np.zeros(4 ** dim)
    for v in range(np_):
        data[v * np_ + 0] = 1.0
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.uniform(0, 1, dim)
        H, g = oracle.hermite_cell(dim, data, [0.3, 0.7, 1.9][:dim], xi)
        assert abs(H - 1.0) < 1e-14
        assert np.max(np.abs(g)) < 1e-13


def _poly_data(coef, dim, origin, h):
    """cell data phi_a^v = d^a p(x_v) of a p-cubic polynomial, computed with
    numpy.polynomial (independent of the oracle)."""
    np_ = 2 ** dim
    data = np.zeros(4 ** dim)
    for v in range(np_):
        x = [origin[i] + h[i] * ((v >> i) & 1) for i in range(dim)]
        for a in range(np_):
            c = coef
            for i in range(dim):
                if (a >> i) & 1:
                    c = P.polyder(c, axis=i)
            data[v * np_ + a] = _polyval(c, x)
    return data


def _polyval(c, x):
    if len(x) == 1:
        return P.polyval(x[0], c)
    if len(x) == 2:
        return P.polyval2d(x[0], x[1], c)
    return P.polyval3d(x[0], x[1], x[2], c)


def _polygrad(c, x):
    return [_polyval(P.polyder(c, axis=i), x) for i in range(len(x))]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_exact_pcubic_reproduction(dim):
    """Theorem (Sec. 2.3): a p-cubic is reproduced exactly from its 4^p data, on
    rectangular cells too (h^|a| -> prod h_i^a_i)."""
    rng = np.random.default_rng(100 + dim)
    for trial in range(5):
        coef = rng.normal(size=(4,) * dim)
        origin = rng.uniform(-1, 1, dim)
        h = rng.uniform(0.05, 0.8, dim)
        data = _poly_data(coef, dim, origin, h)
        for _ in range(10):
            xi = rng.uniform(0, 1, dim)
            x = origin + h * xi
            H, g = oracle.hermite_cell(dim, data, h, xi)
            assert H == pytest.approx(_polyval(coef, x), abs=1e-11)
            assert np.allclose(g, _polygrad(coef, x), atol=1e-10)


def test_degree4_not_reproduced():
    """Control: a quartic term is NOT reproduced, so the exactness test has teeth."""
    coef = np.zeros(5)
    coef[4] = 1.0
    data = np.array([0.0, 0.0, 1.0, 4.0])  # x^4 on [0,1]: p(0)=0, p'(0)=0, p(1)=1, p'(1)=4
    H, g = oracle.hermite_cell(1, data, [1.0], [0.5])
    assert abs(H - 0.5 ** 4) > 1e-3


def test_hermite_1d_midpoint(golden):
    # eq. Hermite_cubic_1D at xi = 1/2: (phi0+phi1)/2 + h (psi0 - psi1)/8
    rng = np.random.default_rng(5)
    for _ in range(10):
        p0, p1, s0, s1 = rng.normal(size=4)
        h = rng.uniform(0.01, 2.0)
        H, _ = oracle.hermite_cell(1, [p0, s0, p1, s1], [h], [0.5])
        assert H == pytest.approx((p0 + p1) / 2 + h * (s0 - s1) / 8, abs=1e-14)
    assert "Hermite_cubic_1D" in golden["hermite_1d_midpoint"]["cite"]


@pytest.mark.parametrize("structure", ["drop", "jet", "film"])
@pytest.mark.parametrize("h", [1.0, 0.1, 1.0 / 64])
def test_subgrid_structures(structure, h, golden):
    """Sec. 3.1: phi = 0.1 on the vertices plus the printed gradients gives a
    structure inside the cell: H(centre) = 0.1 - 1/8 < 0 while H > 0 at vertices."""
    gv = golden["subgrid_structures"]
    data = np.zeros(64)
    for v in range(8):
        vv = np.array([(v >> i) & 1 for i in range(3)], dtype=float)
        if structure == "drop":
            psi = (vv - 0.5) / (3 * h)
        elif structure == "jet":
            psi = np.array([0.0, vv[1] - 0.5, vv[2] - 0.5]) / (2 * h)
        else:
            psi = np.array([0.0, vv[1] - 0.5, 0.0]) / h
        data[v * 8 + 0] = gv["phi_at_vertices"]
        data[v * 8 + 1] = psi[0]
        data[v * 8 + 2] = psi[1]
        data[v * 8 + 4] = psi[2]
    H, g = oracle.hermite_cell(3, data, [h, h, h], [0.5, 0.5, 0.5])
    assert H == pytest.approx(gv["derived_center_value"], abs=1e-13)
    assert np.max(np.abs(g)) < 1e-10  # symmetric structure: centre is a critical point
    for v in range(8):
        corner = [(v >> i) & 1 for i in range(3)]
        Hc, _ = oracle.hermite_cell(3, data, [h, h, h], corner)
        assert Hc == pytest.approx(0.1, abs=1e-14)
