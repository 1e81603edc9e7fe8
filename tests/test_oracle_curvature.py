"""Pins of the oracle's derivative quantities (Sec. 3.4 "Approximation of derivative
quantities", Sec. 6.1.3 "Accuracy of curvature"): second derivatives of the p-cubic
interpolant reproduce p-cubic polynomials exactly, and normals and curvature recovered
from grid data of phi and grad phi converge at the orders the paper states (curvature
second order, everywhere in the domain)."""
import numpy as np
import numpy.polynomial.polynomial as npoly
import pytest

import oracle
from paper_0905_3409_gb300 import inputs


def _poly_derivs(c, dim):
    """{multi-index: coefficient array of that derivative} for a tensor polynomial c."""
    out = {}
    for a in range(1 << dim):
        d = c
        for ax in range(dim):
            if (a >> ax) & 1:
                d = npoly.polyder(d, axis=ax)
        out[a] = d
    return out


def _polyval(c, x):
    return npoly.polyval2d(x[0], x[1], c) if len(x) == 2 else npoly.polyval3d(x[0], x[1], x[2], c)


@pytest.mark.parametrize("dim", [2, 3])
def test_second_derivatives_exact_for_pcubic(dim):
    """Thm. p-cubic accuracy: the interpolant of a p-cubic's 4^p data is that p-cubic, so
    its Hessian is the polynomial's Hessian (derivatives taken by numpy, not by the oracle)."""
    rng = np.random.default_rng(11 + dim)
    for _ in range(5):
        c = rng.normal(size=(4,) * dim)                  # degree <= 3 in each variable
        x0 = rng.uniform(-1, 1, dim)
        h = rng.uniform(0.05, 0.3, dim)
        der = _poly_derivs(c, dim)
        np_ = 1 << dim
        data = np.zeros(np_ * np_)
        for v in range(np_):
            corner = [x0[i] + h[i] * ((v >> i) & 1) for i in range(dim)]
            for a in range(np_):
                data[v * np_ + a] = _polyval(der[a], corner)
        xi = rng.uniform(0, 1, dim)
        x = x0 + xi * h
        H, G, Hs = oracle.hermite_cell2(dim, data, h, xi)
        assert H == pytest.approx(_polyval(c, x), rel=1e-11, abs=1e-11)
        for j in range(dim):
            assert G[j] == pytest.approx(_polyval(npoly.polyder(c, axis=j), x), rel=1e-10, abs=1e-9)
            for k in range(dim):
                cjk = npoly.polyder(npoly.polyder(c, axis=j), axis=k)
                assert Hs[j, k] == pytest.approx(_polyval(cjk, x), rel=1e-9, abs=1e-8)


def _order(errors, hs):
    return [np.log(errors[i] / errors[i + 1]) / np.log(hs[i] / hs[i + 1]) for i in range(len(errors) - 1)]


def test_curvature_second_order_E3():
    """Sec. 6.1.3: phi = ((x-2)(y-x))^3 on [0,1]^2, phi and grad phi at the grid points, the
    cross derivatives reconstructed from them (approach A), curvature from the interpolant
    everywhere; L-infinity error on a fixed finer sampling, second order.  grad phi
    vanishes on y = x (phi has a triple zero there, its level sets are those of
    u = (x-2)(y-x), so the curvature is that of u, finite), and the formula's division by
    |grad phi|^3 ~ u^6 amplifies the interpolation error next to that line; the sampling
    keeps |y - x| >= 0.2."""
    def u(x, y):
        return (x - 2.0) * (y - x)

    def kappa_exact(x, y):   # curvature of the level sets of u (= those of phi = u^3)
        ux, uy, uxx, uxy, uyy = y - 2.0 * x + 2.0, x - 2.0, -2.0, 1.0, 0.0
        return (uxx * uy ** 2 - 2 * ux * uy * uxy + uyy * ux ** 2) / (ux ** 2 + uy ** 2) ** 1.5

    s = np.linspace(0.0, 1.0, 61)
    X, Y = np.meshgrid(s, s)
    keep = np.abs(Y - X) >= 0.2
    pts = np.stack([X[keep], Y[keep]], axis=1)
    errs, hs = [], []
    for n in (17, 33, 65, 129):
        g = oracle.grid((n, n))
        xs = np.linspace(0.0, 1.0, n)
        gx, gy = np.meshgrid(xs, xs)
        uu = u(gx, gy)
        st = np.zeros((4, n, n))
        st[0] = uu ** 3
        st[1] = 3 * uu ** 2 * (gy - 2 * gx + 2)
        st[2] = 3 * uu ** 2 * (gx - 2)
        st = oracle.recon_cross(g, st)
        _, _, K = oracle.curvature_points(g, st, pts)
        errs.append(np.max(np.abs(K - kappa_exact(pts[:, 0], pts[:, 1]))))
        hs.append(1.0 / (n - 1))
    orders = _order(errs, hs)
    assert min(orders) >= 1.7, (errs, orders)


@pytest.mark.parametrize("dim", [2, 3])
def test_sdf_normal_and_curvature_orders(dim):
    """Signed distance to a circle / sphere: n = (x - c)/|x - c| and kappa = (p - 1)/|x - c|
    exactly; from grid data (phi, exact grad phi, cross derivatives by approach A) the
    normal converges at third order (first derivatives, Thm. p-cubic accuracy) and the
    curvature at second order (Sec. 3.4), away from the centre's kink."""
    c = np.array([0.5, 0.5, 0.5][:dim])
    rng = np.random.default_rng(5)
    d = rng.normal(size=(400, dim))
    d /= np.linalg.norm(d, axis=1)[:, None]
    rad = rng.uniform(0.15, 0.3, 400)
    pts = c + d * rad[:, None]
    sizes = (17, 33, 65) if dim == 2 else (17, 33)
    en, ek, hs = [], [], []
    for n in sizes:
        shape = (n,) * dim
        g = oracle.grid(shape)
        st = inputs.circle_sdf(shape, center=tuple(c), r=0.2) if dim == 2 else \
            inputs.sphere_sdf(shape, center=tuple(c), r=0.2)
        st = oracle.recon_cross(g, st.astype(np.float64))
        _, N, K = oracle.curvature_points(g, st, pts)
        en.append(np.max(np.abs(N - d)))
        ek.append(np.max(np.abs(K - (dim - 1) / rad)))
        hs.append(1.0 / (n - 1))
    assert min(_order(en, hs)) >= 2.7, (en, _order(en, hs))
    assert min(_order(ek, hs)) >= 1.7, (ek, _order(ek, hs))
