"""Pins of the oracle's full step (Sec. 4, 5) against the paper: the 1D growth
matrix and its eigenvalues (Sec. 5.4), the exact shift at xi = 1, exact transport
of linear data, cross-derivative reconstruction (Sec. 2.3 approach A), and the
convergence orders of Sec. 6.1.1 and 6.1.2."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs


def _growth_matrix_paper(xi, theta, h):
    """G~_{xi,h}(theta) as printed in Sec. 5.4 (f0=f(xi), f1=f(1-xi), g0=g(xi),
    g1=-g(1-xi), primes are d/dxi)."""
    f = lambda x: 1 - 3 * x * x + 2 * x ** 3
    fp = lambda x: -6 * x + 6 * x * x
    g = lambda x: x * (1 - x) ** 2
    gp = lambda x: (1 - x) ** 2 - 2 * x * (1 - x)
    f0, f1 = f(xi), f(1 - xi)
    g0, g1 = g(xi), -g(1 - xi)
    f0p, f1p = fp(xi), -fp(1 - xi)
    g0p, g1p = gp(xi), gp(1 - xi)
    E = np.exp(1j * theta)
    return np.array([[f0 + E * f1, h * (g0 + E * g1)],
                     [(f0p + E * f1p) / h, g0p + E * g1p]])


def _growth_matrix_oracle(xi, theta, n=40):
    """Apply one oracle step (constant v < 0, 1D) to the Fourier modes
    (phi, psi) = (e^{i theta j}, 0) and (0, e^{i theta j}) and read the matrix off
    an interior node."""
    h = 1.0 / (n - 1)
    dt = 0.01
    v = -xi * h / dt  # foot = x_j + xi h, i.e. in cell [x_j, x_{j+1}]
    g = oracle.grid((n,))
    vel = oracle.velocity("const", c=(v,))
    j = np.arange(n)
    G = np.zeros((2, 2), dtype=complex)
    for col in range(2):
        out = []
        for part in (np.cos, np.sin):
            st = np.zeros((2, n))
            st[col] = part(theta * j)
            out.append(oracle.step(g, vel, st, 0.0, dt))
        res = out[0] + 1j * out[1]
        jj = n // 2
        G[:, col] = res[:, jj] / np.exp(1j * theta * jj)
    return G


@pytest.mark.parametrize("xi", [0.2, 0.4, 0.6, 0.8, 0.37])
@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, 2.5, math.pi])
def test_growth_matrix_matches_paper(xi, theta):
    n = 40
    h = 1.0 / (n - 1)
    G = _growth_matrix_oracle(xi, theta, n)
    assert np.allclose(G, _growth_matrix_paper(xi, theta, h), atol=1e-11)


@pytest.mark.parametrize("xi", [0.2, 0.4, 0.6, 0.8])
def test_theta0_eigenvalues(xi, golden):
    # Sec. 5.4: at theta = 0, lambda1 = 1, lambda2 = 1 - 6 xi (1 - xi)
    G = _growth_matrix_oracle(xi, 0.0)
    lam = np.sort(np.linalg.eigvals(G).real)
    assert lam == pytest.approx(sorted([golden["stability_theta0"]["lambda1"], 1 - 6 * xi * (1 - xi)]), abs=1e-11)


@pytest.mark.parametrize("xi", [0.2, 0.4, 0.6, 0.8])
def test_eigenvalues_inside_unit_circle(xi, golden):
    # figure of Sec. 5.4: for theta != 0 both eigenvalues are strictly inside
    assert xi in golden["stability_unit_circle"]["xi_values"]
    for theta in np.linspace(-math.pi, math.pi, 41):
        if abs(theta) < 1e-12:
            continue
        lam = np.linalg.eigvals(_growth_matrix_oracle(xi, theta))
        assert np.max(np.abs(lam)) < 1.0 - 1e-6


def test_exact_shift_xi1():
    # Sec. 5.4, xi = 1: phi_j^{n+1} = phi_{j+1}^n, psi likewise -- bit-exact
    n = 65
    g = oracle.grid((n,))
    vel = oracle.velocity("const", c=(-1.0,))
    rng = np.random.default_rng(2)
    st = rng.normal(size=(2, n))
    out = oracle.step(g, vel, st, 0.0, 1.0 / 64)
    assert np.array_equal(out[:, :-1], st[:, 1:])


@pytest.mark.parametrize("dim", [2, 3])
def test_integer_cell_shift_bit_exact(dim):
    """A translation by exactly one cell per axis moves every plane by one node
    (h = 2^-6); the rebuilt cross derivatives shift too, away from the boundary."""
    n = 33 if dim == 2 else 17
    h = 1.0 / (n - 1)
    g = oracle.grid((n,) * dim)
    vel = oracle.velocity("const", c=(-1.0,) * dim)
    st = inputs.random_state((oracle.nplanes(dim),) + (n,) * dim, seed=3)
    st = oracle.recon_cross(g, st)
    out = oracle.step(g, vel, st, 0.0, h)
    ncore = 1 + dim
    if dim == 2:
        assert np.array_equal(out[:ncore, :-1, :-1], st[:ncore, 1:, 1:])
        assert np.array_equal(out[ncore:, 1:-2, 1:-2], st[ncore:, 2:-1, 2:-1])
    else:
        assert np.array_equal(out[:ncore, :-1, :-1, :-1], st[:ncore, 1:, 1:, 1:])
        assert np.array_equal(out[ncore:, 1:-2, 1:-2, 1:-2], st[ncore:, 2:-1, 2:-1, 2:-1])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("trace", ["rk3", "euler"])
def test_linear_transport_exact(dim, trace):
    """Linear phi under constant v is transported exactly; cross derivatives stay 0."""
    n = 21 if dim == 2 else 11
    g = oracle.grid((n,) * dim)
    c = np.array([0.31, -0.17, 0.23])[:dim]
    vel = oracle.velocity("const", c=tuple(c))
    a = np.array([0.3, -0.7, 0.2])[:dim]
    st = inputs.linear2d((n,) * 2, a=a) if dim == 2 else inputs.linear3d((n,) * 3, a=a)
    dt = 0.02
    out = oracle.step(g, vel, st, 0.0, dt, trace_scheme=trace)
    X = inputs.node_coords((n,) * dim)
    grids = np.meshgrid(*X[::-1], indexing="ij")[::-1]  # x fastest
    phi_exact = sum(a[i] * (grids[i] - c[i] * dt) for i in range(dim)) + 0.1
    # nodes whose foot lies inside the box
    inside = np.ones(phi_exact.shape, bool)
    for i in range(dim):
        fi = grids[i] - c[i] * dt
        inside &= (fi >= 0) & (fi <= 1)
    assert np.max(np.abs(out[0] - phi_exact)[inside]) < 1e-13
    for i in range(dim):
        assert np.max(np.abs(out[1 + i] - a[i])) < 1e-12
    assert np.max(np.abs(out[1 + dim:])) < 1e-10


def test_cross_recon_exact_on_quadratic_gradients():
    """Approach A (Sec. 2.3): central differences -- and the one-sided boundary
    stencils -- are exact when the differenced gradient is quadratic along the axis:
    phi = x^2 y^3 + x y^2 gives phi_xy exactly."""
    n = (9, 13)
    coef = np.zeros((3, 4))
    coef[2, 3] = 1.0
    coef[1, 2] = 1.0
    st = inputs.polynomial2d(n, coef)
    g = oracle.grid(n)
    pxy_exact = st[3].copy()
    st[3] = 0.0
    rec = oracle.recon_cross(g, st)
    assert np.max(np.abs(rec[3] - pxy_exact)) < 1e-12


def test_cross_recon_3d_quadratic():
    n = (7, 8, 9)
    g = oracle.grid(n)
    X, Y, Z = np.meshgrid(*inputs.node_coords(n)[::-1], indexing="ij")[::-1]
    # phi = x^2 y^2 z^3 : psi_y = 2 x^2 y z^3 (quadratic in x), psi_z = 3 x^2 y^2 z^2
    st = np.zeros((8,) + X.shape)
    st[0] = X ** 2 * Y ** 2 * Z ** 3
    st[1] = 2 * X * Y ** 2 * Z ** 3
    st[2] = 2 * X ** 2 * Y * Z ** 3
    st[3] = 3 * X ** 2 * Y ** 2 * Z ** 2
    rec = oracle.recon_cross(g, st)
    assert np.max(np.abs(rec[4] - 4 * X * Y * Z ** 3)) < 1e-12        # phi_xy
    assert np.max(np.abs(rec[5] - 6 * X * Y ** 2 * Z ** 2)) < 1e-12   # phi_xz
    assert np.max(np.abs(rec[6] - 6 * X ** 2 * Y * Z ** 2)) < 1e-12   # phi_yz
    assert np.max(np.abs(rec[7] - 12 * X * Y * Z ** 2)) < 1e-12       # phi_xyz


def test_step_nodes_equals_full_step():
    n = (23, 19)
    g = oracle.grid(n)
    vel = oracle.velocity("vortex2d", T=8.0)
    st = oracle.recon_cross(g, inputs.circle_sdf(n))
    full = oracle.step(g, vel, st, 0.3, 0.04)
    rng = np.random.default_rng(0)
    sel = np.concatenate([[0, n[0] - 1, n[0] * n[1] - 1], rng.integers(0, n[0] * n[1], 30)])
    part = oracle.step_nodes(g, vel, st, 0.3, 0.04, sel)
    flat = full.reshape(4, -1)
    assert np.array_equal(part, flat[:, sel].T)
    g3 = oracle.grid((9, 8, 7))
    vel3 = oracle.velocity("deform3d", T=3.0)
    st3 = oracle.recon_cross(g3, inputs.sphere_sdf((9, 8, 7), center=(0.4, 0.5, 0.45), r=0.3))
    full3 = oracle.step(g3, vel3, st3, 0.1, 0.05)
    sel3 = np.array([0, 5, 77, 200, 503])
    part3 = oracle.step_nodes(g3, vel3, st3, 0.1, 0.05, sel3)
    assert np.array_equal(part3, full3.reshape(8, -1)[:, sel3].T)


def _pseudo1d_solution(X, Y, t, x0=(0.5, 0.5)):
    d = np.array([math.sqrt(2), math.sqrt(math.pi)]) / math.sqrt(2 + math.pi)
    s = d[0] * X + d[1] * Y
    sf = -np.log(np.exp(-s) + t)
    dsf = np.exp(-s) / (np.exp(-s) + t)
    FX, FY = X + (sf - s) * d[0], Y + (sf - s) * d[1]
    e, gx, gy = inputs.gaussian_bump2d_exact(FX, FY, x0)
    # grad phi(x,t) = (dX/dx)^T grad phi0(X), dX/dx = I + d d^T (dsf - 1)
    m = dsf - 1
    px = gx + d[0] * m * (d[0] * gx + d[1] * gy)
    py = gy + d[1] * m * (d[0] * gx + d[1] * gy)
    return e - math.exp(-0.15 ** 2), px, py


@pytest.mark.parametrize("trace", ["rk3", "heun_psi"])
def test_local_truncation_order_pseudo1d(golden, trace):
    """Sec. 6.1.1: 16 steps with dt = h/2 on the pseudo-1D flow; the error away
    from the boundary converges with order 4 in phi and 3 in grad phi.  The
    region [0.4, 0.7]^2 is outside the numerical domain of dependence of the
    inflow edges and away from the one-sided cross stencils at the outflow edges
    (the paper asks only for a region the boundary does not influence).
    Both the superconsistent RK3 scheme and the CIR scheme with Heun's method for the
    gradients (Sec. 4: RK3 for the characteristic, Heun for eq. cir_evolution_psi) have
    these orders."""
    vel = oracle.velocity("pseudo1d")
    ephi, epsi = [], []
    for n in (129, 257, 513):
        h = 1.0 / (n - 1)
        dt = h / 2
        g = oracle.grid((n, n))
        st = oracle.recon_cross(g, inputs.gaussian_bump2d((n, n)))
        st = oracle.run(g, vel, st, 0.0, dt, 16, trace_scheme=trace)
        X, Y = np.meshgrid(*inputs.node_coords((n, n)), indexing="xy")
        ph, px, py = _pseudo1d_solution(X, Y, 16 * dt)
        region = (X >= 0.4) & (Y >= 0.4) & (X <= 0.7) & (Y <= 0.7)
        ephi.append(np.max(np.abs(st[0] - ph)[region]))
        epsi.append(max(np.max(np.abs(st[1] - px)[region]), np.max(np.abs(st[2] - py)[region])))
    o_phi = math.log2(ephi[-2] / ephi[-1])
    o_psi = math.log2(epsi[-2] / epsi[-1])
    assert golden["local_truncation_order"]["phi"] == 4
    assert o_phi >= 3.7, (ephi, o_phi)
    assert o_psi >= 2.7, (epsi, o_psi)


@pytest.mark.slow
def test_global_error_order_vortex(golden):
    """Sec. 6.1.2: vortex in a box, dt = h, T = 2: the flow returns the data; the
    error at t = T converges with order 3 in phi and 2 in grad phi."""
    vel = oracle.velocity("vortex2d", T=2.0)
    ephi, epsi = [], []
    for n in (65, 129, 257):
        h = 1.0 / (n - 1)
        g = oracle.grid((n, n))
        st0 = oracle.recon_cross(g, inputs.gaussian_bump2d((n, n), x0=(0.5, 0.75)))
        st = oracle.run(g, vel, st0, 0.0, h, int(round(2.0 / h)))
        ephi.append(oracle.emax(st[0], st0[0]))
        epsi.append(max(oracle.emax(st[1], st0[1]), oracle.emax(st[2], st0[2])))
    o_phi = math.log2(ephi[-2] / ephi[-1])
    o_psi = math.log2(epsi[-2] / epsi[-1])
    assert golden["global_error_order"] == {"cite": golden["global_error_order"]["cite"], "phi": 3, "psi": 2}
    assert o_phi >= 2.7, (ephi, o_phi)
    assert o_psi >= 1.7, (epsi, o_psi)


@pytest.mark.parametrize("dim", [2, 3])
def test_step_band_equals_full_step(dim):
    if dim == 2:
        n = (29, 23)
        st = inputs.circle_sdf(n, r=0.3, center=(0.5, 0.5))
        vel = oracle.velocity("vortex2d", T=8.0)
    else:
        n = (11, 10, 9)
        st = inputs.sphere_sdf(n, r=0.3, center=(0.5, 0.5, 0.5))
        vel = oracle.velocity("deform3d", T=3.0)
    g = oracle.grid(n)
    st = oracle.recon_cross(g, st)
    full = oracle.step(g, vel, st, 0.2, 0.03)
    outer = n[-1]
    for b0, b1 in ((0, 3), (4, outer - 1), (outer - 2, outer)):
        band = oracle.step_band(g, vel, st, 0.2, 0.03, b0, b1)
        assert np.array_equal(band, full[:, b0:b1])


def test_heun_psi_constant_velocity_equals_superconsistent():
    """With constant v, grad v = 0: the Heun gradient update is grad H(foot), the same
    as J^T grad H(foot) with J = I."""
    n = (23, 19)
    g = oracle.grid(n)
    st = oracle.recon_cross(g, inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3))
    vel = oracle.velocity("const", c=(0.4, -0.3))
    a = oracle.step(g, vel, st, 0.0, 0.03, trace_scheme="rk3")
    b = oracle.step(g, vel, st, 0.0, 0.03, trace_scheme="heun_psi")
    assert np.array_equal(a, b)


def test_heun_psi_rotation_closed_form():
    """Rigid rotation, grad v constant: Heun's method applied to d psi/d tau = B psi with
    B = -(Dv)^T gives psi+ = (I + dt B + dt^2 B^2 / 2) psi(foot); for linear phi,
    psi(foot) is the constant gradient a at every foot inside the box."""
    n = (33, 33)
    om, dt = 2 * np.pi, 0.01
    g = oracle.grid(n)
    a = np.array([0.3, -0.7])
    st = inputs.linear2d(n, a=a)
    vel = oracle.velocity("rotation", omega=om, center=(0.5, 0.5))
    out = oracle.step(g, vel, st, 0.0, dt, trace_scheme="heun_psi")
    Dv = np.array([[0.0, -om], [om, 0.0]])
    B = -Dv.T
    M = np.eye(2) + dt * B + 0.5 * dt * dt * B @ B
    want = M @ a
    X, Y = np.meshgrid(*inputs.node_coords(n), indexing="xy")
    r = np.hypot(X - 0.5, Y - 0.5)
    inside = r < 0.45   # feet stay inside the box
    assert np.max(np.abs(out[1][inside] - want[0])) < 1e-13
    assert np.max(np.abs(out[2][inside] - want[1])) < 1e-13
    # the superconsistent RK3 update differs from it by O(dt^3) here
    sc = oracle.step(g, vel, st, 0.0, dt, trace_scheme="rk3")
    d = np.max(np.abs(sc[1:3][:, inside] - out[1:3][:, inside]))
    assert 0 < d < 10 * (om * dt) ** 3


def _poly_state(n, dim):
    """A polynomial whose mixed derivatives are linear (phi_xyz constant), with exact
    value and gradient planes and zero cross planes (approach B does not read them)."""
    X = inputs.node_coords(n)
    if dim == 2:
        Y, Xg = np.meshgrid(X[1], X[0], indexing="ij")
        phi = Xg**2 * Y + 2 * Xg * Y**2 + Xg**3 - Y**3 + 0.5 * Xg * Y + 0.3 * Xg - 0.2 * Y
        px = 2 * Xg * Y + 2 * Y**2 + 3 * Xg**2 + 0.5 * Y + 0.3
        py = Xg**2 + 4 * Xg * Y - 3 * Y**2 + 0.5 * Xg - 0.2
        return np.stack([phi, px, py, np.zeros_like(phi)]), (lambda x, y: (
            x**2 * y + 2 * x * y**2 + x**3 - y**3 + 0.5 * x * y + 0.3 * x - 0.2 * y,
            2 * x * y + 2 * y**2 + 3 * x**2 + 0.5 * y + 0.3,
            x**2 + 4 * x * y - 3 * y**2 + 0.5 * x - 0.2))
    Z, Y, Xg = np.meshgrid(X[2], X[1], X[0], indexing="ij")

    def f(x, y, z):
        return (x * y * z + x**2 * y + y**2 * z + z**2 * x + x**3 - 0.5 * y**3,
                y * z + 2 * x * y + z**2 + 3 * x**2,
                x * z + x**2 + 2 * y * z - 1.5 * y**2,
                x * y + y**2 + 2 * z * x)
    p = f(Xg, Y, Z)
    return np.stack(list(p) + [np.zeros_like(p[0])] * 4), f


@pytest.mark.parametrize("dim", [2, 3])
def test_cross_cell_exact_transport(dim):
    """Sec. 2.3 approach (B): edge-centre differences are exact for mixed derivatives
    linear along the differenced direction, and the 3/4, 3/4, -1/4, -1/4 extrapolation
    is exact for linear ones (phi_xyz: the double difference is exact for a constant);
    the interpolant of such a p-cubic is then exact, and a constant velocity translates
    it exactly.  The cross planes of the new state are zero (no node value in (B))."""
    n = (17,) * dim
    g = oracle.grid(n)
    st, f = _poly_state(n, dim)
    c = np.array([0.23, -0.31, 0.17])[:dim]
    vel = oracle.velocity("const", c=tuple(c))
    dt = 0.05
    out = oracle.step(g, vel, st, 0.0, dt, cross="cell")
    X = inputs.node_coords(n)
    grids = np.meshgrid(*X[::-1], indexing="ij")[::-1]
    feet = [grids[i] - c[i] * dt for i in range(dim)]
    want = f(*feet)
    inside = np.ones(grids[0].shape, bool)
    for i in range(dim):
        inside &= (feet[i] >= 0) & (feet[i] <= 1)
    for p in range(1 + dim):
        assert np.max(np.abs(out[p] - want[p])[inside]) < 1e-12, p
    assert not np.any(out[1 + dim:])


def test_cross_cell_converges_to_central():
    """On smooth data the two approaches differ by O(h^2) in the cross derivatives,
    hence by O(h^4) in the interpolated value: one step from the same state, difference
    ratio about 16 per halving of h (accept >= 8)."""
    diffs = []
    vel = oracle.velocity("vortex2d", T=8.0)
    for n in (33, 65):
        g = oracle.grid((n, n))
        st = oracle.recon_cross(g, inputs.gaussian_bump2d((n, n), x0=(0.5, 0.5)))
        h = 1.0 / (n - 1)
        a = oracle.step(g, vel, st, 0.3, h, cross="central")
        b = oracle.step(g, vel, st, 0.3, h, cross="cell")
        inner = (slice(4, -4), slice(4, -4))
        diffs.append(np.max(np.abs(a[0][inner] - b[0][inner])))
    assert diffs[0] / diffs[1] >= 8.0, diffs


def test_cross_cell_diagnostics():
    """The diagnostics of a grid using approach (B) sample the cell-based interpolant: for
    a p-cubic with linear mixed derivatives it is exact, so the sampled area of {phi < c}
    matches that of the exact data with approach (A); with zero cross planes and
    approach (A) it does not."""
    n = (33, 33)
    st, f = _poly_state(n, 2)
    st = st.copy()
    st[0] -= 0.3
    ga = oracle.grid(n)
    gb = oracle.grid(n, cross="cell")
    exact = oracle.recon_cross(ga, st)      # exact cross planes of the polynomial (A is exact here)
    area_a = oracle.measure_negative(ga, exact, 4)
    area_b = oracle.measure_negative(gb, st, 4)  # cross planes zero, rebuilt per cell
    assert area_b == area_a
    # pointwise: the cell-based interpolant equals the exact one; zero cross planes do not
    pts = np.random.default_rng(3).uniform(0.0, 1.0, (200, 2))
    ha, _ = oracle.eval_points(ga, exact, pts)
    hb, _ = oracle.eval_points(gb, st, pts)
    hz, _ = oracle.eval_points(ga, st, pts)
    x, y = pts[:, 0], pts[:, 1]
    want = f(x, y)[0] - 0.3
    assert np.max(np.abs(hb - want)) < 1e-13 and np.max(np.abs(ha - want)) < 1e-13
    assert np.max(np.abs(hz - want)) > 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_step_given_affine_map_exact(dim):
    """A step fed a backward map instead of a trace (the form the learned flow map
    uses): for linear phi = a.x + b and the affine map foot = A x + d, the interpolant
    reproduces phi exactly (Sec. 2.3), so phi+ = a.(A x + d) + b and psi+ = A^T a
    (eq. superconsistency with J = A).  A is not symmetric, so a transposed J fails."""
    n = (9, 8, 7)[:dim]
    g = oracle.grid(n)
    rng = np.random.default_rng(21)
    a = rng.uniform(-1, 1, dim)
    b = 0.3
    A = np.eye(dim) + 0.1 * rng.uniform(-1, 1, (dim, dim))
    d = rng.uniform(-0.01, 0.01, dim)
    axes = [np.linspace(0, 1, m) for m in n]
    X = np.stack(np.meshgrid(*axes[::-1], indexing="ij")[::-1])  # X[c] = coordinate c, x fastest
    st = np.zeros((oracle.nplanes(dim),) + tuple(n[::-1]))
    st[0] = np.tensordot(a, X, 1) + b
    for c in range(dim):
        st[1 + c] = a[c]
    # a contraction about the centre keeps every foot inside the box
    A = 0.7 * A
    foot = np.tensordot(A, X - 0.5, 1) + (0.5 + d).reshape((dim,) + (1,) * dim)
    assert foot.min() >= 0 and foot.max() <= 1
    disp = foot - X
    jac = np.broadcast_to(A.reshape((dim, dim) + (1,) * dim), (dim, dim) + tuple(n[::-1]))
    out = oracle.step_given(g, st, disp, jac)
    assert np.allclose(out[0], np.tensordot(a, foot, 1) + b, atol=1e-13)
    for c in range(dim):
        assert np.allclose(out[1 + c], (A.T @ a)[c], atol=1e-13)
    assert np.allclose(out[1 + dim:], 0.0, atol=1e-9)  # mixed derivatives of linear data


@pytest.mark.parametrize("dim,kind,kw", [(2, "vortex2d", dict(T=8.0)), (3, "deform3d", dict(T=3.0))])
def test_step_given_with_traced_map_equals_step(dim, kind, kw):
    """Fed the RK3 trace's own feet and Jacobians, the given-map step is the RK3 step."""
    n = (13, 11, 9)[:dim]
    g = oracle.grid(n)
    st = inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.25) if dim == 3 else \
        inputs.circle_sdf(n, center=(0.45, 0.55), r=0.25)
    st = oracle.recon_cross(g, np.asarray(st, dtype=np.float64))
    vel = oracle.velocity(kind, **kw)
    t, dt = 0.3, 0.07
    ref = oracle.step(g, vel, st, t, dt)
    disp = np.zeros((dim,) + tuple(n[::-1]))
    jac = np.zeros((dim, dim) + tuple(n[::-1]))
    for idx in np.ndindex(*n[::-1]):
        x = np.array([idx[::-1][c] / (n[c] - 1) for c in range(dim)])
        foot, J = oracle.trace("rk3", vel, dim, x, t, dt)
        disp[(slice(None),) + idx] = foot - x
        jac[(slice(None), slice(None)) + idx] = J
    out = oracle.step_given(g, st, disp, jac)
    assert np.max(np.abs(out - ref)) < 1e-12
