"""GPU parity of the GALS step (through the C ABI) against the FP64 oracle.

Per step, the GPU's FP32 state is widened to FP64, advanced one step by the oracle,
and compared with the GPU's next state: max |dphi| <= 1e-5 and max |dpsi| <= 1e-4 on
O(1)-scaled fields.  Mixed derivatives are checked against the oracle's approach-A
reconstruction of the GPU's own new gradients (tight) and against the oracle step
(bound 4 eps_psi / h that the stencils imply).
"""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_PSI = 1e-5, 1e-4


@pytest.fixture(scope="module")
def gals():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals as G
    return G


def _ovel(kind, **kw):
    return oracle.velocity(kind, **kw)


def _gvel(G, kind, trace="rk3", **kw):
    return G.Velocity(kind, trace=trace, **kw)


def check_step(G, n, state, kind, dt, t0=0.0, steps=1, layout="full", trace="rk3",
               lo=None, hi=None, recon=False, cross="central", **vkw):
    """Advance `steps` steps on the GPU and check each against one oracle step."""
    g = G.Grid(n, lo=lo, hi=hi, layout=layout, cross=cross)
    g.set_state(state.astype(np.float32), t0=t0, recon=recon)
    og = oracle.grid(n, lo=lo, hi=hi, cross=cross)
    ov = _ovel(kind, **vkw)
    gv = _gvel(G, kind, trace=trace, **vkw)
    worst = [0.0, 0.0, 0.0]
    h = min(og.h[i] for i in range(len(n)))
    core = 1 + len(n)
    for _ in range(steps):
        before = g.read_state().astype(np.float64)
        t = g.time
        g.step(gv, dt, 1)
        after = g.read_state().astype(np.float64)
        ref = oracle.step(og, ov, before, t, dt, trace_scheme=trace, cross=cross)
        dphi = np.max(np.abs(after[0] - ref[0]))
        dpsi = np.max(np.abs(after[1:core] - ref[1:core]))
        assert dphi <= TOL_PHI, dphi
        assert dpsi <= TOL_PSI, dpsi
        if cross == "cell":
            # approach B keeps no node values of the mixed derivatives
            assert not np.any(after[core:]) and not np.any(ref[core:])
            worst = [max(worst[0], dphi), max(worst[1], dpsi), 0.0]
            continue
        # mixed derivatives: exact stencil arithmetic on the GPU's own gradients
        rec = oracle.recon_cross(og, after)
        scale = np.max(np.abs(rec[core:])) + 1.0
        dcr = np.max(np.abs(after[core:] - rec[core:]))
        # FP32 rounding of differences of psi (and, for phi_xyz, of differences of the
        # rounded y-differences) amplified by the 1/(2h) factors
        maxpsi = np.max(np.abs(after[1:core]))
        cr_tol = 2e-6 * scale + 1e-6 * maxpsi * (1.0 / h if len(n) == 2 else 1.0 / h ** 2)
        assert dcr <= cr_tol, (dcr, cr_tol)
        dcr_ref = np.max(np.abs(after[core:] - ref[core:]))
        # stencil amplification of a gradient difference: 4/h (one-sided first
        # derivative), 16/h^2 for the 3D double difference phi_xyz
        amp = 4.0 / h if len(n) == 2 else max(4.0 / h, 16.0 / h ** 2)
        assert dcr_ref <= amp * max(dpsi, 1e-7) + 2e-6 * scale
        worst = [max(worst[0], dphi), max(worst[1], dpsi), max(worst[2], dcr)]
    g.close()
    return worst


def test_config1_vortex_64(gals):
    """64x64 nodes, circle SDF, exact gradient, phi_xy = 0 (given, not rebuilt)."""
    n = (64, 64)
    w = check_step(gals, n, inputs.circle_sdf(n), "vortex2d", 1.0 / 63, steps=4, T=8.0)
    print("config1 worst", w)


@pytest.mark.parametrize("layout", ["full", "compact"])
@pytest.mark.parametrize("n", [(37, 29), (130, 67), (4, 4), (5, 257)])
def test_ragged_sizes_vortex(gals, n, layout):
    st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3)
    check_step(gals, n, st, "vortex2d", 0.7 / (max(n) - 1), t0=0.37, steps=2, layout=layout,
               recon=True, T=8.0)


@pytest.mark.parametrize("trace", ["rk3", "euler", "heun_psi"])
def test_rotation_slotted_disk(gals, trace):
    n = (96, 96)
    st = inputs.slotted_disk_sdf(n)
    check_step(gals, n, st, "rotation", (1.0 / 95) / math.pi, steps=2, trace=trace, recon=True,
               omega=2 * math.pi, center=(0.5, 0.5))


def test_pseudo1d_gaussian_rectangular_cells(gals):
    n = (48, 33)
    lo, hi = (0.1, -0.2), (1.3, 0.9)
    st = inputs.gaussian_bump2d(n, x0=(0.6, 0.3), lo=lo, hi=hi)
    check_step(gals, n, st, "pseudo1d", 0.01, steps=2, lo=lo, hi=hi)


@pytest.mark.parametrize("trace", ["rk3", "heun_psi"])
def test_fourier_time_periodic(gals, trace):
    n = (80, 80)
    modes = inputs.fourier_modes(16, seed=5, periodic=True)
    st = inputs.ellipse_sdf(n, (0.5, 0.5), 0.2, 0.1, 0.4)
    vmax = inputs.fourier_speed_bound(modes)
    check_step(gals, n, st, "fourier2d", (1.0 / 79) / vmax, t0=0.3, steps=2, recon=True, modes=modes,
               trace=trace)


@pytest.mark.parametrize("layout", ["full", "compact"])
def test_vortex_heun_psi(gals, layout):
    """The CIR form with Heun's method for the gradients (time-dependent field: the foot's
    velocity gradient is taken at time t, the node's at t + dt)."""
    n = (67, 45)
    st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3)
    check_step(gals, n, st, "vortex2d", 0.8 / 66, t0=0.9, steps=2, layout=layout, trace="heun_psi",
               recon=True, T=8.0)


def test_random_state_high_cfl(gals):
    """Random data and CFL ~2 (feet two cells away): stencil reach is not limited.
    The random values are scaled like a smooth O(1) field sampled on the grid:
    phi ~ h, psi ~ 1, phi_xy ~ 1/h."""
    n = (70, 45)
    h = 1.0 / 69
    st = inputs.random_state((4,) + n[::-1], seed=11)
    st[0] *= h
    st[3] /= h
    check_step(gals, n, st, "const", 0.03, steps=1, c=(1.9, -1.4, 0))


@pytest.mark.parametrize("layout", ["full", "compact"])
@pytest.mark.parametrize("n", [(21, 18, 17), (33, 9, 12), (4, 4, 4), (5, 4, 6), (37, 5, 4)])
def test_3d_deform(gals, n, layout):
    st = inputs.sphere_sdf(n, center=(0.4, 0.45, 0.5), r=0.25)
    check_step(gals, n, st, "deform3d", 0.5 / (max(n) - 1), t0=0.2, steps=2, layout=layout,
               recon=True, T=3.0)


@pytest.mark.parametrize("layout", ["full", "compact"])
def test_3d_deform_heun_psi(gals, layout):
    n = (19, 17, 16)
    st = inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.25)
    check_step(gals, n, st, "deform3d", 0.5 / 18, t0=0.4, steps=2, layout=layout, trace="heun_psi",
               recon=True, T=3.0)


def test_3d_rotation_cube(gals):
    n = (24, 24, 20)
    st = inputs.cube_sdf(n, center=(0.5, 0.6, 0.5), half=0.2)
    check_step(gals, n, st, "rotation", 0.01, steps=1, recon=True, omega=2 * math.pi,
               center=(0.5, 0.5, 0.5))


@pytest.mark.parametrize("layout", ["full", "compact"])
def test_3d_zalesak_sphere_rotation(gals, layout):
    """Zalesak's slotted sphere (Sec. 6.2.3) in rigid rotation about the z-axis, CFL 0.9."""
    n = (26, 24, 20)
    st = inputs.slotted_sphere_sdf(n, center=(0.5, 0.7, 0.5), r=0.2, slot_w=0.1, slot_top=0.8)
    check_step(gals, n, st, "rotation", 0.9 / (25 * math.pi), t0=0.1, steps=3, layout=layout,
               recon=True, omega=2 * math.pi, center=(0.5, 0.5, 0.5))


def test_3d_gaussian_explicit_cross(gals):
    n = (16, 17, 18)
    st = inputs.gaussian_bump3d(n)
    check_step(gals, n, st, "const", 0.02, steps=1, c=(0.3, -0.5, 0.7))


@pytest.mark.parametrize("layout", ["full", "compact"])
def test_vortex_cross_cell(gals, layout):
    """Mixed derivatives by approach (B) (Sec. 2.3), per cell from the vertices' gradients."""
    n = (61, 47)
    st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3)
    check_step(gals, n, st, "vortex2d", 0.9 / 60, t0=0.5, steps=3, layout=layout, cross="cell",
               T=8.0)


@pytest.mark.parametrize("layout", ["full", "compact"])
def test_3d_deform_cross_cell(gals, layout):
    n = (19, 18, 17)
    st = inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.25)
    check_step(gals, n, st, "deform3d", 0.5 / 18, t0=0.3, steps=2, layout=layout, cross="cell", T=3.0)


def test_random_state_cross_cell_high_cfl(gals):
    """Approach (B) with feet two cells away (global-memory gathers) and random data."""
    n = (40, 33)
    h = 1.0 / 39
    st = inputs.random_state((4,) + n[::-1], seed=12)
    st[0] *= h
    check_step(gals, n, st, "const", 0.05, steps=1, cross="cell", c=(1.7, -1.2, 0))


@pytest.mark.parametrize("dim", [2, 3])
def test_diagnostics_cross_cell(gals, dim):
    """The diagnostics sample the approach-(B) interpolant, like the oracle's."""
    n = (48, 40) if dim == 2 else (20, 18, 16)
    st = inputs.circle_sdf(n, r=0.3, center=(0.5, 0.5)) if dim == 2 else inputs.sphere_sdf(
        n, center=(0.5, 0.5, 0.5), r=0.3)
    g = gals.Grid(n, cross="cell")
    g.set_state(st.astype(np.float32))
    d = g.diagnostics(q=4)
    gs = g.read_state().astype(np.float64)
    og = oracle.grid(n, cross="cell")
    area = oracle.measure_negative(og, gs, 4)
    cell = np.prod([1.0 / (v - 1) for v in n]) / 4 ** dim
    assert abs(d["measure_negative"] - area) <= 16 * cell, (d["measure_negative"], area)
    # the state keeps no mixed-derivative planes under approach (B)
    assert not np.any(gs[1 + dim:])
