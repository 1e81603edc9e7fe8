"""GPU parity at the benchmark sizes: the 4096^2 single-vortex case and the 512^3
deformation case, run with the kernels and launch shapes the benchmark times, checked
against the FP64 oracle on windows of the grid.

One step of the GPU state (widened to FP64) by the oracle needs, at a node, only the
state within a few cells (CFL 1: the foot is at most one cell away, its cell one more,
and the approach-A stencil of the mixed derivatives one more).  So each window (random
places, tile edges of the step kernel, edges and corners of the box, the interface) is
advanced by the oracle on a grid of its own with the same spacing and origin, and the
GPU's new state is compared on the window's interior (a margin of MARGIN nodes from
window edges that are not box edges): max |dphi| <= 1e-5, max |dpsi| <= 1e-4, and the
mixed derivatives against the oracle's approach-A reconstruction of the GPU's own new
gradients."""
import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_PSI = 1e-5, 1e-4
MARGIN = 4


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def _windows(n, size, picks):
    """Clip windows of `size` nodes per axis centred on the given node indices."""
    out = []
    for c in picks:
        lo = [min(max(int(c[a]) - size // 2, 0), n[a] - size) for a in range(len(n))]
        out.append(tuple((lo[a], lo[a] + size) for a in range(len(n))))
    return out


def _check_windows(G, g, before, after, n, vel_o, t, dt, windows):
    """before/after: device tensors (planes, [z,] y, x) of the GPU state."""
    dim = len(n)
    core = 1 + dim
    h = 1.0 / (n[0] - 1)
    worst = [0.0, 0.0, 0.0]
    for win in windows:
        # tensor index order is (plane, [z,] y, x); win is per axis (x, y[, z])
        sl = (slice(None),) + tuple(slice(win[a][0], win[a][1]) for a in reversed(range(dim)))
        b = before[sl].double().cpu().numpy()
        a_ = after[sl].double().cpu().numpy()
        wn = tuple(win[a][1] - win[a][0] for a in range(dim))
        og = oracle.grid(wn, lo=[win[a][0] * h for a in range(dim)],
                         hi=[(win[a][1] - 1) * h for a in range(dim)])
        ref = oracle.step(og, vel_o, b, t, dt)
        rec = oracle.recon_cross(og, a_)
        inner = (slice(None),) + tuple(
            slice(0 if win[a][0] == 0 else MARGIN, wn[a] if win[a][1] == n[a] else wn[a] - MARGIN)
            for a in reversed(range(dim)))
        dphi = np.max(np.abs(a_[0][inner[1:]] - ref[0][inner[1:]]))
        dpsi = np.max(np.abs(a_[1:core][inner] - ref[1:core][inner]))
        scale = np.max(np.abs(rec[core:][inner])) + 1.0
        maxpsi = np.max(np.abs(a_[1:core][inner]))
        cr_tol = 2e-6 * scale + 1e-6 * maxpsi * (1.0 / h if dim == 2 else 1.0 / h ** 2)
        dcr = np.max(np.abs(a_[core:][inner] - rec[core:][inner]))
        assert dphi <= TOL_PHI, (win, dphi)
        assert dpsi <= TOL_PSI, (win, dpsi)
        assert dcr <= cr_tol, (win, dcr, cr_tol)
        worst = [max(worst[0], dphi), max(worst[1], dpsi), max(worst[2], dcr)]
    return worst


def test_vortex4096_windows(G):
    """4096^2 nodes, circle SDF r = 0.15 at (0.5, 0.75), single vortex T = 8, dt = h."""
    import torch
    n = (4096, 4096)
    h = 1.0 / 4095
    dt = h
    g = G.Grid(n)
    g.set_state(inputs.circle_sdf(n).astype(np.float32), t0=0.0, recon=True)
    vel = G.Velocity("vortex2d", T=8.0)
    g.step(vel, dt, 3)
    before = torch.empty((4,) + n[::-1], device="cuda")
    after = torch.empty_like(before)
    g.read_state(before)
    t = g.time
    g.step(vel, dt, 1)
    g.read_state(after)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4096)
    picks = [rng.integers(0, 4096, 2) for _ in range(10)]
    picks += [(128 * k, 12 * m) for k, m in ((5, 40), (16, 170), (31, 300))]   # tile edges
    picks += [(0, 0), (4095, 0), (0, 4095), (4095, 4095), (2048, 0), (0, 2048), (4095, 1000)]
    for ang in (0.3, 1.9, 3.5, 5.0):                                         # interface
        picks.append((int((0.5 + 0.15 * np.cos(ang)) * 4095), int((0.75 + 0.15 * np.sin(ang)) * 4095)))
    w = _check_windows(G, g, before, after, n, oracle.velocity("vortex2d", T=8.0), t, dt,
                       _windows(n, 16 + 2 * MARGIN, picks))
    print("vortex4096 worst |dphi| |dpsi| |dcross|:", w)
    g.close()


def test_deform512_windows(G):
    """512^3 nodes, sphere SDF r = 0.15 at (0.35, 0.35, 0.35), deformation T = 3,
    dt = h/2 (max |v_i| = 2)."""
    import torch
    n = (512, 512, 512)
    h = 1.0 / 511
    dt = h / 2
    g = G.Grid(n)
    g.set_state(inputs.sphere_sdf(n, dtype=np.float32), t0=0.0, recon=True)
    vel = G.Velocity("deform3d", T=3.0)
    g.step(vel, dt, 2)
    before = torch.empty((8,) + n[::-1], device="cuda")
    after = torch.empty_like(before)
    g.read_state(before)
    t = g.time
    g.step(vel, dt, 1)
    g.read_state(after)
    torch.cuda.synchronize()
    rng = np.random.default_rng(512)
    picks = [rng.integers(0, 512, 3) for _ in range(6)]
    picks += [(32 * 5, 4 * 30, 4 * 70), (32 * 11, 4 * 101, 4 * 3)]          # tile edges
    picks += [(0, 0, 0), (511, 511, 511), (0, 511, 256), (256, 0, 511)]     # corners, edges
    for ang in (0.4, 2.2):                                                  # interface
        c = 0.35 + 0.15 * np.array([np.cos(ang), np.sin(ang), 0.0])
        picks.append(tuple(int(v * 511) for v in c))
    w = _check_windows(G, g, before, after, n, oracle.velocity("deform3d", T=3.0), t, dt,
                       _windows(n, 8 + 2 * MARGIN, picks))
    print("deform512 worst |dphi| |dpsi| |dcross|:", w)
    g.close()
