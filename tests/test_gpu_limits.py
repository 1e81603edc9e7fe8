"""The largest grids the C ABI accepts, stepped on the GPU and checked against the FP64
oracle (per step max |dphi| <= 1e-5, max |dpsi| <= 1e-4, mixed derivatives against the
oracle's approach-A reconstruction of the GPU's own gradients).

* 2D with n[1] = 917490 rows: 65535 tiles of 14 rows, the most the launch grid's y
  dimension holds (5 columns; a strip of square cells across the single vortex).
* 3D with n[1] = 262140 or n[2] = 262140 levels: 65535 tiles of 4 (4 x 4 nodes across; a
  strip of cubic cells through the deformation field's sphere).
* 2D with 46340 x 46340 nodes: 2,147,395,600 per plane, just under the 2^31 - 1 elements
  a plane may hold (34 GB per state buffer, 4 planes): plane offsets past 2^31 elements.
  Built on the device; checked on windows as at the benchmark size (a node's new state
  depends on the state within three cells only); the diagnostics (area of {phi < 0}) and
  the point evaluation run on the whole grid."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_PHI, TOL_PSI = 1e-5, 1e-4


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def _compare(after, ref, og, h):
    core = 1 + og.dim
    dphi = np.max(np.abs(after[0] - ref[0]))
    dpsi = np.max(np.abs(after[1:core] - ref[1:core]))
    rec = oracle.recon_cross(og, after)
    scale = np.max(np.abs(rec[core:])) + 1.0
    maxpsi = np.max(np.abs(after[1:core]))
    cr_tol = 2e-6 * scale + 1e-6 * maxpsi * (1.0 / h if og.dim == 2 else 1.0 / h ** 2)
    dcr = np.max(np.abs(after[core:] - rec[core:]))
    assert dphi <= TOL_PHI, dphi
    assert dpsi <= TOL_PSI, dpsi
    assert dcr <= cr_tol, (dcr, cr_tol)
    return dphi, dpsi, dcr


def test_2d_most_rows(G):
    n = (5, 917490)
    h = 1.0 / (n[1] - 1)
    lo, hi = (0.3, 0.0), (0.3 + 4 * h, 1.0)            # square cells
    st = inputs.circle_sdf(n, center=(0.3, 0.5), r=0.2, lo=lo, hi=hi).astype(np.float32)
    g = G.Grid(n, lo=lo, hi=hi)
    g.set_state(st, t0=0.1, recon=True)
    before = g.read_state().astype(np.float64)
    dt = 0.8 * h
    g.step(G.Velocity("vortex2d", T=8.0), dt, 1)
    after = g.read_state().astype(np.float64)
    g.close()
    og = oracle.grid(n, lo=lo, hi=hi)
    ref = oracle.step(og, oracle.velocity("vortex2d", T=8.0), before, 0.1, dt)
    print("2D 5 x 917490:", _compare(after, ref, og, h))


@pytest.mark.parametrize("axis", [1, 2])
def test_3d_most_levels(G, axis):
    n = [4, 4, 4]
    n[axis] = 262140
    n = tuple(n)
    h = 1.0 / (262140 - 1)
    lo = [0.35 - 1.5 * h] * 3
    hi = [0.35 + 1.5 * h] * 3
    lo[axis], hi[axis] = 0.0, 1.0
    st = inputs.sphere_sdf(n, center=(0.35, 0.35, 0.35), r=0.15, lo=lo, hi=hi).astype(np.float32)
    g = G.Grid(n, lo=lo, hi=hi)
    g.set_state(st, t0=0.2, recon=True)
    before = g.read_state().astype(np.float64)
    dt = 0.4 * h
    g.step(G.Velocity("deform3d", T=3.0), dt, 1)
    after = g.read_state().astype(np.float64)
    g.close()
    og = oracle.grid(n, lo=lo, hi=hi)
    ref = oracle.step(og, oracle.velocity("deform3d", T=3.0), before, 0.2, dt)
    print(f"3D {n}:", _compare(after, ref, og, h))


def test_2d_largest_plane(G):
    import torch
    N = 46340
    n = (N, N)
    assert N * N <= 2 ** 31 - 1
    h = 1.0 / (N - 1)
    cx, cy, r = 0.5, 0.75, 0.15
    # the circle's signed distance and gradient, built plane by plane on the device
    st = torch.empty((3, N, N), dtype=torch.float32, device="cuda")
    X = (torch.arange(N, device="cuda", dtype=torch.float64) * h).float()
    dx, dy = (X - cx)[None, :], (X - cy)[:, None]
    torch.add(dx * dx, dy * dy, out=st[0])
    st[0].sqrt_()
    torch.div(dx, st[0], out=st[1])
    torch.div(dy, st[0], out=st[2])
    st[0].sub_(r)
    g = G.Grid(n)
    g.set_state(st, t0=0.0, recon=True)
    del st
    torch.cuda.empty_cache()
    rng = np.random.default_rng(46340)
    picks = [rng.integers(0, N, 2) for _ in range(6)]
    picks += [(128 * 361, 14 * 3309), (128 * 100, 14 * 2000)]                # tile edges
    picks += [(0, 0), (N - 1, 0), (0, N - 1), (N - 1, N - 1), (N - 1, N // 2)]
    for ang in (0.3, 2.5, 4.4):                                             # interface
        picks.append((int((cx + r * math.cos(ang)) / h), int((cy + r * math.sin(ang)) / h)))
    size, margin = 24, 4
    wins = []
    for c in picks:
        w0 = [min(max(int(c[a]) - size // 2, 0), N - size) for a in range(2)]
        wins.append(w0)
    buf = torch.empty((4, N, N), dtype=torch.float32, device="cuda")
    g.read_state(buf)
    torch.cuda.synchronize()
    before = [buf[:, w[1]:w[1] + size, w[0]:w[0] + size].double().cpu().numpy() for w in wins]
    t = g.time
    dt = h
    g.step(G.Velocity("vortex2d", T=8.0), dt, 1)
    g.read_state(buf)
    torch.cuda.synchronize()
    after = [buf[:, w[1]:w[1] + size, w[0]:w[0] + size].double().cpu().numpy() for w in wins]
    # diagnostics and point evaluation on the whole grid (64-bit cell and node indices)
    d = g.diagnostics(q=1)
    pts = np.concatenate([(np.asarray(w) + margin + rng.uniform(0, size - 2 * margin - 1, (3, 2))) * h
                          for w in wins])
    Hp, _, _ = g.eval_points(pts)
    g.close()
    assert d["nonfinite"] == 0
    assert abs(d["measure_negative"] - math.pi * r * r) < 1e-5, d["measure_negative"]
    del buf
    torch.cuda.empty_cache()
    worst, worst_h = [0.0, 0.0, 0.0], []
    for w, b, a in zip(wins, before, after):
        og = oracle.grid((size, size), lo=[w[0] * h, w[1] * h], hi=[(w[0] + size - 1) * h, (w[1] + size - 1) * h])
        ref = oracle.step(og, oracle.velocity("vortex2d", T=8.0), b, t, dt)
        ix = slice(0 if w[0] == 0 else margin, size if w[0] + size == N else size - margin)
        iy = slice(0 if w[1] == 0 else margin, size if w[1] + size == N else size - margin)
        a_in, r_in = a[:, iy, ix], ref[:, iy, ix]
        dphi = np.max(np.abs(a_in[0] - r_in[0]))
        dpsi = np.max(np.abs(a_in[1:3] - r_in[1:3]))
        rec = oracle.recon_cross(og, a)[:, iy, ix]
        dcr = np.max(np.abs(a_in[3] - rec[3]))
        cr_tol = 2e-6 * (np.max(np.abs(rec[3])) + 1.0) + 1e-6 * np.max(np.abs(a_in[1:3])) / h
        assert dphi <= TOL_PHI, (w, dphi)
        assert dpsi <= TOL_PSI, (w, dpsi)
        assert dcr <= cr_tol, (w, dcr, cr_tol)
        worst = [max(worst[0], dphi), max(worst[1], dpsi), max(worst[2], dcr)]
        k = len(worst_h)
        Ho, _ = oracle.eval_points(og, a, pts[3 * k:3 * k + 3])
        worst_h.append(np.max(np.abs(Hp[3 * k:3 * k + 3] - Ho)))
        assert worst_h[-1] <= 8 * 2.0 ** -24 * (1.0 + np.max(np.abs(Ho))), (w, worst_h[-1])
    print("2D 46340^2 windows worst |dphi| |dpsi| |dcross|:", worst, "points |dH|:", max(worst_h),
          "area", d["measure_negative"])
