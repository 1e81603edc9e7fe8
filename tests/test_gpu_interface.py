"""Final interface location after whole runs, GPU (FP32) against the FP64 oracle run from the
same initial data: the interface the method leaves must lie within 1e-4 of the oracle's
(2D below; 3D in the last test).

Runs: configuration 1 (64^2 nodes, circle r = 0.15 at (0.5, 0.75) with exact gradient and
phi_xy = 0 as given, single vortex T = 8, dt = h, 504 steps: the flow stretches the circle
and brings it back, Sec. 6.2.2) and the same run on 256^2 nodes (2040 steps).  Interface
error: area of the symmetric difference of {phi < 0} between the final and the initial
state over the circle's perimeter, with q^2 samples of each cell's interpolant (reading of
how the paper measures it).  Checked: the GPU's and the oracle's interface errors agree to
1e-4, and the symmetric difference between the two final interfaces, over the perimeter (the
mean distance between them), is below 1e-4."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu
R0, T, Q = 0.15, 8.0, 8


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


@pytest.mark.parametrize("N", [64, 256])
def test_final_interface_matches_oracle(G, N):
    n = (N, N)
    h = 1.0 / (N - 1)
    steps = int(round(T / h))
    st = inputs.circle_sdf(n).astype(np.float32)
    g = G.Grid(n)
    g.set_state(st, t0=0.0)
    g.step(G.Velocity("vortex2d", T=T), h, steps)
    gpu = g.read_state().astype(np.float64)
    g.close()
    og = oracle.grid(n)
    init = st.astype(np.float64)
    orc = oracle.run(og, oracle.velocity("vortex2d", T=T), init, 0.0, h, steps)
    perim = 2 * math.pi * R0
    e_gpu = oracle.symdiff(og, gpu, init, Q)[0] / perim
    e_orc = oracle.symdiff(og, orc, init, Q)[0] / perim
    apart = oracle.symdiff(og, gpu, orc, Q)[0] / perim
    print(f"{N}^2, {steps} steps: interface error GPU {e_gpu:.6e}, oracle {e_orc:.6e}, "
          f"GPU vs oracle {apart:.3e}, max |dphi| {np.max(np.abs(gpu[0] - orc[0])):.3e}")
    assert abs(e_gpu - e_orc) <= 1e-4
    assert apart <= 1e-4


@pytest.mark.parametrize("N", [40, 64])
def test_final_interface_matches_oracle_3d(G, N):
    """LeVeque's deformation field (T = 3, modulated by cos(pi t / T)), sphere r = 0.15 at
    (0.35, 0.35, 0.35), dt = h (CFL 2: feet up to two cells away) through the whole period:
    the GPU's and the oracle's final interfaces, measured against the initial sphere and
    against each other per unit of the sphere's area."""
    n = (N, N, N)
    h = 1.0 / (N - 1)
    steps = int(math.ceil(3.0 / h - 1e-9))
    dt = 3.0 / steps
    st = inputs.sphere_sdf(n, center=(0.35, 0.35, 0.35), r=R0).astype(np.float32)
    g = G.Grid(n)
    g.set_state(st, t0=0.0, recon=True)
    init = g.read_state().astype(np.float64)  # mixed derivatives as the GPU rebuilt them
    g.step(G.Velocity("deform3d", T=3.0), dt, steps)
    gpu = g.read_state().astype(np.float64)
    g.close()
    og = oracle.grid(n)
    orc = oracle.run(og, oracle.velocity("deform3d", T=3.0), init, 0.0, dt, steps)
    area = 4 * math.pi * R0 ** 2
    qq = 4
    e_gpu = oracle.symdiff(og, gpu, init, qq)[0] / area
    e_orc = oracle.symdiff(og, orc, init, qq)[0] / area
    apart = oracle.symdiff(og, gpu, orc, qq)[0] / area
    print(f"{N}^3, {steps} steps: interface error GPU {e_gpu:.6e}, oracle {e_orc:.6e}, "
          f"GPU vs oracle {apart:.3e}, max |dphi| {np.max(np.abs(gpu[0] - orc[0])):.3e}")
    assert abs(e_gpu - e_orc) <= 1e-4
    assert apart <= 1e-4


def test_vortex_refinement_to_benchmark_size(G):
    """Configuration 1's run (circle r = 0.15 at (0.5, 0.75), single vortex T = 8, dt = h)
    on 64^2 to 4096^2 nodes (the benchmark's grid: 32760 steps): the interface error
    against the initial circle falls at every refinement."""
    errs, areas = [], []
    for N in (64, 128, 256, 512, 1024, 2048, 4096):
        n = (N, N)
        h = 1.0 / (N - 1)
        st = inputs.circle_sdf(n).astype(np.float32)
        g, ref = G.Grid(n), G.Grid(n)
        g.set_state(st, t0=0.0)
        ref.set_state(st, t0=0.0)
        g.step(G.Velocity("vortex2d", T=T), h, int(round(T / h)))
        d = g.diagnostics(q=4, reference=ref)
        g.close()
        ref.close()
        assert d["nonfinite"] == 0
        errs.append(d["measure_symdiff"] / (2 * math.pi * R0))
        areas.append(d["measure_negative"] / (math.pi * R0 * R0) - 1.0)
    print("single vortex, N = 64 ... 4096: interface error",
          ", ".join(f"{e:.3e}" for e in errs), "; area change", ", ".join(f"{a:+.2e}" for a in areas))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs


def test_zalesak_disk_revolution_at_benchmark_size(G):
    """Zalesak's slotted disk (Sec. 6.2.3) through one revolution of the rigid rotation
    omega = 2 pi about (0.5, 0.5) on 4096^2 nodes, dt = h / pi (12865 steps): the disk comes
    back with an interface error (symmetric difference over 2 pi r) below 1e-3 and its area
    within 1e-3."""
    N = 4096
    n = (N, N)
    h = 1.0 / (N - 1)
    steps = int(math.ceil(math.pi / h - 1e-9))
    st = inputs.slotted_disk_sdf(n).astype(np.float32)
    g, ref = G.Grid(n), G.Grid(n)
    g.set_state(st, t0=0.0, recon=True)
    ref.set_state(st, t0=0.0, recon=True)
    g.step(G.Velocity("rotation", omega=2 * math.pi, center=(0.5, 0.5, 0.0)), 1.0 / steps, steps)
    d = g.diagnostics(q=4, reference=ref)
    a0 = ref.diagnostics(q=4)["measure_negative"]
    g.close()
    ref.close()
    e = d["measure_symdiff"] / (2 * math.pi * R0)
    da = d["measure_negative"] / a0 - 1.0
    print(f"Zalesak disk, 4096^2, one revolution ({steps} steps): interface error {e:.3e}, "
          f"area change {da:+.3e}")
    assert d["nonfinite"] == 0 and e < 1e-3 and abs(da) < 1e-3
