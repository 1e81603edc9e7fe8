"""Row bands of the 2D multi-step graph: a call of several steps is captured as bands of
tile rows, each band of step s depending on bands b - 1, b, b + 1 of step s - 1 only.  The
results must equal one eager launch per step bit for bit (the per-node arithmetic does
not depend on how the grid is cut into launches), also where the feet reach several rows
and where the band heights are uneven, and the library's launch count must follow the
band rule: up to 4 bands of whole 14-row tiles, each at least 2 tiles and the velocity's
reach plus 4 rows high."""
import math

import numpy as np
import pytest

from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu

TILE_ROWS = 14


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def expected_bands(n1, reach_rows):
    tiles = -(-n1 // TILE_ROWS)
    min_rows = math.ceil(reach_rows) + 4
    min_tiles = max(2, -(-min_rows // TILE_ROWS))
    nb = min(4, tiles // min_tiles)
    return nb if nb >= 2 else 1


def _vel(G, kind):
    if kind == "vortex2d":
        return G.Velocity("vortex2d", T=8.0)
    if kind == "waves2d":
        return G.Velocity("waves2d", modes=inputs.wave_modes(32, seed=41))
    if kind == "rotation":
        return G.Velocity("rotation", omega=2 * math.pi)
    if kind == "fourier2d":
        return G.Velocity("fourier2d", modes=inputs.fourier_modes(16, seed=31))
    return G.Velocity("vortex2d", T=8.0, trace="heun_psi")


CASES = [
    # (n0, n1), field, CFL, layout, cross
    ((300, 200), "vortex2d", 0.8, "full", "central"),
    ((257, 131), "fourier2d", 0.9, "full", "central"),
    ((129, 97), "rotation", 6.0, "full", "central"),     # feet up to 6 rows away
    ((190, 450), "vortex2d", 0.8, "compact", "central"),
    ((140, 170), "heun", 0.8, "full", "central"),
    ((201, 150), "vortex2d", 0.8, "full", "cell"),
    ((260, 140), "waves2d", 0.8, "full", "central"),
]


@pytest.mark.parametrize("n,kind,cfl,layout,cross", CASES)
def test_banded_graph_equals_single_steps(G, n, kind, cfl, layout, cross):
    st = inputs.circle_sdf(n).astype(np.float32)
    dt = cfl / (max(n) - 1)
    vel = _vel(G, kind)
    a = G.Grid(n, layout=layout, cross=cross)
    b = G.Grid(n, layout=layout, cross=cross)
    for g in (a, b):
        g.set_state(st, recon=True)
    nsteps = 6
    a.step(vel, dt, nsteps)  # one captured graph of row bands
    for _ in range(nsteps):
        b.step(vel, dt, 1)   # one eager launch per step, whole grid
    # (plane waves: amplitudes,) coefficients, step, clock
    assert b.last_step_launches() == (4 if kind == "waves2d" else 3)
    ra, rb = a.read_state(), b.read_state()
    assert np.array_equal(ra, rb, equal_nan=True)
    assert np.isfinite(ra).all()


def test_band_launch_counts(G):
    """The launch count of a banded call: 4 bands on a tall grid, fewer where the grid has
    few tile rows or the feet reach far, none on a grid of 3 tile rows."""
    vel = G.Velocity("rotation", omega=2 * math.pi)
    for n, cfl in [((256, 512), 0.5), ((256, 60), 0.5), ((128, 256), 20.0), ((64, 40), 0.5)]:
        g = G.Grid(n)
        g.set_state(inputs.circle_sdf(n).astype(np.float32), recon=True)
        dt = cfl / (max(n) - 1)
        g.step(vel, dt, 5)
        # the library's speed bound of the rotation on [0,1]^2 about (0.5, 0.5): |omega| times
        # the largest distance from the centre along one axis
        reach = dt * 2 * math.pi * 0.5 * (n[1] - 1)
        nb = expected_bands(n[1], reach)
        assert g.last_step_launches() == 5 * nb + 2, (n, cfl, nb, g.last_step_launches())
        g.step(vel, dt, 0)
        assert g.last_step_launches() == 0


def test_long_call_replays_bounded_graphs(G):
    """A call of more steps than one graph holds (256) replays graphs of 256 steps and one of
    the rest: the same result as one launch per step, bit for bit, for an odd total (the
    last graph flips the ping-pong buffers), and the launch count of every replay."""
    n, nsteps = (128, 100), 601
    vel = G.Velocity("rotation", omega=2 * math.pi)
    dt = 0.5 / (max(n) - 1)
    st = inputs.circle_sdf(n).astype(np.float32)
    a, b = G.Grid(n), G.Grid(n)
    for g in (a, b):
        g.set_state(st, recon=True)
    a.step(vel, dt, nsteps)
    for _ in range(nsteps):
        b.step(vel, dt, 1)
    nb = expected_bands(n[1], dt * 2 * math.pi * 0.5 * (n[1] - 1))
    assert a.last_step_launches() == 2 * (256 * nb + 2) + (89 * nb + 2)
    assert np.array_equal(a.read_state(), b.read_state())
    assert a.time == pytest.approx(b.time, rel=0, abs=1e-12)


def test_bench_configuration_bands_equal_single_steps(G):
    """The benchmark's launch configuration: the 4096^2 single vortex at CFL 1, stepped as
    the bench times it (a multi-step call: four bands of 73 and 74 tile rows per step),
    equals one whole-grid launch per step bit for bit."""
    n = (4096, 4096)
    st = inputs.circle_sdf(n).astype(np.float32)
    vel = G.Velocity("vortex2d", T=8.0)
    dt = 1.0 / (n[0] - 1)
    a, b = G.Grid(n), G.Grid(n)
    for g in (a, b):
        g.set_state(st, recon=True)
    a.step(vel, dt, 4)
    assert a.last_step_launches() == 4 * 4 + 2
    for _ in range(4):
        b.step(vel, dt, 1)
    ra, rb = a.read_state(), b.read_state()
    assert np.array_equal(ra, rb)
    a.close()
    b.close()


def test_banded_graph_explicit_cross_compact(G):
    """COMPACT layout with the mixed derivatives given explicitly (zero, as configuration 1
    sets them): only the first step of the call reads the given planes, later ones rebuild
    them; a banded multi-step call equals single steps bit for bit."""
    n = (230, 170)
    st = inputs.circle_sdf(n).astype(np.float32)
    st[3] = 0.0
    vel = G.Velocity("vortex2d", T=8.0)
    dt = 0.8 / (max(n) - 1)
    a, b = G.Grid(n, layout="compact"), G.Grid(n, layout="compact")
    for g in (a, b):
        g.set_state(st, recon=False)
    a.step(vel, dt, 5)
    for _ in range(5):
        b.step(vel, dt, 1)
    assert np.array_equal(a.read_state(), b.read_state())
