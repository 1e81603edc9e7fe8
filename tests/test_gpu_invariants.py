"""GPU invariants of the step: bit-exact integer-cell shift, exact linear transport,
COMPACT == FULL bitwise, CUDA-graph replay == one launch per call, checkpoint/resume,
argument errors, and the diagnostics against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


@pytest.mark.parametrize("dim", [2, 3])
def test_integer_cell_shift_bit_exact(G, dim):
    """A translation by one cell per step (h = 2^-k) moves every plane by one node
    exactly (Sec. 5.4, xi = 1 of the previous cell = xi = 0 of the next): bit for bit for
    nodes whose foot is an interior node, and to rounding where the foot is clamped onto
    the last node of an axis (the inflow edge, where the paper's shift argument does not
    apply and the foot's cell is the last one, at its far end).  The rebuilt mixed
    derivatives shift with their stencils' nodes."""
    n = (65, 33) if dim == 2 else (17, 17, 9)
    g = G.Grid(n, hi=[(nn - 1) / 64.0 for nn in n])  # h = 1/64 on every axis
    st = inputs.random_state((4 if dim == 2 else 8,) + n[::-1], seed=2).astype(np.float32)
    g.set_state(st, recon=True)
    st = g.read_state()
    vel = G.Velocity("const", c=(-1.0,) * dim + (0.0,) * (3 - dim))
    g.step(vel, 1.0 / 64, 1)
    out = g.read_state()
    core = 1 + dim
    inner = (slice(None),) + (slice(None, -2),) * dim      # foot on an interior node
    shifted = (slice(None),) + (slice(1, -1),) * dim
    edge = (slice(None),) + (slice(None, -1),) * dim       # including feet on the last node
    edge_src = (slice(None),) + (slice(1, None),) * dim
    assert np.array_equal(out[:core][inner], st[:core][shifted])
    np.testing.assert_allclose(out[:core][edge], st[:core][edge_src], rtol=1e-6, atol=1e-6)
    cin = (slice(None),) + (slice(1, -3),) * dim
    csrc = (slice(None),) + (slice(2, -2),) * dim
    assert np.array_equal(out[core:][cin], st[core:][csrc])
    cedge = (slice(None),) + (slice(1, -2),) * dim
    cedge_src = (slice(None),) + (slice(2, -1),) * dim
    np.testing.assert_allclose(out[core:][cedge], st[core:][cedge_src], rtol=1e-5, atol=1e-4)


def test_linear_transport(G):
    n = (40, 31)
    a = (0.3, -0.7)
    g = G.Grid(n)
    g.set_state(inputs.linear2d(n, a=a).astype(np.float32))
    c, dt = (0.21, 0.13), 0.02
    g.step(G.Velocity("const", c=c + (0.0,)), dt, 3)
    out = g.read_state()
    X, Y = np.meshgrid(*inputs.node_coords(n), indexing="xy")
    # outside the numerical domain of dependence of the inflow edges x = 0, y = 0:
    # each step reaches back by the displacement plus two cells (the foot cell and the
    # neighbour column its phi_xy stencil reads)
    h = 1.0 / 39
    inside = (X - 3 * (c[0] * dt + 2 * h) >= 0) & (Y - 3 * (c[1] * dt + 2 * h) >= 0)
    exact = a[0] * (X - 3 * c[0] * dt) + a[1] * (Y - 3 * c[1] * dt) + 0.1
    assert np.max(np.abs(out[0] - exact)[inside]) < 2e-6
    # FP32 rounding of psi_y differences enters through phi_xy (x 1/(2h)) and back
    # through h phi_xy terms: a few 1e-6 at most
    assert np.max(np.abs(out[1] - a[0])[inside]) < 1e-5
    assert np.max(np.abs(out[2] - a[1])[inside]) < 1e-5
    inner = inside.copy()
    inner[:, np.argmax(inside[0]) if inside[0].any() else 0] = False  # one more column for phi_xy
    assert np.max(np.abs(out[3])[inner]) < 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_equals_full_bitwise(G, dim):
    n = (45, 38) if dim == 2 else (20, 19, 18)
    if dim == 2:
        st = inputs.circle_sdf(n, center=(0.5, 0.6), r=0.25)
        vel = G.Velocity("vortex2d", T=8.0)
    else:
        st = inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.3)
        vel = G.Velocity("deform3d", T=3.0)
    outs = []
    for layout in ("full", "compact"):
        g = G.Grid(n, layout=layout)
        g.set_state(st.astype(np.float32), recon=True)
        g.step(vel, 0.6 / (max(n) - 1), 5)
        outs.append(g.read_state())
        g.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n0", [129, 130, 131, 256, 300])
@pytest.mark.parametrize("cfl", [0.9, 2.5])
def test_full_equals_compact_across_tiles(G, n0, cfl):
    """Grids several 128-column tiles wide, five steps in one call (one CUDA graph).  The
    FULL step writes phi_xy+ of a tile's edge columns from the new psi_y of the halo
    columns it updates itself; COMPACT rebuilds every mixed derivative from psi_y when it
    reads it.  The two layouts must agree bit for bit, also with feet outside the staged
    tile (CFL 2.5, read from global memory) and with a last tile one to three columns wide."""
    n = (n0, 23)
    st = inputs.circle_sdf(n, center=(0.5, 0.5), r=0.3).astype(np.float32)
    vel = G.Velocity("vortex2d", T=8.0)
    outs = []
    for layout in ("full", "compact"):
        g = G.Grid(n, layout=layout)
        g.set_state(st, t0=0.3, recon=True)
        g.step(vel, cfl / (n0 - 1), 5)
        outs.append(g.read_state())
        g.close()
    assert np.array_equal(outs[0], outs[1])


def test_graph_replay_equals_single_steps(G):
    """A steady field, so the result cannot depend on how the clock sums dt."""
    n = (50, 50)
    st = inputs.circle_sdf(n).astype(np.float32)
    vel = G.Velocity("rotation", omega=2 * math.pi, center=(0.5, 0.5, 0.0))
    a = G.Grid(n)
    a.set_state(st)
    a.step(vel, 0.02, 7)          # one CUDA graph
    a.step(vel, 0.02, 7)          # replay of the cached graph
    b = G.Grid(n)
    b.set_state(st)
    for _ in range(14):
        b.step(vel, 0.02, 1)
    assert a.time == pytest.approx(b.time, abs=1e-15)
    assert np.array_equal(a.read_state(), b.read_state())


def test_checkpoint_resume_bitwise(G):
    n = (33, 40)
    st = inputs.circle_sdf(n, r=0.2).astype(np.float32)
    vel = G.Velocity("vortex2d", T=8.0)
    a = G.Grid(n)
    a.set_state(st)
    a.step(vel, 0.03, 10)
    full = a.read_state()
    b = G.Grid(n)
    b.set_state(st)
    b.step(vel, 0.03, 4)
    ck, t = b.read_state(), b.time
    c = G.Grid(n)
    c.set_state(ck, t0=t)
    c.step(vel, 0.03, 6)
    assert np.array_equal(c.read_state(), full)


def test_device_memspace_roundtrip(G):
    import torch
    n = (20, 24)
    st = torch.tensor(inputs.circle_sdf(n).astype(np.float32), device="cuda")
    g = G.Grid(n)
    g.set_state(st)
    out = torch.empty_like(st)
    g.read_state(out)
    assert torch.equal(out, st)


def test_argument_errors(G):
    n = (16, 16)
    g = G.Grid(n)
    with pytest.raises(G.GalsError) as e:
        g.step(G.Velocity("vortex2d", T=8.0), 0.01, 1)
    assert e.value.status == G.ERR_STATE
    g.set_state(inputs.circle_sdf(n).astype(np.float32))
    for dt in (0.0, -1.0, float("nan")):
        with pytest.raises(G.GalsError) as e:
            g.step(G.Velocity("vortex2d", T=8.0), dt, 1)
        assert e.value.status == G.ERR_ARG
    with pytest.raises(G.GalsError) as e:
        g.step(G.Velocity("deform3d", T=3.0), 0.01, 1)
    assert e.value.status == G.ERR_UNSUPPORTED
    with pytest.raises(G.GalsError) as e:
        g.step(G.Velocity("fourier2d", modes=np.array([[0.1, 5, 1, 0, 0]])), 0.01, 1)
    assert e.value.status == G.ERR_ARG
    before = g.read_state()
    g.step(G.Velocity("vortex2d", T=8.0), 0.01, 0)
    assert np.array_equal(before, g.read_state())


def test_diagnostics_against_oracle(G):
    n = (96, 96)
    st = inputs.circle_sdf(n, r=0.2, center=(0.5, 0.5)).astype(np.float32)
    ref = inputs.circle_sdf(n, r=0.22, center=(0.52, 0.5)).astype(np.float32)
    a = G.Grid(n)
    a.set_state(st, recon=True)
    b = G.Grid(n)
    b.set_state(ref, recon=True)
    q = 6
    d = a.diagnostics(q=q, reference=b)
    og = oracle.grid(n)
    sa = a.read_state().astype(np.float64)
    sb = b.read_state().astype(np.float64)
    area = oracle.measure_negative(og, sa, q)
    sym, amb = oracle.symdiff(og, sa, sb, q, eps=1e-5)
    sample = (1.0 / 95) ** 2 / q ** 2
    assert abs(d["measure_negative"] - area) <= (amb + 0.5) * sample
    assert abs(d["measure_symdiff"] - sym) <= (amb + 0.5) * sample
    assert d["emax_phi"] == pytest.approx(float(np.max(np.abs(sa[0] - sb[0]))), abs=1e-7)
    assert d["emax_psi"] == pytest.approx(float(np.max(np.abs(sa[1:3] - sb[1:3]))), abs=1e-7)
    l2 = math.sqrt(np.sum((sa[0] - sb[0]) ** 2) * (1.0 / 95) ** 2)
    assert d["l2_phi"] == pytest.approx(l2, rel=1e-12)
    assert d["nonfinite"] == 0
    bad = st.copy()
    bad[2, 5, 7] = np.nan
    a.set_state(bad)
    assert a.diagnostics(q=0)["nonfinite"] == 1
