"""GPU normals and curvature of the interpolant at points (gals_eval_points, Sec. 3.4)
against the FP64 oracle evaluated on the GPU's own state.

The GPU evaluates in FP32 from FP32 data; the oracle in FP64 from the same data widened.
The difference is rounding: a second derivative sums terms of size up to ~6 |psi| / h
(slopes times g'' / h, value differences times f'' / h^2), each rounded at 2^-24 relative,
and kappa divides it by |grad H|; the bound below takes 16 such roundings."""
import numpy as np
import pytest

import oracle
from paper_0905_3409_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def _points(rng, n, dim, h):
    """Random points inside, a few outside the box, on nodes and on cell edges."""
    p = rng.uniform(0.0, 1.0, (n, dim))
    p[:8] = rng.uniform(-0.2, 1.2, (8, dim))                       # clamped into the box
    idx = rng.integers(0, int(round(1.0 / min(h))), (8, dim))
    p[8:16] = idx * np.asarray(h)                                  # nodes
    p[16:24, 0] = idx[:, 0] * h[0]                                 # cell edges in x
    return p


def _check(G, g, og, dim, pts, hmin):
    H, N, K = g.eval_points(pts)
    st = g.read_state().astype(np.float64)
    Ho, No, Ko = oracle.curvature_points(og, st, pts)
    maxpsi = np.max(np.abs(st[1:1 + dim]))
    gn = np.linalg.norm(No, axis=1)                                # |n| = 1 where grad H != 0
    _, Go = oracle.eval_points(og, st, pts)
    gmag = np.linalg.norm(Go, axis=1)
    ok = gmag > 0.3 * maxpsi                                       # away from kinks / extrema
    assert np.max(np.abs(H - Ho)) <= 8 * EPS32 * (1.0 + np.max(np.abs(Ho)))
    tol_n = 16 * EPS32 * 6 * maxpsi / gmag[ok] + 1e-6
    assert np.all(np.abs(N[ok] - No[ok]).max(axis=1) <= tol_n)
    tol_k = 16 * EPS32 * 6 * maxpsi / hmin / gmag[ok] + 1e-5 * np.abs(Ko[ok])
    dk = np.abs(K[ok] - Ko[ok])
    assert np.all(dk <= tol_k), (dk.max(), tol_k[np.argmax(dk)])
    assert np.allclose(gn[ok], 1.0)
    return dk.max(), np.abs(N[ok] - No[ok]).max()


def test_eval_points_2d_against_oracle(G):
    n = (161, 129)
    st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.25).astype(np.float32)
    g = G.Grid(n)
    g.set_state(st, recon=True)
    g.step(G.Velocity("vortex2d", T=8.0), 0.6 / 160, 3)           # a state the method made
    og = oracle.grid(n)
    pts = _points(np.random.default_rng(1), 4000, 2, og.h[:2])
    _check(G, g, og, 2, pts, min(og.h[:2]))


def test_eval_points_3d_against_oracle(G):
    n = (24, 20, 28)
    st = inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.3).astype(np.float32)
    g = G.Grid(n)
    g.set_state(st, recon=True)
    g.step(G.Velocity("deform3d", T=3.0), 0.4 / 27, 2)
    og = oracle.grid(n)
    pts = _points(np.random.default_rng(2), 3000, 3, og.h[:3])
    _check(G, g, og, 3, pts, min(og.h[:3]))


@pytest.mark.parametrize("dim", [2, 3])
def test_eval_points_approach_B(G, dim):
    n = (64, 56) if dim == 2 else (20, 18, 22)
    st = inputs.circle_sdf(n, center=(0.5, 0.5), r=0.3) if dim == 2 else \
        inputs.sphere_sdf(n, center=(0.5, 0.5, 0.5), r=0.3)
    g = G.Grid(n, cross="cell")
    g.set_state(st.astype(np.float32))
    og = oracle.grid(n, cross="cell")
    pts = _points(np.random.default_rng(3), 2000, dim, og.h[:dim])
    _check(G, g, og, dim, pts, min(og.h[:dim]))


def test_eval_points_layouts_and_memspaces_agree(G):
    import torch
    n = (90, 70)
    st = inputs.circle_sdf(n, center=(0.5, 0.5), r=0.3).astype(np.float32)
    pts = np.random.default_rng(4).uniform(0, 1, (1000, 2))
    out = []
    for layout in ("full", "compact"):
        g = G.Grid(n, layout=layout)
        g.set_state(st, recon=True)
        g.step(G.Velocity("vortex2d", T=8.0), 0.5 / 89, 2)
        out.append(g.eval_points(pts))
        Hd, Nd, Kd = g.eval_points(torch.tensor(pts, device="cuda"))
        assert np.array_equal(Hd.cpu().numpy(), out[-1][0])
        assert np.array_equal(Nd.cpu().numpy(), out[-1][1])
        assert np.array_equal(Kd.cpu().numpy(), out[-1][2])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_eval_points_circle_curvature(G):
    """The curvature of the signed distance to a circle is 1/|x - c| and its normal
    (x - c)/|x - c|.  From an FP32 state the second derivatives carry the rounding of the
    stored phi times 6 / h^2 (about 3e-3 at h = 1/128, order 1 at h = 1/4095), so this
    check runs on 129^2 nodes: kappa to 5e-3 relative, n to 1e-4."""
    n = (129, 129)
    c = np.array([0.5, 0.75])
    g = G.Grid(n)
    g.set_state(inputs.circle_sdf(n).astype(np.float32), recon=True)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(5000, 2))
    d /= np.linalg.norm(d, axis=1)[:, None]
    rad = rng.uniform(0.1, 0.2, 5000)
    _, N, K = g.eval_points(c + d * rad[:, None])
    assert np.max(np.abs(K * rad - 1.0)) < 5e-3
    assert np.max(np.abs(N - d)) < 1e-4


def test_eval_points_argument_errors(G):
    n = (16, 16)
    g = G.Grid(n)
    with pytest.raises(G.GalsError) as e:
        g.eval_points(np.zeros((3, 2)))
    assert e.value.status == G.ERR_STATE
    g.set_state(inputs.circle_sdf(n).astype(np.float32))
    H, N, K = g.eval_points(np.zeros((0, 2)))
    assert H.shape == (0,)
