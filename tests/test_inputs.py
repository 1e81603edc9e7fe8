"""The seeded input generators: exact signed distances checked by brute force."""
import math

import numpy as np

from paper_0905_3409_gb300 import inputs


def _brute(points, curve):
    d = np.sqrt(((points[:, None, :] - curve[None, :, :]) ** 2).sum(-1))
    return d.min(1)


def test_ellipse_sdf_brute_force():
    n = (25, 23)
    c, a, b, ang = (0.47, 0.52), 0.18, 0.07, 0.6
    st = inputs.ellipse_sdf(n, c, a, b, ang)
    t = np.linspace(0, 2 * math.pi, 20001)
    ca, sa = math.cos(ang), math.sin(ang)
    ex, ey = a * np.cos(t), b * np.sin(t)
    curve = np.stack([c[0] + ca * ex - sa * ey, c[1] + sa * ex + ca * ey], 1)
    X, Y = np.meshgrid(*inputs.node_coords(n), indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    d = _brute(pts, curve)
    assert np.max(np.abs(np.abs(st[0].ravel()) - d)) < 2e-5
    g = np.hypot(st[1], st[2])
    assert np.allclose(g, 1.0, atol=1e-12)


def test_slotted_disk_brute_force():
    n = (41, 41)
    st = inputs.slotted_disk_sdf(n)
    cx, cy, r, hw, top = 0.5, 0.75, 0.15, 0.025, 0.85
    yb = cy - math.sqrt(r * r - hw * hw)
    th = np.linspace(0, 2 * math.pi, 60001)
    arc = np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], 1)
    keep = ~((np.abs(arc[:, 0] - cx) < hw) & (arc[:, 1] < top))
    s = np.linspace(0, 1, 5001)[:, None]
    wl = np.concatenate([np.full_like(s, cx - hw), yb + s * (top - yb)], 1)
    wr = np.concatenate([np.full_like(s, cx + hw), yb + s * (top - yb)], 1)
    tp = np.concatenate([cx - hw + s * 2 * hw, np.full_like(s, top)], 1)
    curve = np.concatenate([arc[keep], wl, wr, tp])
    X, Y = np.meshgrid(*inputs.node_coords(n), indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    d = _brute(pts, curve)
    assert np.max(np.abs(np.abs(st[0].ravel()) - d)) < 5e-5  # brute-force sampling spacing
    # inside the slot and outside the disk are positive, the disk body negative
    assert st[0][28, 20] > 0      # (x=0.5, y=0.7) is in the slot
    assert st[0][30, 16] < 0      # (x=0.4, y=0.75) in the body


def test_cube_and_sphere_gradients_unit():
    st = inputs.cube_sdf((17, 17, 17))
    assert np.allclose(st[1] ** 2 + st[2] ** 2 + st[3] ** 2, 1.0)
    st = inputs.sphere_sdf((16, 16, 16))
    assert np.allclose(st[1] ** 2 + st[2] ** 2 + st[3] ** 2, 1.0)


def test_batch_problems_deterministic():
    a = inputs.batch_problems(8, seed=5)
    b = inputs.batch_problems(8, seed=5)
    assert [p.n for p in a] == [p.n for p in b]
    assert all(128 <= p.n <= 1024 for p in a)
    assert all(np.array_equal(p.modes, q.modes) for p, q in zip(a, b))
