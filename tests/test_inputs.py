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


def test_slotted_sphere_sign_gradient_and_slices():
    """Zalesak's slotted sphere: the sign at known nodes, a unit gradient that matches
    one-sided differences of phi wherever those agree (away from the kinks of the max),
    phi exact (|x - c| - r) on the sphere away from the slot, and z_range slices."""
    n = (33, 33, 33)                                  # h = 1/32: 0.5 and 0.75 are nodes
    st = inputs.slotted_sphere_sdf(n)
    phi = st[0]
    assert phi[16, 24, 16] > 0                        # the centre lies in the slot
    assert phi[16, 22, 16] > 0                        # (0.5, 0.6875, 0.5): slot, lower
    assert phi[16, 28, 16] < 0                        # (0.5, 0.875, 0.5): above the slot end
    assert phi[16, 24, 13] < 0                        # (0.40625, 0.75, 0.5): the body
    assert phi[16, 24, 24] > 0                        # (0.75, 0.75, 0.5): outside
    assert np.allclose(st[1] ** 2 + st[2] ** 2 + st[3] ** 2, 1.0)
    assert not np.any(st[4:])
    eps = 1e-6
    for ax in range(3):
        lo, hi = [0.0] * 3, [1.0] * 3
        lo[ax] += eps
        hi[ax] += eps
        fp = inputs.slotted_sphere_sdf(n, lo=lo, hi=hi)[0]
        lo[ax] -= 2 * eps
        hi[ax] -= 2 * eps
        fm = inputs.slotted_sphere_sdf(n, lo=lo, hi=hi)[0]
        fwd, bwd = (fp - phi) / eps, (phi - fm) / eps
        smooth = np.abs(fwd - bwd) < 1e-4
        assert smooth.mean() > 0.95
        assert np.max(np.abs(st[1 + ax][smooth] - 0.5 * (fwd + bwd)[smooth])) < 1e-4
    X, Y, Z = np.meshgrid(*inputs.node_coords(n), indexing="xy")
    X, Y, Z = (a.transpose(2, 0, 1) for a in (X, Y, Z))   # to [z][y][x]
    d = np.sqrt((X - 0.5) ** 2 + (Y - 0.75) ** 2 + (Z - 0.5) ** 2)
    far = (np.abs(X - 0.5) > 0.1) | (Y > 0.95)
    assert np.allclose(phi[far], d[far] - 0.15, atol=1e-15)
    part = inputs.slotted_sphere_sdf(n, z_range=(5, 12))
    assert np.array_equal(part, st[:, 5:12])
