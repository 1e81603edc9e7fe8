"""Seeded synthetic inputs for the GALS step: initial level set states and the
random tables of the velocity fields.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests.  It holds none of the method's arithmetic (no trace, no Hermite
interpolation, no cross-derivative reconstruction): it only produces initial
data -- signed distance functions with their exact gradients, smooth test
functions with exact derivatives -- and the random numbers the velocity fields
draw.  Everything is FP64 numpy, seeded explicitly.

State arrays have shape (nplanes, [nz,] ny, nx) with x fastest:
  2D planes [phi, phi_x, phi_y, phi_xy]; 3D [phi, phi_x, phi_y, phi_z, phi_xy,
  phi_xz, phi_yz, phi_xyz].  Signed distance inputs carry zero cross planes; the
  consumer rebuilds them from the gradients when the configuration asks for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 9053409


def node_coords(n, lo=None, hi=None):
    """1D coordinate arrays x_i = lo + i h, h = (hi-lo)/(n-1), per axis."""
    dim = len(n)
    lo = [0.0] * dim if lo is None else list(lo)
    hi = [1.0] * dim if hi is None else list(hi)
    return [lo[d] + np.arange(n[d], dtype=np.float64) * ((hi[d] - lo[d]) / (n[d] - 1))
            for d in range(dim)]


def _mesh(n, lo=None, hi=None):
    axes = node_coords(n, lo, hi)
    if len(n) == 2:
        Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
        return X, Y
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X, Y, Z


def _unit(vx, vy, vz=None):
    if vz is None:
        r = np.hypot(vx, vy)
        safe = np.where(r > 0, r, 1.0)
        return np.where(r > 0, vx / safe, 0.0), np.where(r > 0, vy / safe, 0.0)
    r = np.sqrt(vx * vx + vy * vy + vz * vz)
    safe = np.where(r > 0, r, 1.0)
    return (np.where(r > 0, vx / safe, 0.0), np.where(r > 0, vy / safe, 0.0),
            np.where(r > 0, vz / safe, 0.0))


def _state2d(phi, px, py, pxy=None):
    pxy = np.zeros_like(phi) if pxy is None else pxy
    return np.stack([phi, px, py, pxy]).astype(np.float64)


def _state3d(phi, px, py, pz, cross=None):
    z = np.zeros_like(phi)
    cr = [z, z, z, z] if cross is None else list(cross)
    return np.stack([phi, px, py, pz] + cr).astype(np.float64)


# ------------------------------------------------------------------ 2D initial data

def circle_sdf(n, center=(0.5, 0.75), r=0.15, lo=None, hi=None):
    """Signed distance to a circle (negative inside), exact gradient, zero phi_xy.
    The gradient is set to 0 at the centre, where it is undefined."""
    X, Y = _mesh(n, lo, hi)
    dx, dy = X - center[0], Y - center[1]
    d = np.hypot(dx, dy)
    ux, uy = _unit(dx, dy)
    return _state2d(d - r, ux, uy)


def gaussian_bump2d(n, x0=(0.5, 0.5), r0=0.15, lo=None, hi=None):
    """phi = exp(-|x-x0|^2) - exp(-r0^2) with exact phi_x, phi_y, phi_xy."""
    X, Y = _mesh(n, lo, hi)
    dx, dy = X - x0[0], Y - x0[1]
    e = np.exp(-(dx * dx + dy * dy))
    return _state2d(e - math.exp(-r0 * r0), -2 * dx * e, -2 * dy * e, 4 * dx * dy * e)


def gaussian_bump2d_exact(X, Y, x0=(0.5, 0.5)):
    dx, dy = X - x0[0], Y - x0[1]
    e = np.exp(-(dx * dx + dy * dy))
    return e, -2 * dx * e, -2 * dy * e


def _seg_closest(px, py, ax, ay, bx, by):
    """closest point on segment [a,b] to p (vectorised over p)."""
    ex, ey = bx - ax, by - ay
    L2 = ex * ex + ey * ey
    t = np.clip(((px - ax) * ex + (py - ay) * ey) / L2, 0.0, 1.0)
    return ax + t * ex, ay + t * ey


def slotted_disk_sdf(n, center=(0.5, 0.75), r=0.15, slot_w=0.05, slot_top=0.85,
                     lo=None, hi=None):
    """Exact signed distance to Zalesak's slotted disk and its gradient.

    The shape is the disk minus the slot {|x - cx| < w/2, y < slot_top}: the slot
    opens through the bottom of the disk and ends at y = slot_top (depth 0.25 for
    the default disk).  The boundary is the remaining arc, the two slot walls and
    the slot's top edge; the distance is the minimum over these four features,
    ties going to the first feature (arc, left wall, right wall, top)."""
    X, Y = _mesh(n, lo, hi)
    cx, cy = center
    hw = slot_w / 2
    yb = cy - math.sqrt(r * r - hw * hw)  # where the walls meet the circle
    # feature 0: the arc (circle minus its bottom part between the walls)
    dx, dy = X - cx, Y - cy
    rr = np.hypot(dx, dy)
    ux, uy = _unit(dx, dy)
    # points of the circle in direction (ux, uy); if that point is cut away by the slot,
    # the nearest arc point is one of the two arc endpoints
    qx, qy = cx + r * ux, cy + r * uy
    qx = np.where(rr > 0, qx, cx + r)
    qy = np.where(rr > 0, qy, cy)
    cut = (np.abs(qx - cx) < hw) & (qy < slot_top)
    e1x, e1y = cx - hw, yb
    e2x, e2y = cx + hw, yb
    d_e1 = np.hypot(X - e1x, Y - e1y)
    d_e2 = np.hypot(X - e2x, Y - e2y)
    use1 = d_e1 <= d_e2
    qx = np.where(cut, np.where(use1, e1x, e2x), qx)
    qy = np.where(cut, np.where(use1, e1y, e2y), qy)
    feats = [(qx, qy)]
    feats.append(_seg_closest(X, Y, cx - hw, yb, cx - hw, slot_top))
    feats.append(_seg_closest(X, Y, cx + hw, yb, cx + hw, slot_top))
    feats.append(_seg_closest(X, Y, cx - hw, slot_top, cx + hw, slot_top))
    dists = np.stack([np.hypot(X - fx, Y - fy) for fx, fy in feats])
    best = np.argmin(dists, axis=0)  # first minimum on ties
    d = np.take_along_axis(dists, best[None], 0)[0]
    bx = np.choose(best, [f[0] for f in feats])
    by = np.choose(best, [f[1] for f in feats])
    inside_disk = rr < r
    in_slot = (np.abs(X - cx) < hw) & (Y < slot_top)
    inside = inside_disk & ~in_slot
    sgn = np.where(inside, -1.0, 1.0)
    gx, gy = _unit(X - bx, Y - by)
    return _state2d(sgn * d, sgn * gx, sgn * gy)


def ellipse_sdf(n, center, a, b, angle, lo=None, hi=None, iters=120):
    """Exact signed distance to an ellipse with semi-axes a, b rotated by `angle`.

    Closest points come from the standard root-finding formulation of the
    point-to-ellipse distance (D. Eberly, "Distance from a point to an ellipse"):
    in the ellipse frame, first quadrant, with a >= b, the closest point is
    (a^2 y0/(t+a^2), b^2 y1/(t+b^2)) where t is the root of
    F(t) = (a y0/(t+a^2))^2 + (b y1/(t+b^2))^2 - 1 in (-b^2, inf); F decreases
    there, so bisection finds it.  On the major axis (y1 = 0) inside the evolute
    the closest point leaves the axis and has a closed form."""
    X, Y = _mesh(n, lo, hi)
    if a < b:
        a, b = b, a
        angle = angle + math.pi / 2
    ca, sa = math.cos(angle), math.sin(angle)
    px, py = X - center[0], Y - center[1]
    # ellipse frame
    ex = ca * px + sa * py
    ey = -sa * px + ca * py
    sx, sy = np.sign(ex), np.sign(ey)
    y0, y1 = np.abs(ex), np.abs(ey)
    lo_t = np.full_like(y0, -b * b)
    hi_t = np.sqrt(a * a * y0 * y0 + b * b * y1 * y1) + 1e-300
    hi_t = np.maximum(hi_t, 0.0)
    def ratio(num, den, coord):
        # num/den where the coordinate is non-zero, 0 on the axis (where den may reach 0)
        return np.divide(num, den, out=np.zeros_like(num), where=coord > 0)

    for _ in range(iters):
        mid = 0.5 * (lo_t + hi_t)
        F = ratio(a * y0, mid + a * a, y0) ** 2 + ratio(b * y1, mid + b * b, y1) ** 2 - 1.0
        pos = F > 0
        lo_t = np.where(pos, mid, lo_t)
        hi_t = np.where(pos, hi_t, mid)
    t = 0.5 * (lo_t + hi_t)
    x0 = ratio(a * a * y0, t + a * a, y0)
    x1 = ratio(b * b * y1, t + b * b, y1)
    # major-axis special case
    axis = (y1 == 0)
    thr = (a * a - b * b) / a
    spec = axis & (y0 < thr)
    xs0 = a * a * y0 / (a * a - b * b)
    xs1 = b * np.sqrt(np.clip(1 - (xs0 / a) ** 2, 0.0, None))
    x0 = np.where(spec, xs0, np.where(axis, a, x0))
    x1 = np.where(spec, xs1, np.where(axis, 0.0, x1))
    d = np.hypot(y0 - x0, y1 - x1)
    inside = (y0 / a) ** 2 + (y1 / b) ** 2 < 1.0
    sgn = np.where(inside, -1.0, 1.0)
    # gradient: unit vector from the closest point, in the ellipse frame
    gx_e, gy_e = _unit(y0 - x0, y1 - x1)
    # on the curve itself, fall back to the ellipse normal
    nx_e, ny_e = _unit(x0 / (a * a), x1 / (b * b))
    on = d == 0
    gx_e = np.where(on, nx_e, sgn * gx_e)
    gy_e = np.where(on, ny_e, sgn * gy_e)
    gx_e *= np.where(sx == 0, 1.0, sx)
    gy_e *= np.where(sy == 0, 1.0, sy)
    # back to the grid frame
    gx = ca * gx_e - sa * gy_e
    gy = sa * gx_e + ca * gy_e
    return _state2d(sgn * d, gx, gy)


def linear2d(n, a=(0.3, -0.7), c=0.1, lo=None, hi=None):
    """phi = a.x + c (exact, zero cross derivative)."""
    X, Y = _mesh(n, lo, hi)
    phi = a[0] * X + a[1] * Y + c
    return _state2d(phi, np.full_like(phi, a[0]), np.full_like(phi, a[1]))


def polynomial2d(n, coef, lo=None, hi=None):
    """phi = sum_{p,q} coef[p,q] x^p y^q with exact phi_x, phi_y, phi_xy."""
    X, Y = _mesh(n, lo, hi)
    C = np.asarray(coef, dtype=np.float64)
    phi = np.zeros_like(X); px = np.zeros_like(X); py = np.zeros_like(X); pxy = np.zeros_like(X)
    for p in range(C.shape[0]):
        for q in range(C.shape[1]):
            c = C[p, q]
            if c == 0.0:
                continue
            phi += c * X ** p * Y ** q
            if p > 0:
                px += c * p * X ** (p - 1) * Y ** q
            if q > 0:
                py += c * q * X ** p * Y ** (q - 1)
            if p > 0 and q > 0:
                pxy += c * p * q * X ** (p - 1) * Y ** (q - 1)
    return _state2d(phi, px, py, pxy)


# ------------------------------------------------------------------ 3D initial data

def sphere_sdf(n, center=(0.35, 0.35, 0.35), r=0.15, lo=None, hi=None, dtype=np.float64,
               z_range=None):
    """Signed distance to a sphere with exact gradient and zero cross planes, built one
    z-slice at a time (so 512^3 fits in memory as float32).  z_range=(z0, z1) returns
    only those slices."""
    axes = node_coords(n, lo, hi)
    z0, z1 = (0, n[2]) if z_range is None else z_range
    out = np.zeros((8, z1 - z0, n[1], n[0]), dtype=dtype)
    Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
    dx, dy = X - center[0], Y - center[1]
    for k in range(z0, z1):
        dz = axes[2][k] - center[2]
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        safe = np.where(d > 0, d, 1.0)
        out[0, k - z0] = d - r
        out[1, k - z0] = np.where(d > 0, dx / safe, 0.0)
        out[2, k - z0] = np.where(d > 0, dy / safe, 0.0)
        out[3, k - z0] = np.where(d > 0, dz / safe, 0.0)
    return out


def slotted_sphere_sdf(n, center=(0.5, 0.75, 0.5), r=0.15, slot_w=0.05, slot_top=0.85,
                       lo=None, hi=None, dtype=np.float64, z_range=None):
    """Zalesak's slotted sphere (Sec. 6.2.3, rescaled to the unit box): the sphere minus
    the slot {|x - cx| < w/2, y < slot_top} (all z), which opens through the bottom of
    the sphere and ends at y = slot_top (depth 0.25 for the default sphere).  Level set
    function max(d_sphere, -d_slot) with d the signed distances to the sphere and to the
    slot region: its zero set is the slotted sphere exactly; it is the distance to that
    surface except near the slot's edges.  Gradient of the active branch (the sphere's
    on ties); zero cross planes.  Built one z-slice at a time; z_range=(z0, z1) returns
    only those slices."""
    axes = node_coords(n, lo, hi)
    z0, z1 = (0, n[2]) if z_range is None else z_range
    out = np.zeros((8, z1 - z0, n[1], n[0]), dtype=dtype)
    Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
    dx, dy = X - center[0], Y - center[1]
    hw = slot_w / 2
    # signed distance to the slot region and its gradient (independent of z)
    qx, qy = np.abs(dx) - hw, Y - slot_top
    sx = np.where(dx >= 0, 1.0, -1.0)
    ox, oy = np.maximum(qx, 0.0), np.maximum(qy, 0.0)
    dout = np.hypot(ox, oy)
    d_slot = dout + np.minimum(np.maximum(qx, qy), 0.0)
    safe = np.where(dout > 0, dout, 1.0)
    gsx = np.where(dout > 0, ox / safe * sx, np.where(qx >= qy, sx, 0.0))
    gsy = np.where(dout > 0, oy / safe, np.where(qx >= qy, 0.0, 1.0))
    for k in range(z0, z1):
        dz = axes[2][k] - center[2]
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        sd = np.where(d > 0, d, 1.0)
        d_sph = d - r
        use_sph = d_sph >= -d_slot
        out[0, k - z0] = np.where(use_sph, d_sph, -d_slot)
        out[1, k - z0] = np.where(use_sph, np.where(d > 0, dx / sd, 0.0), -gsx)
        out[2, k - z0] = np.where(use_sph, np.where(d > 0, dy / sd, 0.0), -gsy)
        out[3, k - z0] = np.where(use_sph, np.where(d > 0, dz / sd, 0.0), 0.0)
    return out


def cube_sdf(n, center=(0.35, 0.35, 0.35), half=0.15, lo=None, hi=None):
    """Exact signed distance to an axis-aligned cube and its gradient."""
    X, Y, Z = _mesh(n, lo, hi)
    P = [X - center[0], Y - center[1], Z - center[2]]
    q = [np.abs(p) - half for p in P]
    qp = [np.maximum(c, 0.0) for c in q]
    out = np.sqrt(qp[0] ** 2 + qp[1] ** 2 + qp[2] ** 2)
    qmax = np.maximum(np.maximum(q[0], q[1]), q[2])
    phi = out + np.minimum(qmax, 0.0)
    sg = [np.where(p >= 0, 1.0, -1.0) for p in P]
    safe = np.where(out > 0, out, 1.0)
    g_out = [np.where(out > 0, qp[i] / safe * sg[i], 0.0) for i in range(3)]
    # inside: gradient along the axis with the largest q (first on ties)
    ax = np.argmax(np.stack(q), axis=0)
    g_in = [np.where(ax == i, sg[i], 0.0) for i in range(3)]
    isout = qmax > 0
    g = [np.where(isout, g_out[i], g_in[i]) for i in range(3)]
    return _state3d(phi, g[0], g[1], g[2])


def linear3d(n, a=(0.3, -0.7, 0.2), c=0.1, lo=None, hi=None):
    X, Y, Z = _mesh(n, lo, hi)
    phi = a[0] * X + a[1] * Y + a[2] * Z + c
    return _state3d(phi, np.full_like(phi, a[0]), np.full_like(phi, a[1]),
                    np.full_like(phi, a[2]))


def gaussian_bump3d(n, x0=(0.5, 0.5, 0.5), r0=0.15, lo=None, hi=None):
    """exp(-|x-x0|^2) - exp(-r0^2) with all exact derivatives up to phi_xyz."""
    X, Y, Z = _mesh(n, lo, hi)
    dx, dy, dz = X - x0[0], Y - x0[1], Z - x0[2]
    e = np.exp(-(dx * dx + dy * dy + dz * dz))
    return _state3d(e - math.exp(-r0 * r0), -2 * dx * e, -2 * dy * e, -2 * dz * e,
                    [4 * dx * dy * e, 4 * dx * dz * e, 4 * dy * dz * e, -8 * dx * dy * dz * e])


# ------------------------------------------------------------------ velocity tables

def fourier_modes(nmodes, seed=DEFAULT_SEED, periodic=False, amp=0.1, kmax=4):
    """Random stream-function modes (a, k, l, n, chi) per row:
    a ~ N(0, amp^2), k, l uniform in {1..kmax}; steady fields have n = 0 and
    chi = 0; time-periodic ones n in {1, 2} and chi uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, amp, nmodes)
    k = rng.integers(1, kmax + 1, nmodes).astype(np.float64)
    l = rng.integers(1, kmax + 1, nmodes).astype(np.float64)
    if periodic:
        nn = rng.integers(1, 3, nmodes).astype(np.float64)
        chi = rng.uniform(0.0, 2 * math.pi, nmodes)
    else:
        nn = np.zeros(nmodes)
        chi = np.zeros(nmodes)
    return np.stack([a, k, l, nn, chi], axis=1)


def fourier_speed_bound(modes):
    """Upper bound on max_x,t |u| and |v| of the Fourier stream-function field:
    |u| <= sum |a| l pi, |v| <= sum |a| k pi."""
    m = np.asarray(modes)
    return float(max(np.sum(np.abs(m[:, 0]) * m[:, 2]) * math.pi,
                     np.sum(np.abs(m[:, 0]) * m[:, 1]) * math.pi))


def wave_modes(nmodes, seed=DEFAULT_SEED, amp=0.4, kmin=math.pi, kmax=4 * math.pi, periodic=True):
    """Random plane-wave stream-function modes (a, kx, ky, phase, n, chi) per row for the
    WAVES2D field Psi = sum a sin(kx x + ky y + phase) cos(2 pi n t + chi): wave vectors of
    uniform direction and length uniform in [kmin, kmax], a ~ N(0, (amp / sqrt(nmodes))^2)
    (the field's typical speed does not grow with the number of modes), phase uniform in
    [0, 2 pi); time-periodic fields (period 1) have n in {1, 2} and chi uniform in
    [0, 2 pi), steady ones n = chi = 0."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, amp / math.sqrt(nmodes), nmodes)
    ang = rng.uniform(0.0, 2 * math.pi, nmodes)
    kk = rng.uniform(kmin, kmax, nmodes)
    phase = rng.uniform(0.0, 2 * math.pi, nmodes)
    if periodic:
        nn = rng.integers(1, 3, nmodes).astype(np.float64)
        chi = rng.uniform(0.0, 2 * math.pi, nmodes)
    else:
        nn = np.zeros(nmodes)
        chi = np.zeros(nmodes)
    return np.stack([a, kk * np.cos(ang), kk * np.sin(ang), phase, nn, chi], axis=1)


def wave_velocity(modes, x, y, t):
    """(u, v) of the WAVES2D field at points (x, y) (arrays) and time t, in FP64 (numpy);
    for sampling the field's speed, not a reference of the method."""
    m = np.asarray(modes)
    u = np.zeros(np.broadcast(x, y).shape)
    v = np.zeros_like(u)
    for a, kx, ky, ph, n, chi in m:
        c = a * math.cos(2 * math.pi * n * t + chi) * np.cos(kx * x + ky * y + ph)
        u -= ky * c
        v += kx * c
    return u, v


def wave_speed_sampled(modes, samples=129, times=12):
    """max over [0,1]^2 and one period of max(|u|, |v|), sampled on a samples^2 grid at
    `times` phases, times 1.1 (the CFL rule of the Fourier configurations, with margin)."""
    xs = np.linspace(0.0, 1.0, samples)
    X, Y = np.meshgrid(xs, xs)
    best = 0.0
    for k in range(times):
        u, v = wave_velocity(modes, X, Y, k / times)
        best = max(best, float(np.max(np.abs(u))), float(np.max(np.abs(v))))
    return 1.1 * best


def wave_speed_bound(modes):
    """Upper bound of max |u|, |v| of the WAVES2D field: sum |a| |k| (the library's)."""
    m = np.asarray(modes)
    return float(np.sum(np.abs(m[:, 0]) * np.hypot(m[:, 1], m[:, 2])))


def steps_for(T, h, vmax, cfl=1.0):
    """nsteps = ceil(T / dt_cfl) with dt_cfl = cfl h / vmax; dt = T / nsteps."""
    nsteps = int(math.ceil(T / (cfl * h / vmax) - 1e-9))
    return nsteps, T / nsteps


@dataclass
class BatchProblem:
    n: int
    center: tuple
    a: float
    b: float
    angle: float
    modes: np.ndarray = field(repr=False)
    dt: float = 0.0


def batch_problems(count=256, seed=DEFAULT_SEED, nmin=128, nmax=1024, nmodes=8):
    """Independent 2D problems of uneven size: side n uniform in [nmin, nmax], an
    ellipse (semi-axes uniform in [0.05, 0.2], centre uniform in [0.3, 0.7]^2,
    angle uniform in [0, pi)) and its own steady Fourier field; dt from CFL 1."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        c = (float(rng.uniform(0.3, 0.7)), float(rng.uniform(0.3, 0.7)))
        a = float(rng.uniform(0.05, 0.2))
        b = float(rng.uniform(0.05, 0.2))
        ang = float(rng.uniform(0.0, math.pi))
        modes = fourier_modes(nmodes, seed=int(rng.integers(0, 2 ** 31)))
        vmax = fourier_speed_bound(modes)
        h = 1.0 / (n - 1)
        dt = h / vmax
        probs.append(BatchProblem(n=n, center=c, a=a, b=b, angle=ang, modes=modes, dt=dt))
    return probs


def random_state(shape_planes, seed=DEFAULT_SEED, scale=1.0):
    """O(1) random values for parity tests of a single step (any plane count)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, shape_planes)
