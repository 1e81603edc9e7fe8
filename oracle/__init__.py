"""FP64 CPU oracle for the gradient-augmented level set (GALS) step.

TEST INFRASTRUCTURE ONLY.  This package implements the scheme of Nave, Rosales
and Seibold (arXiv 0905.3409) as plain, slow, direct C code (``*.c`` beside this
file) so that the CUDA path can be checked against it.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library and never loads it.

The binding below only marshals numpy arrays into the C functions declared in
``gals_oracle.h``; all arithmetic of the method lives in the C sources.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["hermite.c", "velocity.c", "trace.c", "step.c", "diag.c", "mlp.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# enums of gals_oracle.h
VEL_CONST, VEL_ROTATION, VEL_VORTEX2D, VEL_DEFORM3D, VEL_PSEUDO1D, VEL_FOURIER2D, VEL_WAVES2D = range(7)
TRACE_EULER, TRACE_RK3, TRACE_HEUN_PSI = 0, 1, 2
CROSS_CENTRAL, CROSS_ZERO, CROSS_CELL = 0, 1, 2
_CROSS_NAMES = {"central": CROSS_CENTRAL, "zero": CROSS_ZERO, "cell": CROSS_CELL}

_VEL_NAMES = {
    "const": VEL_CONST, "rotation": VEL_ROTATION, "vortex2d": VEL_VORTEX2D,
    "deform3d": VEL_DEFORM3D, "pseudo1d": VEL_PSEUDO1D, "fourier2d": VEL_FOURIER2D,
    "waves2d": VEL_WAVES2D,
}
_TRACE_NAMES = {"euler": TRACE_EULER, "rk3": TRACE_RK3, "heun_psi": TRACE_HEUN_PSI}


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``liboracle.so`` (gcc, OpenMP, no FMA
    contraction so that x86 and Arm hosts round identically)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "gals_oracle.h")])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Velocity(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("T", ctypes.c_double), ("omega", ctypes.c_double),
                ("center", ctypes.c_double * 3), ("c", ctypes.c_double * 3),
                ("nmodes", ctypes.c_int), ("modes", ctypes.POINTER(ctypes.c_double))]


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("h", ctypes.c_double * 3), ("cross", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(dp)
            L.orc_basis1d.argtypes = [ctypes.c_double, dp, dp]
            L.orc_hermite_cell.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
            L.orc_vel_eval.argtypes = [ctypes.POINTER(_Velocity), ctypes.c_int, dp,
                                       ctypes.c_double, dp, dp]
            L.orc_trace.argtypes = [ctypes.c_int, ctypes.POINTER(_Velocity), ctypes.c_int, dp,
                                    ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_flowmap_rk4.argtypes = [ctypes.POINTER(_Velocity), ctypes.c_int, dp,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
            L.orc_recon_cross.argtypes = [ctypes.POINTER(_Grid), pp]
            L.orc_node_update.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Velocity),
                                          ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, pp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, dp, dp]
            L.orc_step.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Velocity), ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double, pp, pp,
                                   ctypes.c_int]
            L.orc_step_given.argtypes = [ctypes.POINTER(_Grid), ctypes.c_int, pp, pp, pp, pp,
                                         ctypes.c_int]
            L.orc_step_nodes.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Velocity),
                                         ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, pp, ctypes.c_long,
                                         ctypes.POINTER(ctypes.c_long), dp, ctypes.c_int]
            L.orc_step_band.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Velocity),
                                        ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, pp, ctypes.c_int, ctypes.c_int, pp,
                                        ctypes.c_int]
            L.orc_run.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Velocity), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  pp, pp, ctypes.c_int]
            L.orc_emax.argtypes = [ctypes.c_long, dp, dp]
            L.orc_emax.restype = ctypes.c_double
            L.orc_measure_negative.argtypes = [ctypes.POINTER(_Grid), pp, ctypes.c_int,
                                               ctypes.c_int]
            L.orc_measure_negative.restype = ctypes.c_double
            L.orc_symdiff.argtypes = [ctypes.POINTER(_Grid), pp, pp, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_long),
                                      ctypes.c_int]
            L.orc_symdiff.restype = ctypes.c_double
            L.orc_eval_points.argtypes = [ctypes.POINTER(_Grid), pp, ctypes.c_long, dp, dp, dp]
            L.orc_hermite_cell2.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_curvature_points.argtypes = [ctypes.POINTER(_Grid), pp, ctypes.c_long, dp, dp,
                                               dp, dp]
            _mlp_bind(L)
            _lib = L
    return _lib


def _mlp_bind(L):
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_mlp_forward.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, ctypes.c_long,
                                  dp, dp, dp]
    L.orc_mlp_backward.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, ctypes.c_long,
                                   dp, dp, dp, dp]
    L.orc_mlp_backward.restype = ctypes.c_double
    L.orc_adam_update.argtypes = [ctypes.c_long, dp, dp, dp, dp, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int]


def default_threads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


# ---------------------------------------------------------------- marshalling helpers

def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def velocity(kind: str, T: float = 1.0, omega: float = 0.0, center=(0.5, 0.5, 0.5),
             c=(0.0, 0.0, 0.0), modes=None):
    """Build the oracle's velocity descriptor.  ``modes``: (m,5) array of
    (a, k, l, n, chi) for the Fourier stream-function field, (m,6) array of
    (a, kx, ky, phase, n, chi) for the plane-wave field."""
    v = _Velocity()
    v.kind = _VEL_NAMES[kind]
    v.T = float(T)
    v.omega = float(omega)
    for i in range(3):
        v.center[i] = float(center[i]) if i < len(center) else 0.0
        v.c[i] = float(c[i]) if i < len(c) else 0.0
    if modes is not None:
        m = _f64(modes).reshape(-1, 6 if kind == "waves2d" else 5)
        v._modes_keep = m  # keep alive
        v.nmodes = m.shape[0]
        v.modes = _dp(m)
    else:
        v.nmodes = 0
        v.modes = None
    return v


def grid(n, lo=None, hi=None, cross="central"):
    """Grid of ``n`` nodes per axis on [lo, hi] (both ends are nodes).  ``cross``: the
    cross derivatives the diagnostics' interpolant uses ("central": the stored planes,
    "cell": approach (B) per cell)."""
    dim = len(n)
    lo = [0.0] * dim if lo is None else list(lo)
    hi = [1.0] * dim if hi is None else list(hi)
    g = _Grid()
    g.dim = dim
    g.cross = _CROSS_NAMES[cross]
    for i in range(3):
        g.n[i] = int(n[i]) if i < dim else 1
        g.lo[i] = float(lo[i]) if i < dim else 0.0
        g.h[i] = (float(hi[i]) - float(lo[i])) / (int(n[i]) - 1) if i < dim else 1.0
    return g


def nplanes(dim: int) -> int:
    return {1: 2, 2: 4, 3: 8}[dim]


def _planes_ptr(planes):
    arr = (ctypes.POINTER(ctypes.c_double) * len(planes))(*[_dp(p) for p in planes])
    return arr


def _state_list(state, g):
    """state: array (nplanes, *shape) with x fastest -> list of contiguous planes."""
    st = _f64(state)
    np_ = nplanes(g.dim)
    assert st.shape[0] == np_, (st.shape, np_)
    return [np.ascontiguousarray(st[p]).reshape(-1) for p in range(np_)]


# ---------------------------------------------------------------- public oracle calls

def basis1d(xi: float):
    w = np.zeros(4)
    dw = np.zeros(4)
    lib().orc_basis1d(float(xi), _dp(w), _dp(dw))
    return w, dw


def hermite_cell(dim: int, data, h, xi):
    data = _f64(data).reshape(-1)
    assert data.size == 4 ** dim
    hh = _f64(list(h) + [1.0] * (3 - len(h)))
    xx = _f64(list(xi) + [0.0] * (3 - len(xi)))
    H = np.zeros(1)
    g = np.zeros(3)
    lib().orc_hermite_cell(dim, _dp(data), _dp(hh), _dp(xx), _dp(H), _dp(g))
    return H[0], g[:dim].copy()


def vel_eval(vel, dim, x, t):
    xx = _f64(list(x) + [0.0] * (3 - len(x)))
    v = np.zeros(3)
    D = np.zeros(9)
    lib().orc_vel_eval(ctypes.byref(vel), dim, _dp(xx), float(t), _dp(v), _dp(D))
    return v[:dim].copy(), D.reshape(3, 3)[:dim, :dim].copy()


def trace(scheme: str, vel, dim, x, t, dt):
    xx = _f64(list(x) + [0.0] * (3 - len(x)))
    foot = np.zeros(3)
    J = np.zeros(9)
    lib().orc_trace(_TRACE_NAMES[scheme], ctypes.byref(vel), dim, _dp(xx), float(t), float(dt),
                    _dp(foot), _dp(J))
    return foot[:dim].copy(), J.reshape(3, 3)[:dim, :dim].copy()


def flowmap_rk4(vel, dim, x, t, dt, m=32):
    xx = _f64(list(x) + [0.0] * (3 - len(x)))
    foot = np.zeros(3)
    J = np.zeros(9)
    lib().orc_flowmap_rk4(ctypes.byref(vel), dim, _dp(xx), float(t), float(dt), int(m),
                          _dp(foot), _dp(J))
    return foot[:dim].copy(), J.reshape(3, 3)[:dim, :dim].copy()


def recon_cross(g, state):
    planes = [p.copy() for p in _state_list(state, g)]
    lib().orc_recon_cross(ctypes.byref(g), _planes_ptr(planes))
    return np.stack(planes).reshape(np.shape(state))


def step(g, vel, state, t, dt, trace_scheme="rk3", cross="central", nthreads=None):
    shape = np.shape(state)
    ins = _state_list(state, g)
    outs = [np.empty_like(p) for p in ins]
    lib().orc_step(ctypes.byref(g), ctypes.byref(vel), _TRACE_NAMES[trace_scheme],
                   _CROSS_NAMES[cross], float(t), float(dt),
                   _planes_ptr(ins), _planes_ptr(outs),
                   default_threads() if nthreads is None else int(nthreads))
    return np.stack(outs).reshape(shape)


def step_given(g, state, disp, jac, cross="central", nthreads=None):
    """One step with the backward map given per node instead of traced: ``disp`` is
    (dim, *grid) of foot - x, ``jac`` is (dim, dim, *grid) with jac[a, b] = d foot_a / d x_b."""
    shape = np.shape(state)
    ins = _state_list(state, g)
    dim = g.dim
    d = [np.ascontiguousarray(np.asarray(disp[a], dtype=np.float64)).ravel() for a in range(dim)]
    J = [np.ascontiguousarray(np.asarray(jac[a][b], dtype=np.float64)).ravel()
         for a in range(dim) for b in range(dim)]
    outs = [np.empty_like(p) for p in ins]
    lib().orc_step_given(ctypes.byref(g), _CROSS_NAMES[cross], _planes_ptr(ins), _planes_ptr(d),
                         _planes_ptr(J), _planes_ptr(outs),
                         default_threads() if nthreads is None else int(nthreads))
    return np.stack(outs).reshape(shape)


def step_nodes(g, vel, state, t, dt, nodes, trace_scheme="rk3", cross="central",
               nthreads=None):
    """New state (all planes) at flat node indices ``nodes`` -> (len(nodes), nplanes)."""
    ins = _state_list(state, g)
    sel = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((sel.size, nplanes(g.dim)))
    lib().orc_step_nodes(ctypes.byref(g), ctypes.byref(vel), _TRACE_NAMES[trace_scheme],
                         _CROSS_NAMES[cross], float(t),
                         float(dt), _planes_ptr(ins), sel.size,
                         sel.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out),
                         default_threads() if nthreads is None else int(nthreads))
    return out


def step_band(g, vel, state, t, dt, b0, b1, trace_scheme="rk3", cross="central", nthreads=None,
              planes=None):
    """New state of the outermost-axis band [b0, b1) (rows in 2D, z-slices in 3D);
    returns (nplanes, b1-b0, ...) with the inner axes of the grid.  ``planes``: the
    state already split by ``state_planes`` (avoids re-copying a large state)."""
    ins = planes if planes is not None else _state_list(state, g)
    inner = (g.n[0],) if g.dim == 2 else (g.n[1], g.n[0])
    outs = [np.empty((b1 - b0) * int(np.prod(inner))) for _ in ins]
    lib().orc_step_band(ctypes.byref(g), ctypes.byref(vel), _TRACE_NAMES[trace_scheme],
                        _CROSS_NAMES[cross], float(t), float(dt),
                        _planes_ptr(ins), int(b0), int(b1), _planes_ptr(outs),
                        default_threads() if nthreads is None else int(nthreads))
    return np.stack(outs).reshape((len(ins), b1 - b0) + inner)


def state_planes(g, state):
    """Split a state into the contiguous FP64 planes the C calls take."""
    return _state_list(state, g)


def run(g, vel, state, t0, dt, nsteps, trace_scheme="rk3", cross="central", nthreads=None):
    shape = np.shape(state)
    st = [p.copy() for p in _state_list(state, g)]  # never write into the caller's array
    scratch = [np.empty_like(p) for p in st]
    lib().orc_run(ctypes.byref(g), ctypes.byref(vel), _TRACE_NAMES[trace_scheme],
                  _CROSS_NAMES[cross], float(t0), float(dt),
                  int(nsteps), _planes_ptr(st), _planes_ptr(scratch),
                  default_threads() if nthreads is None else int(nthreads))
    return np.stack(st).reshape(shape)


def emax(a, b) -> float:
    a = _f64(a).reshape(-1)
    b = _f64(b).reshape(-1)
    return lib().orc_emax(a.size, _dp(a), _dp(b))


def measure_negative(g, state, q, nthreads=None) -> float:
    planes = _state_list(state, g)
    return lib().orc_measure_negative(ctypes.byref(g), _planes_ptr(planes), int(q),
                                      default_threads() if nthreads is None else int(nthreads))


def symdiff(g, a, b, q, eps=0.0, nthreads=None):
    pa = _state_list(a, g)
    pb = _state_list(b, g)
    amb = ctypes.c_long(0)
    v = lib().orc_symdiff(ctypes.byref(g), _planes_ptr(pa), _planes_ptr(pb), int(q), float(eps),
                          ctypes.byref(amb),
                          default_threads() if nthreads is None else int(nthreads))
    return v, amb.value


def eval_points(g, state, pts):
    planes = _state_list(state, g)
    P = _f64(pts).reshape(-1, g.dim)
    H = np.zeros(P.shape[0])
    G = np.zeros(P.shape)
    lib().orc_eval_points(ctypes.byref(g), _planes_ptr(planes), P.shape[0], _dp(P), _dp(H), _dp(G))
    return H, G


def hermite_cell2(dim: int, data, h, xi):
    """H, grad H and the Hessian of the p-cubic interpolant of one cell (Sec. 3.4)."""
    d = _f64(data).ravel()
    H = np.zeros(1)
    G = np.zeros(dim)
    Hs = np.zeros(dim * dim)
    lib().orc_hermite_cell2(dim, _dp(d), _dp(_f64(h)), _dp(_f64(xi)), _dp(H), _dp(G), _dp(Hs))
    return H[0], G, Hs.reshape(dim, dim)


def curvature_points(g, state, pts):
    """H, unit normal and curvature at points from the interpolant (Sec. 3.4)."""
    planes = _state_list(state, g)
    P = _f64(pts).reshape(-1, g.dim)
    H = np.zeros(P.shape[0])
    N = np.zeros(P.shape)
    K = np.zeros(P.shape[0])
    lib().orc_curvature_points(ctypes.byref(g), _planes_ptr(planes), P.shape[0], _dp(P), _dp(H),
                               _dp(N), _dp(K))
    return H, N, K


# ---------------------------------------------------------------- MLP (surrogate oracle)

def mlp_param_count(sizes) -> int:
    return int(sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1)))


def mlp_forward(sizes, params, X):
    sz = (ctypes.c_int * len(sizes))(*sizes)
    p = _f64(params)
    Xc = _f64(X).reshape(-1, sizes[0])
    Y = np.zeros((Xc.shape[0], sizes[-1]))
    lib().orc_mlp_forward(len(sizes) - 1, sz, _dp(p), Xc.shape[0], _dp(Xc), _dp(Y), None)
    return Y


def mlp_backward(sizes, params, X, T):
    """MSE loss over batch and outputs and its gradient w.r.t. the flat parameters."""
    sz = (ctypes.c_int * len(sizes))(*sizes)
    p = _f64(params)
    Xc = _f64(X).reshape(-1, sizes[0])
    Tc = _f64(T).reshape(-1, sizes[-1])
    grad = np.zeros(p.size)
    loss = lib().orc_mlp_backward(len(sizes) - 1, sz, _dp(p), Xc.shape[0], _dp(Xc), _dp(Tc),
                                  _dp(grad), None)
    return loss, grad


def adam_update(params, grad, m, v, lr, b1, b2, eps, step):
    """In-place Adam step on float64 arrays (returns them for convenience)."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(grad)
    lib().orc_adam_update(params.size, _dp(params), _dp(g), _dp(m), _dp(v), float(lr), float(b1),
                          float(b2), float(eps), int(step))
    return params, m, v
