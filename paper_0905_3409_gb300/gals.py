"""Thin Python binding of the C ABI in ``include/gals.h`` (ctypes).

Only argument marshalling happens here: every step of the method runs in the CUDA
kernels of ``libgals.so``.  PyTorch is used for device memory (device tensors are
passed by pointer) and for streams.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GALS_LIB selects another build of the same ABI (the checked build, libgals_checked.so)
LIB_PATH = os.environ.get("GALS_LIB") or os.path.join(_HERE, "libgals.so")

# enums of gals.h
OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE, ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
MEM_HOST, MEM_DEVICE = 0, 1
LAYOUT_FULL, LAYOUT_COMPACT = 0, 1
VEL = {"const": 0, "rotation": 1, "vortex2d": 2, "deform3d": 3, "pseudo1d": 4, "fourier2d": 5,
       "waves2d": 6}
TRACE = {"euler": 0, "rk3": 1, "surrogate": 2, "heun_psi": 3}
SET_RECON_CROSS = 1
MAX_MODES = 64
MAX_WAVES = 1024

# every symbol include/gals.h declares
EXPORTS = [
    "gals_create_grid", "gals_destroy_grid", "gals_set_state", "gals_step", "gals_read_state",
    "gals_diagnostics", "gals_synchronize", "gals_step_host", "gals_step_host_async", "gals_eval_points", "gals_time", "gals_state_planes", "gals_last_error",
    "gals_version",
    "gals_create_batch", "gals_destroy_batch", "gals_batch_set_state", "gals_batch_step",
    "gals_batch_read_state", "gals_batch_synchronize", "gals_batch_autotune",
    "gals_batch_set_tuning", "gals_batch_get_tuning", "gals_batch_nodes", "gals_batch_last_error",
    "gals_diagnostics_noalloc", "gals_noalloc_max_nodes", "gals_noalloc_last_error",
    "gals_checked_wait_test", "gals_set_time_loop", "gals_last_step_launches",
    "gals_surrogate_create", "gals_surrogate_destroy", "gals_surrogate_train",
    "gals_surrogate_set_check", "gals_surrogate_stats", "gals_surrogate_get_params",
    "gals_surrogate_set_params", "gals_surrogate_bind", "gals_surrogate_forward",
    "gals_surrogate_gradient", "gals_surrogate_targets", "gals_surrogate_last_error",
    "gals_surrogate_forward_device", "gals_surrogate_save", "gals_surrogate_load",
]


class BatchTuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("blocks", ctypes.c_int), ("ms_per_step", ctypes.c_double),
                ("loop", ctypes.c_int)]


class GalsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gals status {status}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("layout", ctypes.c_int), ("cross_scheme", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class VelocityDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("trace", ctypes.c_int), ("T", ctypes.c_double),
                ("omega", ctypes.c_double), ("center", ctypes.c_double * 3), ("c", ctypes.c_double * 3),
                ("nmodes", ctypes.c_int), ("modes", ctypes.POINTER(ctypes.c_double)),
                ("surrogate", ctypes.c_void_p)]


class MlpDesc(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("lr_min", ctypes.c_double), ("substeps", ctypes.c_int), ("seed", ctypes.c_uint64)]


class TrainReport(ctypes.Structure):
    _fields_ = [("initial_loss", ctypes.c_double), ("final_loss", ctypes.c_double),
                ("seconds", ctypes.c_double), ("steps", ctypes.c_int)]


MLP_PARAMS = 50822
MLP_SIZES = [3, 128, 128, 128, 128, 6]


class DiagRequest(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("reference", ctypes.c_void_p)]


class DiagOut(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("n_negative", ctypes.c_int64), ("measure_negative", ctypes.c_double),
                ("n_symdiff", ctypes.c_int64), ("measure_symdiff", ctypes.c_double),
                ("emax_phi", ctypes.c_double), ("emax_psi", ctypes.c_double),
                ("l2_phi", ctypes.c_double), ("nonfinite", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load ``libgals.so`` (built by ``paper_0905_3409_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.gals_create_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
        L.gals_destroy_grid.argtypes = [vp]
        L.gals_set_state.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int]
        L.gals_step.argtypes = [vp, ctypes.POINTER(VelocityDesc), ctypes.c_double, ctypes.c_int]
        L.gals_read_state.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
        L.gals_diagnostics.argtypes = [vp, ctypes.POINTER(DiagRequest), ctypes.POINTER(DiagOut)]
        L.gals_synchronize.argtypes = [vp]
        L.gals_step_host.argtypes = [vp, ctypes.POINTER(VelocityDesc), ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.gals_step_host_async.argtypes = L.gals_step_host.argtypes
        L.gals_eval_points.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int, vp, vp, vp]
        L.gals_time.argtypes = [vp]
        L.gals_time.restype = ctypes.c_double
        L.gals_state_planes.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64)]
        L.gals_last_error.argtypes = [vp]
        L.gals_last_error.restype = ctypes.c_char_p
        L.gals_version.restype = ctypes.c_char_p
        L.gals_create_batch.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int, ctypes.POINTER(vp)]
        L.gals_destroy_batch.argtypes = [vp]
        L.gals_batch_set_state.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.gals_batch_step.argtypes = [vp, ctypes.POINTER(VelocityDesc),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.gals_batch_read_state.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int,
                                            ctypes.c_int]
        L.gals_batch_synchronize.argtypes = [vp]
        L.gals_batch_autotune.argtypes = [vp, ctypes.POINTER(VelocityDesc),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                          ctypes.POINTER(BatchTuning)]
        L.gals_batch_set_tuning.argtypes = [vp, ctypes.POINTER(BatchTuning)]
        L.gals_batch_get_tuning.argtypes = [vp, ctypes.POINTER(BatchTuning)]
        L.gals_batch_nodes.argtypes = [vp]
        L.gals_batch_nodes.restype = ctypes.c_int64
        L.gals_batch_last_error.argtypes = [vp]
        L.gals_batch_last_error.restype = ctypes.c_char_p
        L.gals_diagnostics_noalloc.argtypes = [
            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
            ctypes.POINTER(ctypes.c_double), vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
            vp, ctypes.POINTER(DiagOut)]
        L.gals_noalloc_max_nodes.restype = ctypes.c_int64
        L.gals_noalloc_last_error.restype = ctypes.c_char_p
        L.gals_checked_wait_test.argtypes = [ctypes.c_uint32, ctypes.c_int]
        L.gals_last_step_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        fp = ctypes.POINTER(ctypes.c_float)
        L.gals_surrogate_create.argtypes = [ctypes.POINTER(MlpDesc), ctypes.POINTER(vp)]
        L.gals_surrogate_destroy.argtypes = [vp]
        L.gals_surrogate_train.argtypes = [vp, ctypes.POINTER(VelocityDesc), ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(TrainOpts),
                                           ctypes.POINTER(TrainReport)]
        L.gals_surrogate_set_check.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.gals_surrogate_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        L.gals_surrogate_get_params.argtypes = [vp, fp, fp]
        L.gals_surrogate_set_params.argtypes = [vp, fp, fp]
        L.gals_surrogate_bind.argtypes = [vp, ctypes.POINTER(VelocityDesc), ctypes.c_double,
                                          ctypes.c_double]
        L.gals_surrogate_forward.argtypes = [vp, fp, ctypes.c_int, fp]
        L.gals_surrogate_forward_device.argtypes = [vp, vp, ctypes.c_int64, vp]
        L.gals_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        L.gals_surrogate_load.argtypes = [vp, ctypes.c_char_p]
        L.gals_surrogate_gradient.argtypes = [vp, fp, fp, ctypes.c_int, fp,
                                              ctypes.POINTER(ctypes.c_double)]
        L.gals_surrogate_targets.argtypes = [vp, ctypes.POINTER(VelocityDesc), ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, fp, ctypes.c_int, fp]
        L.gals_surrogate_last_error.argtypes = [vp]
        L.gals_surrogate_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, handle=None):
    if status != OK:
        msg = lib().gals_last_error(handle)
        raise GalsError(status, msg.decode() if msg else "")


@dataclass
class Velocity:
    """Analytic velocity field descriptor (see gals.h for the kinds)."""
    kind: str
    trace: str = "rk3"
    T: float = 1.0
    omega: float = 0.0
    center: tuple = (0.5, 0.5, 0.5)
    c: tuple = (0.0, 0.0, 0.0)
    modes: np.ndarray | None = None
    surrogate: "Surrogate | None" = None

    def desc(self) -> VelocityDesc:
        d = VelocityDesc()
        d.kind = VEL[self.kind]
        d.trace = TRACE[self.trace]
        d.T = float(self.T)
        d.omega = float(self.omega)
        for i in range(3):
            d.center[i] = float(self.center[i]) if i < len(self.center) else 0.0
            d.c[i] = float(self.c[i]) if i < len(self.c) else 0.0
        if self.modes is not None:
            m = np.ascontiguousarray(self.modes, dtype=np.float64).reshape(-1, 6 if self.kind == "waves2d" else 5)
            d._keep = m
            d.nmodes = m.shape[0]
            d.modes = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if self.surrogate is not None:
            d.surrogate = self.surrogate.handle.value
        return d


def _nplanes(dim):
    return 4 if dim == 2 else 8


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Grid:
    """A GALS grid on the current CUDA device.

    ``n``: nodes per axis (x first); the state arrays have shape
    (nplanes, [nz,] ny, nx) with x fastest."""

    def __init__(self, n, lo=None, hi=None, layout: str = "full", stream=None, cross: str = "central"):
        dim = len(n)
        d = GridDesc()
        d.dim = dim
        lo = [0.0] * dim if lo is None else list(lo)
        hi = [1.0] * dim if hi is None else list(hi)
        for i in range(3):
            d.n[i] = int(n[i]) if i < dim else 1
            d.lo[i] = float(lo[i]) if i < dim else 0.0
            d.hi[i] = float(hi[i]) if i < dim else 1.0
        d.layout = LAYOUT_FULL if layout == "full" else LAYOUT_COMPACT
        d.cross_scheme = {"central": 0, "cell": 1}[cross]
        if stream is not None:
            d.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        h = ctypes.c_void_p()
        _check(lib().gals_create_grid(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.nplanes = _nplanes(dim)
        self.shape = (self.nplanes,) + tuple(reversed(self.n))
        self._pending_host = []  # host arrays of asynchronous host steps, until synchronize()

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().gals_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- state
    def set_state(self, state, t0: float = 0.0, recon: bool = False):
        """state: numpy array (host) or torch CUDA tensor (device), float32 planes;
        1+dim planes (cross derivatives rebuilt) or all planes.  The data is copied before
        the call returns."""
        nf = state.shape[0]
        if _is_torch(state):
            import torch
            assert state.is_cuda and state.dtype == torch.float32
            st = state.contiguous()
            torch.cuda.current_stream().synchronize()  # producer work on torch's stream
            ptrs = (ctypes.c_void_p * nf)(*[st[p].data_ptr() for p in range(nf)])
            mem = MEM_DEVICE
        else:
            st = np.ascontiguousarray(state, dtype=np.float32)
            ptrs = (ctypes.c_void_p * nf)(*[st[p].ctypes.data for p in range(nf)])
            mem = MEM_HOST
        _check(lib().gals_set_state(self._h, ptrs, nf, mem, float(t0),
                                    SET_RECON_CROSS if recon else 0), self._h)

    def step(self, vel: Velocity, dt: float, nsteps: int = 1):
        d = vel.desc()
        _check(lib().gals_step(self._h, ctypes.byref(d), float(dt), int(nsteps)), self._h)

    def set_time_loop(self, mode: str):
        """"launches" (one launch per step, the default) or "persistent" (one launch per
        multi-step call where it applies)."""
        _check(lib().gals_set_time_loop(self._h, {"launches": 0, "persistent": 1}[mode]), self._h)

    def last_step_launches(self) -> int:
        """Kernel launches of the last step() call (step kernels per band, coefficient and
        clock kernels)."""
        n = ctypes.c_int64(0)
        _check(lib().gals_last_step_launches(self._h, ctypes.byref(n)), self._h)
        return n.value

    def read_state(self, out=None, nfields=None):
        """Copy the state into ``out`` (numpy or torch CUDA tensor of self.shape);
        returns a new host array if out is None."""
        nf = self.nplanes if nfields is None else int(nfields)
        if out is None:
            out = np.empty((nf,) + self.shape[1:], dtype=np.float32)
        if _is_torch(out):
            import torch
            assert out.is_cuda and out.is_contiguous()
            torch.cuda.current_stream().synchronize()
            ptrs = (ctypes.c_void_p * nf)(*[out[p].data_ptr() for p in range(nf)])
            mem = MEM_DEVICE
        else:
            assert out.dtype == np.float32 and out.flags.c_contiguous
            ptrs = (ctypes.c_void_p * nf)(*[out[p].ctypes.data for p in range(nf)])
            mem = MEM_HOST
        _check(lib().gals_read_state(self._h, ptrs, nf, mem), self._h)
        return out

    def diagnostics(self, q: int = 0, reference: "Grid | None" = None) -> dict:
        req = DiagRequest()
        req.q = int(q)
        req.reference = reference._h.value if reference is not None else None
        out = DiagOut()
        _check(lib().gals_diagnostics(self._h, ctypes.byref(req), ctypes.byref(out)), self._h)
        return {f: getattr(out, f) for f, _ in DiagOut._fields_}

    def synchronize(self):
        _check(lib().gals_synchronize(self._h), self._h)
        self._pending_host = []

    def eval_points(self, points):
        """Value, unit normal and curvature of the interpolant at points (npts x dim).
        Host arrays (numpy) or CUDA tensors (torch, float64 points): the results live in
        the same memory as the points."""
        dim = len(self.n)
        if _is_torch(points):
            import torch
            P = points.contiguous()
            assert P.is_cuda and P.dtype == torch.float64 and P.shape[-1] == dim
            m = P.numel() // dim
            H = torch.empty(m, dtype=torch.float32, device=P.device)
            N = torch.empty((m, dim), dtype=torch.float32, device=P.device)
            K = torch.empty(m, dtype=torch.float32, device=P.device)
            torch.cuda.current_stream().synchronize()
            _check(lib().gals_eval_points(self._h, P.data_ptr(), m, MEM_DEVICE, H.data_ptr(),
                                          N.data_ptr(), K.data_ptr()), self._h)
            return H, N, K
        P = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, dim)
        m = P.shape[0]
        H = np.empty(m, dtype=np.float32)
        N = np.empty((m, dim), dtype=np.float32)
        K = np.empty(m, dtype=np.float32)
        _check(lib().gals_eval_points(self._h, P.ctypes.data, m, MEM_HOST, H.ctypes.data,
                                      N.ctypes.data, K.ctypes.data), self._h)
        return H, N, K

    def step_host(self, vel: Velocity, dt: float, t0: float, state, out=None, wait=True):
        """One step from the host state ``state`` (all planes, at time t0) to ``out`` (a new
        host array if None), with the copies overlapped with the step in bands; the grid
        keeps the new state.  Page-locked (pinned) arrays let the copies overlap.  With
        ``wait=False`` (gals_step_host_async) the call returns once the work is queued:
        ``state`` must be a C-contiguous float32 array, and neither it may be changed nor
        ``out`` read before synchronize(); the grid keeps both arrays alive until then."""
        if wait:
            st = np.ascontiguousarray(state, dtype=np.float32)
        else:
            st = state
            assert isinstance(st, np.ndarray) and st.dtype == np.float32 and st.flags.c_contiguous
        assert st.shape == self.shape, (st.shape, self.shape)
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.shape == self.shape
        nf = self.nplanes
        pin = (ctypes.c_void_p * nf)(*[st[p].ctypes.data for p in range(nf)])
        pout = (ctypes.c_void_p * nf)(*[out[p].ctypes.data for p in range(nf)])
        d = vel.desc()
        call = lib().gals_step_host if wait else lib().gals_step_host_async
        _check(call(self._h, ctypes.byref(d), float(dt), float(t0), pin, pout), self._h)
        if not wait:
            self._pending_host.append((st, out))
        return out

    @property
    def time(self) -> float:
        return lib().gals_time(self._h)

    def state_planes(self):
        ptrs = (ctypes.c_void_p * self.nplanes)()
        pitch = ctypes.c_int64()
        _check(lib().gals_state_planes(self._h, ptrs, self.nplanes, ctypes.byref(pitch)), self._h)
        return [p for p in ptrs], pitch.value


def version() -> str:
    return lib().gals_version().decode()


def _bcheck(status: int, handle=None):
    if status != OK:
        msg = lib().gals_batch_last_error(handle)
        raise GalsError(status, msg.decode() if msg else "")


class Batch:
    """Independent 2D problems advanced together (gals_batch_* of gals.h).
    ``sizes``: list of (nx, ny); every problem lives on [0,1]^2 unless lo/hi given."""

    def __init__(self, sizes, lo=None, hi=None, layout: str = "full", stream=None):
        count = len(sizes)
        descs = (GridDesc * count)()
        for p, n in enumerate(sizes):
            d = descs[p]
            d.dim = 2
            for i in range(2):
                d.n[i] = int(n[i])
                d.lo[i] = 0.0 if lo is None else float(lo[p][i])
                d.hi[i] = 1.0 if hi is None else float(hi[p][i])
            d.n[2] = 1
            d.layout = LAYOUT_FULL if layout == "full" else LAYOUT_COMPACT
            if stream is not None and p == 0:
                d.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        h = ctypes.c_void_p()
        _bcheck(lib().gals_create_batch(descs, count, ctypes.byref(h)))
        self._h = h
        self.sizes = [tuple(int(v) for v in n) for n in sizes]
        self.count = count

    def close(self):
        if getattr(self, "_h", None):
            lib().gals_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nodes(self) -> int:
        return lib().gals_batch_nodes(self._h)

    def set_state(self, index, state, t0=0.0, recon=False):
        st = np.ascontiguousarray(state, dtype=np.float32)
        nf = st.shape[0]
        ptrs = (ctypes.c_void_p * nf)(*[st[p].ctypes.data for p in range(nf)])
        _bcheck(lib().gals_batch_set_state(self._h, int(index), ptrs, nf, MEM_HOST, float(t0),
                                           SET_RECON_CROSS if recon else 0), self._h)

    def _vels(self, vels, dts):
        assert len(vels) == self.count and len(dts) == self.count
        descs = (VelocityDesc * self.count)()
        keep = []
        for p, v in enumerate(vels):
            d = v.desc()
            keep.append(d)
            descs[p] = d
        dt = (ctypes.c_double * self.count)(*[float(x) for x in dts])
        return descs, dt, keep

    def step(self, vels, dts, nsteps=1):
        descs, dt, keep = self._vels(vels, dts)
        _bcheck(lib().gals_batch_step(self._h, descs, dt, int(nsteps)), self._h)

    def autotune(self, vels, dts, trial_steps=3):
        descs, dt, keep = self._vels(vels, dts)
        t = BatchTuning()
        _bcheck(lib().gals_batch_autotune(self._h, descs, dt, int(trial_steps), ctypes.byref(t)), self._h)
        return {"variant": t.variant, "blocks": t.blocks, "ms_per_step": t.ms_per_step,
                "loop": "persistent" if t.loop == 1 else "launches"}

    def set_tuning(self, variant, blocks, loop="launches"):
        t = BatchTuning(int(variant), int(blocks), 0.0, {"launches": 0, "persistent": 1}[loop])
        _bcheck(lib().gals_batch_set_tuning(self._h, ctypes.byref(t)), self._h)

    def read_state(self, index, nfields=4):
        nx, ny = self.sizes[index]
        out = np.empty((nfields, ny, nx), dtype=np.float32)
        ptrs = (ctypes.c_void_p * nfields)(*[out[p].ctypes.data for p in range(nfields)])
        _bcheck(lib().gals_batch_read_state(self._h, int(index), ptrs, nfields, MEM_HOST), self._h)
        return out

    def synchronize(self):
        _bcheck(lib().gals_batch_synchronize(self._h), self._h)


def _scheck(status: int, handle=None):
    if status != OK:
        msg = lib().gals_surrogate_last_error(handle)
        raise GalsError(status, msg.decode() if msg else "")


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Surrogate:
    """The learned flow map of the backward trace (gals_surrogate_* of gals.h)."""

    def __init__(self, seed: int = 1, stream=None):
        d = MlpDesc()
        d.seed = int(seed)
        if stream is not None:
            d.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        h = ctypes.c_void_p()
        _scheck(lib().gals_surrogate_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().gals_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, vel: Velocity, dt, h, steps=2000, batch=16384, lr=1e-3, lr_min=1e-5,
              substeps=32, seed=9053409):
        o = TrainOpts(int(steps), int(batch), float(lr), float(lr_min), int(substeps), int(seed))
        r = TrainReport()
        d = vel.desc()
        _scheck(lib().gals_surrogate_train(self._h, ctypes.byref(d), float(dt), float(h), ctypes.byref(o),
                                           ctypes.byref(r)), self._h)
        return {"initial_loss": r.initial_loss, "final_loss": r.final_loss, "seconds": r.seconds,
                "steps": r.steps}

    def set_check(self, tol_x=0.05, tol_J=0.05, samples=4):
        _scheck(lib().gals_surrogate_set_check(self._h, float(tol_x), float(tol_J), int(samples)), self._h)

    def stats(self, reset=False):
        t = ctypes.c_int64()
        f = ctypes.c_int64()
        _scheck(lib().gals_surrogate_stats(self._h, ctypes.byref(t), ctypes.byref(f), int(reset)), self._h)
        return t.value, f.value

    def get_params(self):
        p = np.empty(MLP_PARAMS, dtype=np.float32)
        sc = np.empty(6, dtype=np.float32)
        _scheck(lib().gals_surrogate_get_params(self._h, _fp(p), _fp(sc)), self._h)
        return p, sc

    def set_params(self, params, scales):
        p = np.ascontiguousarray(params, dtype=np.float32)
        sc = np.ascontiguousarray(scales, dtype=np.float32)
        assert p.size == MLP_PARAMS and sc.size == 6
        _scheck(lib().gals_surrogate_set_params(self._h, _fp(p), _fp(sc)), self._h)

    def bind(self, vel: Velocity, dt, h):
        d = vel.desc()
        _scheck(lib().gals_surrogate_bind(self._h, ctypes.byref(d), float(dt), float(h)), self._h)

    def forward(self, inputs):
        X = np.ascontiguousarray(inputs, dtype=np.float32).reshape(-1, 3)
        Y = np.empty((X.shape[0], 6), dtype=np.float32)
        _scheck(lib().gals_surrogate_forward(self._h, _fp(X), X.shape[0], _fp(Y)), self._h)
        return Y

    def save(self, path):
        _scheck(lib().gals_surrogate_save(self._h, os.fsencode(path)), self._h)

    def load(self, path):
        _scheck(lib().gals_surrogate_load(self._h, os.fsencode(path)), self._h)

    def forward_device(self, inputs_ptr: int, n: int, outputs_ptr: int):
        """Device-memory forward pass (n x 3 floats in, n x 6 out), enqueued on the
        surrogate's stream; the pointers are raw device addresses (e.g. tensor.data_ptr())."""
        _scheck(lib().gals_surrogate_forward_device(self._h, ctypes.c_void_p(inputs_ptr), int(n),
                                                    ctypes.c_void_p(outputs_ptr)), self._h)

    def gradient(self, inputs, targets):
        X = np.ascontiguousarray(inputs, dtype=np.float32).reshape(-1, 3)
        T = np.ascontiguousarray(targets, dtype=np.float32).reshape(-1, 6)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _scheck(lib().gals_surrogate_gradient(self._h, _fp(X), _fp(T), X.shape[0], _fp(g),
                                              ctypes.byref(loss)), self._h)
        return loss.value, g

    def targets(self, vel: Velocity, dt, h, points, substeps=32):
        P = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
        T = np.empty((P.shape[0], 6), dtype=np.float32)
        d = vel.desc()
        _scheck(lib().gals_surrogate_targets(self._h, ctypes.byref(d), float(dt), float(h), int(substeps),
                                             _fp(P), P.shape[0], _fp(T)), self._h)
        return T
