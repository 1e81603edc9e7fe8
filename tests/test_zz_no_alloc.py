"""gals_diagnostics_noalloc: the diagnostics of a state in caller memory without any
device allocation (for callers whose device memory is reserved up front, or that must
not let an allocation synchronise the device).  Called through the C ABI and checked
against gals_diagnostics on the same state, on two calls in a row (the shared scratch
keeps the previous call's contents, so the second call shows it is cleared), on states
in the library's layout and in a padded caller layout; the call leaves free device memory
unchanged and works with almost none left.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

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


def _noalloc(G, grid, ref, q):
    L = G.lib()
    planes, pitch = grid.state_planes()
    ref_ptr = ref.state_planes()[0][0] if ref is not None else None
    dim = grid.dim
    n = (ctypes.c_int * 3)(*(list(grid.n) + [1] * (3 - dim)))
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    plane_stride = planes[1] - planes[0]
    assert plane_stride % 4 == 0
    out = G.DiagOut()
    st = L.gals_diagnostics_noalloc(dim, n, lo, hi, planes[0], ref_ptr, pitch, plane_stride // 4, q,
                                    None, ctypes.byref(out))
    assert st == G.OK, L.gals_noalloc_last_error()
    return {f: getattr(out, f) for f, _ in G.DiagOut._fields_}


def _same(a, b):
    for key in ("samples", "n_negative", "n_symdiff", "nonfinite"):
        assert a[key] == b[key], key
    for key in ("measure_negative", "measure_symdiff", "emax_phi", "emax_psi"):
        assert a[key] == pytest.approx(b[key], rel=1e-12, abs=0.0), key
    # FP64 partial sums over another block partition: agreement to rounding
    assert a["l2_phi"] == pytest.approx(b["l2_phi"], rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_matches_diagnostics_twice(G, dim):
    if dim == 2:
        n = (160, 131)
        a_st = inputs.circle_sdf(n, r=0.2, center=(0.5, 0.5))
        b_st = inputs.circle_sdf(n, r=0.23, center=(0.52, 0.49))
    else:
        n = (40, 37, 33)
        a_st = inputs.sphere_sdf(n, r=0.25, center=(0.5, 0.5, 0.5))
        b_st = inputs.sphere_sdf(n, r=0.27, center=(0.52, 0.5, 0.48))
    a = G.Grid(n)
    a.set_state(a_st.astype(np.float32), recon=True)
    b = G.Grid(n)
    b.set_state(b_st.astype(np.float32), recon=True)
    q = 4
    ref = a.diagnostics(q=q, reference=b)
    first = _noalloc(G, a, b, q)
    second = _noalloc(G, a, b, q)
    _same(first, ref)
    _same(second, ref)
    # without a reference, and a state with a non-finite value
    assert _noalloc(G, a, None, 0)["nonfinite"] == 0
    bad = a_st.astype(np.float32)
    bad[1].flat[17] = np.inf
    a.set_state(bad)
    assert _noalloc(G, a, None, 0)["nonfinite"] == a.diagnostics(q=0)["nonfinite"] == 1


def test_noalloc_at_its_node_limit(G):
    """16384 x 16384 nodes, the most the fixed scratch serves (one FP64 partial per 16384
    nodes): the results of gals_diagnostics, with and without a reference state."""
    import torch
    N = 16384
    n = (N, N)
    h = 1.0 / (N - 1)
    grids = []
    for cx, cy, r in ((0.5, 0.75, 0.15), (0.51, 0.74, 0.16)):
        st = torch.empty((3, N, N), dtype=torch.float32, device="cuda")
        X = (torch.arange(N, device="cuda", dtype=torch.float64) * h).float()
        dx, dy = (X - cx)[None, :], (X - cy)[:, None]
        torch.add(dx * dx, dy * dy, out=st[0])
        st[0].sqrt_()
        torch.div(dx, st[0], out=st[1])
        torch.div(dy, st[0], out=st[2])
        st[0].sub_(r)
        g = G.Grid(n)
        g.set_state(st, recon=True)
        del st
        grids.append(g)
    torch.cuda.empty_cache()
    a, b = grids
    _same(_noalloc(G, a, b, 1), a.diagnostics(q=1, reference=b))
    _same(_noalloc(G, a, None, 2), a.diagnostics(q=2))
    a.close()
    b.close()


def test_noalloc_rejects_oversize_and_bad_args(G):
    L = G.lib()
    assert L.gals_noalloc_max_nodes() == 16384 * 16384
    n = (ctypes.c_int * 3)(4096, 4096, 17)
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    out = G.DiagOut()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check rejects first
    st = L.gals_diagnostics_noalloc(3, n, lo, hi, fake, None, 4096, 4096 * 4096 * 17, 0, None,
                                    ctypes.byref(out))
    assert st == G.ERR_ARG
    assert b"no-allocation" in L.gals_noalloc_last_error()
    n2 = (ctypes.c_int * 3)(16, 16, 1)
    st = L.gals_diagnostics_noalloc(2, n2, lo, hi, fake, None, 8, 256, 0, None, ctypes.byref(out))
    assert st == G.ERR_ARG  # row pitch smaller than the grid


def _padded_copy(torch, grid, row_pitch, plane_stride):
    """The grid's state in a caller buffer of another layout: rows of row_pitch floats,
    planes plane_stride floats apart, every padding float NaN."""
    st = torch.from_numpy(grid.read_state()).cuda()
    npl = st.shape[0]
    rows = int(np.prod(st.shape[1:-1]))
    n0 = st.shape[-1]
    buf = torch.full((npl * plane_stride,), float("nan"), dtype=torch.float32, device="cuda")
    for p in range(npl):
        view = buf[p * plane_stride:p * plane_stride + rows * row_pitch].view(rows, row_pitch)
        view[:, :n0] = st[p].reshape(rows, n0)
    return buf


def _noalloc_raw(G, dim, n, ptr, ref_ptr, pitch, stride, q):
    L = G.lib()
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - dim)))
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    out = G.DiagOut()
    st = L.gals_diagnostics_noalloc(dim, nn, lo, hi, ctypes.c_void_p(ptr),
                                    ctypes.c_void_p(ref_ptr) if ref_ptr else None, pitch, stride, q,
                                    None, ctypes.byref(out))
    assert st == G.OK, L.gals_noalloc_last_error()
    return {f: getattr(out, f) for f, _ in G.DiagOut._fields_}


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_caller_layout_with_padding(G, dim):
    """A state held by the caller in its own layout (wider rows, padded planes, NaN in
    every padding float): the results of gals_diagnostics on the grid, and no padding
    float is read (the non-finite count stays 0)."""
    import torch
    if dim == 2:
        n = (150, 97)
        a_st = inputs.circle_sdf(n, r=0.2, center=(0.5, 0.5))
        b_st = inputs.circle_sdf(n, r=0.22, center=(0.51, 0.5))
    else:
        n = (30, 27, 25)
        a_st = inputs.sphere_sdf(n, r=0.25, center=(0.5, 0.5, 0.5))
        b_st = inputs.sphere_sdf(n, r=0.26, center=(0.5, 0.49, 0.5))
    a = G.Grid(n)
    a.set_state(a_st.astype(np.float32), recon=True)
    b = G.Grid(n)
    b.set_state(b_st.astype(np.float32), recon=True)
    rows = int(np.prod(n[1:]))
    pitch = n[0] + 13
    stride = rows * pitch + 77
    A = _padded_copy(torch, a, pitch, stride)
    B = _padded_copy(torch, b, pitch, stride)
    torch.cuda.synchronize()
    for q in (0, 3):
        got = _noalloc_raw(G, dim, n, A.data_ptr(), B.data_ptr(), pitch, stride, q)
        _same(got, a.diagnostics(q=q, reference=b))
        assert got["nonfinite"] == 0


def test_noalloc_allocates_nothing(G):
    """Free device memory is the same before and after a call (after a first call, which
    may load the library's device code and its scratch), and the call still succeeds
    when the caller has taken all but 256 MB of the device's free memory."""
    import torch
    n = (300, 211)
    a = G.Grid(n)
    a.set_state(inputs.circle_sdf(n, r=0.2, center=(0.5, 0.5)).astype(np.float32), recon=True)
    b = G.Grid(n)
    b.set_state(inputs.circle_sdf(n, r=0.21, center=(0.5, 0.5)).astype(np.float32), recon=True)
    ref = a.diagnostics(q=4, reference=b)
    _same(_noalloc(G, a, b, 4), ref)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _same(_noalloc(G, a, b, 4), ref)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    hold = torch.empty(max(free1 - (256 << 20), 0), dtype=torch.uint8, device="cuda")
    try:
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] <= (300 << 20)
        _same(_noalloc(G, a, b, 4), ref)
        _same(_noalloc(G, a, b, 4), ref)
    finally:
        del hold
        torch.cuda.empty_cache()
    a.close()
    b.close()
