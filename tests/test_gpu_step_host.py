"""gals_step_host: one step from a host state to a host state with the copies overlapped
with the step in bands of rows (2D) or z-levels (3D).  It must give the result of
gals_set_state + gals_step + gals_read_state bit for bit, leave the grid holding the new
state at t0 + dt, and refuse what it does not serve."""
import math

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


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float32).pin_memory().numpy()


def _state(G, n, dim):
    """A state with reconstructed mixed derivatives, as a host array of all planes."""
    g = G.Grid(n)
    st = inputs.circle_sdf(n, center=(0.45, 0.55), r=0.3) if dim == 2 else \
        inputs.sphere_sdf(n, center=(0.45, 0.5, 0.5), r=0.3)
    g.set_state(st.astype(np.float32), recon=True)
    full = g.read_state()
    g.close()
    return full


CASES = [
    # (n, velocity kwargs, dt in cells): several bands each, ragged last band
    ((150, 200), dict(kind="vortex2d", T=8.0), 0.8),
    ((129, 61), dict(kind="rotation", omega=2 * math.pi, center=(0.5, 0.5, 0.0)), 2.5),
    ((24, 20, 37), dict(kind="deform3d", T=3.0), 0.4),
    # feet six cells away: a band's step needs rows beyond the next band's first rows
    ((70, 64), dict(kind="rotation", omega=2 * math.pi, center=(0.5, 0.5, 0.0)), 6.0),
]


@pytest.mark.parametrize("n,vel,cells", CASES)
def test_step_host_equals_set_step_read(G, n, vel, cells):
    dim = len(n)
    st = _state(G, n, dim)
    h = 1.0 / (max(n) - 1)
    dt, t0 = cells * h, 0.3
    v = G.Velocity(**vel)
    a = G.Grid(n)
    pin_in = _pinned(st.shape)
    pin_in[...] = st
    pin_out = _pinned(st.shape)
    a.step_host(v, dt, t0, pin_in, pin_out)
    b = G.Grid(n)
    b.set_state(st, t0=t0)           # all planes: mixed derivatives as given
    b.step(v, dt, 1)
    ref = b.read_state()
    assert np.array_equal(pin_out, ref)
    assert a.time == pytest.approx(t0 + dt, abs=1e-15)
    # the grid holds the new state: later steps continue from it
    a.step(v, dt, 2)
    b.step(v, dt, 2)
    assert np.array_equal(a.read_state(), b.read_state())
    a.close()
    b.close()


def test_step_host_in_place_and_pageable(G):
    n = (140, 90)
    st = _state(G, n, 2)
    v = G.Velocity("vortex2d", T=8.0)
    dt = 0.7 / 139
    b = G.Grid(n)
    b.set_state(st, t0=0.0)
    b.step(v, dt, 1)
    ref = b.read_state()
    a = G.Grid(n)
    buf = st.copy()                  # pageable, and in == out
    a.step_host(v, dt, 0.0, buf, buf)
    assert np.array_equal(buf, ref)


def test_step_host_refuses_what_it_does_not_serve(G):
    n = (40, 30)
    st = _state(G, n, 2)
    v = G.Velocity("vortex2d", T=8.0)
    c = G.Grid(n, layout="compact")
    with pytest.raises(G.GalsError) as e:
        c.step_host(v, 0.01, 0.0, st)
    assert e.value.status == G.ERR_UNSUPPORTED
    g = G.Grid(n)
    for dt in (0.0, -1.0, float("nan")):
        with pytest.raises(G.GalsError) as e:
            g.step_host(v, dt, 0.0, st)
        assert e.value.status == G.ERR_ARG
    with pytest.raises(G.GalsError) as e:
        g.step_host(G.Velocity("deform3d", T=3.0), 0.01, 0.0, st)
    assert e.value.status == G.ERR_UNSUPPORTED


@pytest.mark.parametrize("n,vel,cells", CASES)
def test_async_host_loop_equals_synchronous(G, n, vel, cells):
    """gals_step_host_async as a host-side time loop (each call's output array is the next
    call's input, the calls queued back to back, one wait at the end) gives the states of
    the same loop of synchronous calls bit for bit, and so does a chain into a separate
    output array followed by a device step and a read (the other calls wait for the
    pending copies)."""
    dim = len(n)
    st = _state(G, n, dim)
    h = 1.0 / (max(n) - 1)
    dt, t0 = cells * h, 0.1
    v = G.Velocity(**vel)
    nsteps = 4
    # synchronous reference loop
    a = G.Grid(n)
    ref = _pinned(st.shape)
    ref[:] = st
    for k in range(nsteps):
        a.step_host(v, dt, t0 + k * dt, ref, ref)
    # the same loop queued: one array is each call's input and output
    b = G.Grid(n)
    buf = _pinned(st.shape)
    buf[:] = st
    for k in range(nsteps):
        b.step_host(v, dt, t0 + k * dt, buf, buf, wait=False)
    b.synchronize()
    assert np.array_equal(buf, ref)
    assert np.array_equal(b.read_state(), a.read_state())
    assert b.time == pytest.approx(t0 + nsteps * dt, abs=1e-12)
    # queued calls from a fixed input into another array, then other calls on the grid
    c = G.Grid(n)
    pin_in, pin_out = _pinned(st.shape), _pinned(st.shape)
    pin_in[:] = st
    c.step_host(v, dt, t0, pin_in, pin_out, wait=False)
    c.step_host(v, dt, t0, pin_in, pin_out, wait=False)
    c.step(v, dt, 1)                        # waits for the pending copies
    after = c.read_state()
    d = G.Grid(n)
    d.set_state(st, t0=t0)
    d.step(v, dt, 2)
    assert np.array_equal(after, d.read_state())
    c.synchronize()
    one = G.Grid(n)
    one.set_state(st, t0=t0)
    one.step(v, dt, 1)
    assert np.array_equal(pin_out, one.read_state())
    for g in (a, b, c, d, one):
        g.close()
