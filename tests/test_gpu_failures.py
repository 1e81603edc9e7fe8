"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the checked build's test hook makes the step
  kernel's wait for its staged tile short and skips the copy that would complete it (an
  mbarrier that nothing arms).  The kernel records the timeout in the grid's error word
  and returns; the next synchronising call returns GALS_ERR_TIMEOUT, the context stays
  usable, and a fresh grid steps to the normal build's result bit for bit.  The checked
  library runs in a child process (GALS_LIB).
* A device allocation that fails: with the device's memory taken by the caller,
  gals_create_grid and gals_create_batch return GALS_ERR_NOMEM, and once memory is back a
  grid steps to the same result as before (the failed call leaves no error behind)."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0905_3409_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

N = (100, 14)  # one tile column of 128 and one tile row of 14 nodes: one block per step


def _state():
    return inputs.circle_sdf(N, center=(0.45, 0.55), r=0.3).astype(np.float32)


def _step_fresh(G):
    g = G.Grid(N)
    g.set_state(_state(), t0=0.2, recon=True)
    g.step(G.Velocity("vortex2d", T=8.0), 0.9 / (N[0] - 1), 1)
    out = g.read_state()
    g.close()
    return out


def child(dst):
    """Runs with the checked library: the timeout, then a fresh grid without the hook."""
    from paper_0905_3409_gb300 import gals as G
    assert G.LIB_PATH.endswith("libgals_checked.so"), G.LIB_PATH
    L = G.lib()
    assert L.gals_checked_wait_test(0, 1) == G.ERR_ARG
    assert L.gals_checked_wait_test(2048, 1) == G.OK
    g = G.Grid(N)
    g.set_state(_state(), t0=0.2, recon=True)
    g.step(G.Velocity("vortex2d", T=8.0), 0.9 / (N[0] - 1), 1)
    try:
        g.synchronize()
        status, msg = G.OK, ""
    except G.GalsError as e:
        status, msg = e.status, str(e)
    g.synchronize()  # the error word was cleared: the grid answers again
    g.close()
    assert L.gals_checked_wait_test(1 << 24, 0) == G.OK
    after = _step_fresh(G)
    np.savez(dst, status=np.array(status), msg=np.array(msg), after=after)


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_0905_3409_gb300 import gals
    return gals


def test_staged_tile_wait_runs_out_and_returns_timeout(G, tmp_path):
    from paper_0905_3409_gb300 import build
    checked = build.build_checked()
    dst = str(tmp_path / "timeout.npz")
    env = dict(os.environ, GALS_LIB=checked)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), dst], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = np.load(dst)
    assert int(got["status"]) == G.ERR_TIMEOUT, str(got["msg"])
    assert "bounded device wait" in str(got["msg"])
    assert np.array_equal(got["after"], _step_fresh(G))
    # the normal build has no hook and says so
    assert G.lib().gals_checked_wait_test(2048, 1) == G.ERR_UNSUPPORTED


def test_failed_allocation_returns_nomem_and_leaves_library_usable(G):
    import torch
    before = _step_fresh(G)
    free, _ = torch.cuda.mem_get_info()
    hold = torch.empty(max(free - (2 << 30), 0), dtype=torch.uint8, device="cuda")
    try:
        # 2 buffers x 4 planes x 20000^2 floats = 12.8 GB, far more than the 2 GB left
        with pytest.raises(G.GalsError) as ei:
            G.Grid((20000, 20000))
        assert ei.value.status == G.ERR_NOMEM
        with pytest.raises(G.GalsError) as eb:
            G.Batch([(16000, 16000), (64, 64)])
        assert eb.value.status == G.ERR_NOMEM
    finally:
        del hold
        torch.cuda.empty_cache()
    assert np.array_equal(_step_fresh(G), before)


if __name__ == "__main__":
    child(sys.argv[1])
