"""The multi-GPU path of the benchmark (independent replicas, one per rank) on CPU: two
gloo ranks each advance their own replica with the FP64 oracle, then the timing protocol
(barrier, maximum of the per-rank times, whole-job throughput) runs over the process
group exactly as it does over NCCL on GPUs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import oracle
    from paper_0905_3409_gb300 import inputs, replicas
    R = replicas.init("gloo")
    n = (17, 17)
    g = oracle.grid(n)
    st = oracle.recon_cross(g, inputs.circle_sdf(n))
    v = oracle.velocity("vortex2d", T=8.0)
    replicas.barrier(R)
    for k in range(2):
        st = oracle.step(g, v, st, k / 16.0, 1.0 / 16.0)
    # per-rank "time": deliberately different so that the maximum is visible
    t_local = 0.5 + rank
    t_max = replicas.max_over_ranks(R, t_local)
    value = replicas.throughput(np.prod(n) * 2, R.world, t_max)
    replicas.barrier(R)
    q.put((rank, R.world, R.leader, t_max, value, float(st[0].sum())))
    replicas.finish(R)


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == world for r in res)
    assert res[0][2] and not res[1][2]                       # rank 0 alone reports
    assert all(r[3] == 1.5 for r in res)                      # max over ranks, on every rank
    assert all(r[4] == pytest.approx(17 * 17 * 2 * world / 1.5) for r in res)
    assert res[0][5] == res[1][5]                             # identical independent replicas


def test_single_process_defaults(monkeypatch):
    from paper_0905_3409_gb300 import replicas
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    R = replicas.init("gloo")
    assert (R.rank, R.world, R.local, R.dist) == (0, 1, 0, None) and R.leader
    assert replicas.max_over_ranks(R, 2.5) == 2.5
    assert replicas.throughput(100, 1, 0.5) == 200
