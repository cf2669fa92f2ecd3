"""Multi-rank host logic of bench.py on the CPU: world-size-2 gloo process
group, ranks with different per-rank times and seeds.  The job time is the
max over ranks on every rank, the whole-job value counts the units of all
ranks over that time, and each rank gets its own box seed (weak scaling with
independent boxes, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, lr = bench.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = 10.0 + 5.0 * r  # rank 1 is the slow one
    ms_max = bench.reduce_max(ms, dist, "cpu")
    out.put((r, w, lr, bench.rank_seed(r), ms_max, bench.job_value(w, 1000, 4, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_timing_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert res[0][3] != res[1][3]  # independent boxes per rank
    assert all(r[4] == pytest.approx(15.0) for r in res)  # slowest rank's time everywhere
    assert res[0][5] == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (0, 1, 0)
    assert bench.reduce_max(3.0, None, "cpu") == 3.0
    assert bench.job_value(1, 10, 2, 1.0) == pytest.approx(2e4)
