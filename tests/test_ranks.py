"""Multi-GPU layout on the CPU: two gloo ranks (world size 2) exercise the
cross-rank reduction of the job's rate (MAX of the times, SUM of the units)
and the disjoint per-rank batches; no GPU and no library call."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2510_26180_gb300.ranks import job_rate, rank_seed
    from synth import draw_xi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = [1000.0, 3000.0][rank]
        ms = [40.0, 50.0][rank]
        rate, ms_max, total = job_rate(units, ms)
        xi = draw_xi(4, 3, rank_seed(7, rank))
        gathered = [torch.zeros(12, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(xi.ravel().copy()))
        out.put((rank, rate, ms_max, total, [g.numpy() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_job_rate_and_draw_disjoint_batches():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max, total, xs in res:
        assert ms_max == 50.0 and total == 4000.0
        assert rate == pytest.approx(4000.0 / 0.05)
        assert not np.allclose(xs[0], xs[1])        # each rank its own batch


def test_single_process_keeps_the_local_rate():
    from paper_2510_26180_gb300.ranks import job_rate, rank_seed
    assert job_rate(500, 25.0) == (500 / 0.025, 25.0, 500.0)
    assert rank_seed(7, 0) == 7 and rank_seed(7, 3) == 3007
