"""The N > 1 path of bench.py on CPU: two ranks in a gloo process group (the
launch torchrun makes, with 127.0.0.1 rendezvous). The block does not shard,
so every rank runs an independent replica; what the ranks share is the
job's time (the slowest rank's, an all-reduce MAX) and the whole-job rate
(all ranks' units over that time); the reference arm runs on rank 0 alone."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.env_rank()
        ms = 10.0 * (rank + 1)  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, device="cpu")
        rate = bench.job_rate(1000, w, ms_max * 1e-3)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            if rank != 0:  # the reference arm: ranks other than 0 return at once, printing nothing
                bench.run_reference(type("A", (), {"steps": 1, "warmup": 1, "gpus": w})(), rank, w)
        dist.barrier()
        q.put((rank, r, w, local, ms_max, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_slowest_time_and_the_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, r, w, local, ms_max, rate, printed in res:
        assert (r, w, local) == (rank, 2, rank)
        assert ms_max == 20.0                      # the slowest rank's time on every rank
        assert abs(rate - 1000 * 2 / 0.020) < 1e-9  # all ranks' units over it
        if rank == 1:
            assert printed == ""
