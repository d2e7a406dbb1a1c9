"""The multi-GPU path of bench.py is independent replicas (the solve does
not shard): the per-step time is the MAX over ranks and the whole-job time
per realization divides it by the number of ranks.  Checked with two gloo
ranks on the CPU."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    t_max, t_job = bench.whole_job(10.0 * (rank + 1), world)
    q.put((rank, t_max, t_job))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_timing_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, t_job in got:
        assert t_max == 20.0  # the slower rank sets the step time
        assert t_job == 10.0  # two realizations per step


def test_whole_job_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.whole_job(7.5, 1) == (7.5, 7.5)
