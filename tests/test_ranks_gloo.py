"""The N > 1 path of bench.py (replicas only): barrier and max/sum of the
per-rank results over two gloo ranks on CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = bench.Ranks(world, "cpu")
    r.barrier()
    t = 10.0 + rank            # per-rank time
    nli = 100 * (rank + 1)     # per-rank NCG iterations
    q.put((rank, r.max(t), r.sum(nli)))
    r.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, nsum in out:
        assert tmax == 11.0
        assert nsum == 300.0


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5 and r.sum(7) == 7
