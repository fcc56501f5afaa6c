"""Host logic of `bench.py --gpus N` (independent replicas, one rank per GPU):
the whole-job throughput is the bytes all ranks moved over the slowest rank's
time.  Two gloo ranks on CPU (127.0.0.1), no GPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    moved = [3.0e9, 5.0e9][rank]
    seconds = [0.5, 0.8][rank]
    out.put((rank, bench.replica_throughput(moved, seconds, world, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = (3.0e9 + 5.0e9) / 0.8 / 1e9
    assert abs(res[0] - want) < 1e-12 and abs(res[1] - want) < 1e-12


def test_replica_throughput_single():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(6.0e9, 2.0, 1) == 3.0
