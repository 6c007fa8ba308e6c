"""The benchmark's multi-GPU path runs independent replicas (the apply does not shard): the job
value is the units of all ranks over the slowest rank's time.  Checked here with two gloo ranks
on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [2.0, 5.0][rank]  # rank 1 is the slowest
    value, ms = bench.replica_throughput(ms_local, 1_000_000_000, world, dist, device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            value, ms = out[r]
            assert ms == 5.0
            assert abs(value - 2 * 1e9 / 5e-3 / 1e9) < 1e-9
