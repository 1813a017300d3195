"""The multi-GPU form of the bench is replicas only: every rank steps its own
halo (seed 1 + rank) and the ranks share two scalars at the end, the slowest
rank's time and the total number of updates.  This runs that host logic on
two gloo ranks on the CPU (no GPU, no data-path collective)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, u = bench.reduce_over_ranks(10.0 + 3.0 * rank, 1000 * (rank + 1), "cpu")
        w, masks = bench._workload(seed_offset=rank, n=4096)
        q.put((rank, t, u, float(w["particles"].pos[0, 0]), int(masks.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_time_and_updates():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    res = sorted(q.get() for _ in range(2))
    # both ranks see the slowest time and the summed updates
    for rank, t, u, _, _ in res:
        assert t == 13.0 and u == 3000.0, (rank, t, u)
    # each rank steps a halo of its own
    assert res[0][3] != res[1][3]
    assert res[0][4] > 0 and res[1][4] > 0
