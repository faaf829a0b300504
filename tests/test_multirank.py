"""The replica path of bench.py under several ranks (gloo on the CPU, world
size 2): per-rank seeds differ, and rank 0 gets the slowest rank's time and
the summed counts. No GPU: the ranks exchange only host tensors."""
import os
import socket
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 10.0 - rank]  # per-rank device and e2e seconds
    counts = [1000 * (rank + 1), 7 + rank, 3]
    t, n = bench.combine_ranks(times, counts, world, "cpu")
    out.put((rank, t, n, bench.replica_seed(rank)))
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_ranks_combine_max_time_and_summed_counts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, seed in res:
        assert t == [2.0, 10.0]            # slowest rank per figure
        assert n == [3000, 15, 6]          # summed over ranks
    assert res[0][3] != res[1][3]          # independent replicas


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks([1.5, 2.5], [4, 5], 1, "cpu") == ([1.5, 2.5], [4, 5])
