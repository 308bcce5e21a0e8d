"""The N > 1 host logic of bench.py on CPU: two gloo ranks share one generated graph
(rank 0 writes it, rank 1 maps it) and combine their figures (max of times, sum of edge
counts), as the torchrun launch does with one rank per GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, need_bytes=None):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_env()
    assert (w, r, loc) == (world, rank, rank)
    g, _ = bench.share_graph("pp1000", world, rank, dist.barrier, need_bytes=need_bytes)
    times, counts = bench.aggregate_over_ranks([1.0 + rank, 10.0 * (rank + 1)],
                                               [100.0, 7.0 + rank], world,
                                               torch.device("cpu"))
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), off=np.asarray(g.offsets),
             idx=np.asarray(g.indices), times=np.array(times), counts=np.array(counts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("need_bytes", [None, 1 << 62])  # shared file / one copy per rank
def test_two_gloo_ranks_share_the_graph_and_combine(tmp_path, need_bytes):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), need_bytes), nprocs=world,
             join=True)
    ref = bench.make_graph("pp1000")
    for rank in range(world):
        z = np.load(tmp_path / f"rank{rank}.npz")
        assert np.array_equal(z["off"], ref.offsets) and np.array_equal(z["idx"], ref.indices)
        assert z["times"].tolist() == [2.0, 20.0]          # max over ranks
        assert z["counts"].tolist() == [200.0, 15.0]       # sum over ranks


def test_single_rank_aggregation_is_the_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_over_ranks([3.5], [7], 1, None) == ([3.5], [7.0])
