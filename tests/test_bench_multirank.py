"""The N > 1 host logic of bench.py on CPU: two gloo ranks share one generated graph
(rank 0 writes it, rank 1 maps it) and combine their figures (max of times, sum of edge
counts), as the torchrun launch does with one rank per GPU.  Whether the graph is shared
is rank 0's decision, so ranks that see different free space still take the same path."""
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


def _rank_main(rank, world, port, out_dir, need_bytes=None, free_bytes=None, local_world=None):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_env()
    assert (w, r, loc) == (world, rank, rank)
    free = None if free_bytes is None else free_bytes[rank]
    g, _ = bench.share_graph("pp1000", world, rank, dist.barrier, need_bytes=need_bytes,
                             free_bytes=free, local_world=local_world)
    np.save(os.path.join(out_dir, f"mapped{rank}.npy"),
            np.array([isinstance(g.indices, np.memmap)]))
    times, counts = bench.aggregate_over_ranks([1.0 + rank, 10.0 * (rank + 1)],
                                               [100.0, 7.0 + rank], world,
                                               torch.device("cpu"))
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), off=np.asarray(g.offsets),
             idx=np.asarray(g.indices), times=np.array(times), counts=np.array(counts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
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


@pytest.mark.timeout(300)
@pytest.mark.parametrize("free_bytes,local_world,shared", [
    ((1 << 62, 0), None, True),    # rank 1 sees no room: rank 0's decision (share) holds
    ((0, 1 << 62), None, False),   # rank 0 sees no room: nobody shares, nobody waits
    ((1 << 62, 1 << 62), 1, False),  # ranks on different nodes never share a file
])
def test_ranks_follow_rank0_decision(tmp_path, free_bytes, local_world, shared):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), 1 << 20, free_bytes,
                               local_world), nprocs=world, join=True)
    ref = bench.make_graph("pp1000")
    for rank in range(world):
        z = np.load(tmp_path / f"rank{rank}.npz")
        assert np.array_equal(z["off"], ref.offsets) and np.array_equal(z["idx"], ref.indices)
    # rank 1 maps rank 0's file exactly when the graph is shared
    assert bool(np.load(tmp_path / "mapped1.npy")[0]) == shared
