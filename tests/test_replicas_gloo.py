"""The multi-GPU host logic of bench.py: every rank times its own k-point shard and the reported time is
the maximum over ranks (exercised with two gloo ranks on the CPU); the ranks' k-point shards partition
one k-point set."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == [2.0, 10.0] and out[1] == [2.0, 10.0]


def test_max_over_ranks_without_process_group():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu") == [3.0, 4.0]


def test_rank_systems_partition_one_k_point_set():
    """Under torchrun each rank holds its own shifted copy of the base k-points with the weights divided by
    the number of ranks: the ranks' k-points are distinct and their weights sum to one."""
    import numpy as np
    import bench
    from paper_1711_08935_gb300 import synth
    base = synth.oxide_system(n=24, nk=2)
    for ws in (1, 2, 4, 8):
        parts = [bench.rank_system(base, r, ws) for r in range(ws)]
        k = np.concatenate([np.asarray(p.kpts) for p in parts])
        w = np.concatenate([np.asarray(p.wk) for p in parts])
        assert k.shape == (ws * base.nk, 3)
        assert abs(w.sum() - 1.0) < 1e-12
        d = np.linalg.norm(k[:, None, :] - k[None, :, :], axis=-1) + np.eye(len(k))
        assert d.min() > 1e-6
    assert bench.rank_system(base, 0, 1) is base
