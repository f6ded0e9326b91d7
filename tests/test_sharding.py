"""Origin sharding across ranks (world size 2, gloo on CPU): each rank computes
its origin range with the oracle and the merge reproduces the whole problem.
The same merge is used by multi-GPU runs of the CUDA library."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2106_13706_gb300 import sharding
from paper_2106_13706_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, T = wl.random_pair(11, 130, 170, 3, kind="int", dtype=np.float64)
        a, b = sharding.shard_range(300, world, rank)
        part = orc.ddks(P, T, origins=(a, b))
        merged = sharding.all_merge(part)
        if rank == 0:
            q.put(merged)
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_exactly():
    for n in (1, 2, 7, 300, 40001):
        for w in (1, 2, 3, 8):
            rs = [sharding.shard_range(n, w, r) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_merge_picks_lowest_origin_on_ties():
    parts = [dict(num_max=5, denom=9, argmax_origin=7, argmax_orthant=1),
             dict(num_max=5, denom=9, argmax_origin=3, argmax_orthant=2),
             dict(num_max=4, denom=9, argmax_origin=0, argmax_orthant=0),
             dict(num_max=0, denom=9, argmax_origin=-1, argmax_orthant=0)]
    m = sharding.merge_results(parts)
    assert (m["num_max"], m["argmax_origin"], m["argmax_orthant"]) == (5, 3, 2)


def test_two_rank_gloo_merge_equals_whole():
    from oracle import oracle as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    P, T = wl.random_pair(11, 130, 170, 3, kind="int", dtype=np.float64)
    whole = orc.ddks(P, T)
    assert (merged["num_max"], merged["argmax_origin"], merged["argmax_orthant"]) == \
        (whole["num_max"], whole["argmax_origin"], whole["argmax_orthant"])


def _perm_rank_main(rank, world, port, q):
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, T = wl.random_pair(12, 40, 50, 2, kind="normal", dtype=np.float64)
        B = 23
        a, b = sharding.shard_range(B, world, rank)
        # this rank's relabellings, each drawn from (seed, b) alone
        ref = orc.permutation_test(P, T, B, 99)
        mine = ref["perm_num_max"][a:b]
        count = int((mine >= ref["num_obs"]).sum())
        p = sharding.all_merge_perm(count, B)
        if rank == 0:
            q.put(p)
    finally:
        dist.destroy_process_group()


def test_perm_count_merge():
    assert sharding.merge_perm_counts([3, 4], 99) == 8 / 100
    assert sharding.merge_perm_counts([], 0) == 1.0
    with pytest.raises(ValueError):
        sharding.merge_perm_counts([-1], 5)


def test_two_rank_gloo_permutation_shards_equal_whole():
    from oracle import oracle as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_perm_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    p_merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    P, T = wl.random_pair(12, 40, 50, 2, kind="normal", dtype=np.float64)
    assert p_merged == orc.permutation_test(P, T, 23, 99)["p_value"]
