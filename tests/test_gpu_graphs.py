"""Graph replay of repeated calls (ddks_config.graphs): results stay bit-exact
against the oracle on every replay, follow new input values written at the
same addresses, survive scratch reallocation by other calls, and permutation
tests replayed with changing seeds match the same tests run kernel by kernel.
"""
import numpy as np
import pytest

import paper_2106_13706_gb300 as pkg
from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2106_13706_gb300 import build as b
    b.build()
    return t


def _dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _key(r):
    return (r["num_max"], r["denom"], r["argmax_origin"], r["argmax_orthant"])


def _okey(r):
    return (r["num_max"], r["denom"], r["argmax_origin"], r["argmax_orthant"])


@pytest.mark.parametrize("path,d,n", [(pkg.PATH_AUTO, 3, 300), (pkg.PATH_REGISTER, 4, 5000),
                                      (pkg.PATH_LANE, 5, 900), (pkg.PATH_WARP, 9, 700),
                                      (pkg.PATH_SORT, 12, 500)])
def test_replay_matches_oracle_and_follows_inputs(torch, path, d, n):
    P, T = wl.random_pair(41 + d, n, n + 17, d, kind="int", dtype=np.float32)
    ref = orc.ddks(P, T)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    with pkg.Context(device=0, path=path) as c:
        for _ in range(5):
            assert _key(c.distance(Pd, Td)) == _okey(ref)
        st = c.stats()
        assert st["graph_captures"] == 1 and st["graph_replays"] == 3
        # new values at the same device addresses: the replayed graph reads them
        P2, T2 = wl.random_pair(99 + d, n, n + 17, d, kind="normal", dtype=np.float32)
        Pd.copy_(_dev(torch, P2))
        Td.copy_(_dev(torch, T2))
        assert _key(c.distance(Pd, Td)) == _okey(orc.ddks(P2, T2))
        assert c.stats()["graph_replays"] == 4


def test_replay_after_scratch_reallocation(torch):
    P, T = wl.random_pair(5, 400, 380, 3, kind="int", dtype=np.float32)
    Pb, Tb = wl.random_pair(6, 6000, 6100, 3, kind="normal", dtype=np.float32)
    ref, refb = orc.ddks(P, T), orc.ddks(Pb, Tb)
    Pd, Td, Pbd, Tbd = _dev(torch, P), _dev(torch, T), _dev(torch, Pb), _dev(torch, Tb)
    with pkg.Context(device=0) as c:
        for _ in range(3):
            assert _key(c.distance(Pd, Td)) == _okey(ref)
        cap = c.stats()["graph_captures"]
        assert cap == 1
        # a larger problem grows (reallocates) the context's scratch
        assert _key(c.distance(Pbd, Tbd)) == _okey(refb)
        for _ in range(3):
            assert _key(c.distance(Pd, Td)) == _okey(ref)
        assert c.stats()["graph_captures"] == cap + 1  # the stale graph was captured again


def test_host_inputs_replay(torch):
    """Host inputs are staged into context scratch first, so calls with
    different host arrays of one shape share a graph."""
    with pkg.Context(device=0) as c:
        for s in range(5):
            P, T = wl.random_pair(200 + s, 777, 650, 4, kind="int", dtype=np.float64)
            assert _key(c.distance(P, T)) == _okey(orc.ddks(P, T))
        assert c.stats()["graph_replays"] == 3


def test_range_and_off_switch(torch):
    P, T = wl.random_pair(8, 900, 800, 3, kind="int", dtype=np.float32)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    N = 1700
    with pkg.Context(device=0, graphs=False) as c0, pkg.Context(device=0) as c1:
        for ob, oe in [(0, 500), (500, 1700), (0, 500), (500, 1700), (0, 500), (500, 1700)]:
            ref = orc.ddks(P, T, origins=(ob, oe))
            for c in (c0, c1):
                r = c.distance_range(Pd, Td, ob, oe)
                assert r["num_max"] == ref["num_max"]
        assert c0.stats()["graph_captures"] == 0 and c0.stats()["graph_replays"] == 0
        assert c1.stats()["graph_replays"] == 2
        assert N == 1700


def test_stage_timing_runs_kernel_by_kernel(torch):
    """Stage timing brackets each stage with events, so it turns replay off."""
    P, T = wl.random_pair(9, 3000, 3000, 2, kind="int", dtype=np.float32)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    ref = orc.ddks(P, T)
    with pkg.Context(device=0) as c:
        c.set_stage_timing(True)
        for _ in range(4):
            assert _key(c.distance(Pd, Td)) == _okey(ref)
            enc, cnt, red = c.stage_times()
            assert enc > 0 and cnt > 0 and red > 0
        assert c.stats()["graph_replays"] == 0
        c.set_stage_timing(False)
        for _ in range(3):
            assert _key(c.distance(Pd, Td)) == _okey(ref)
        assert c.stats()["graph_replays"] == 1


@pytest.mark.parametrize("d,n,B", [(3, 500, 96), (6, 300, 70)])
def test_perm_replay_with_changing_seeds(torch, d, n, B):
    P, T = wl.random_pair(70 + d, n, n - 20, d, kind="normal", dtype=np.float32)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    with pkg.Context(device=0, graphs=False) as c0, pkg.Context(device=0) as c1:
        for seed in (11, 12, 13, 14, 15):
            a = c0.permutation_test(Pd, Td, B, seed)
            b = c1.permutation_test(Pd, Td, B, seed)
            assert a["p_value"] == b["p_value"]
            assert np.array_equal(a["perm_num_max"], b["perm_num_max"])
            assert _key(a["observed"]) == _key(b["observed"])
        assert c1.stats()["graph_replays"] == 3
        o = orc.permutation_test(P, T, B, 15)
        assert np.array_equal(b["perm_num_max"], o["perm_num_max"])
        assert b["p_value"] == o["p_value"]


def test_batch_replay(torch):
    probs = [wl.random_pair(300 + i, 50 + 37 * i, 60 + 23 * i, 2 + i % 7, kind="int", dtype=np.float32)
             for i in range(12)]
    dev = [(_dev(torch, P), _dev(torch, T)) for P, T in probs]
    refs = [orc.ddks(P, T) for P, T in probs]
    with pkg.Context(device=0) as c:
        for _ in range(4):
            got = c.batch_distance(dev)
            assert [_key(g) for g in got] == [_okey(r) for r in refs]
        assert c.stats()["graph_replays"] == 2
