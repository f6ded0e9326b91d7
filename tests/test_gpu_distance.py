"""Parity of the CUDA exact-ddKS path with the CPU oracle, through the C ABI.

The bar is bit-exact: the integer numerator max|cP*NT - cT*NP|, the
denominator, the arg-max origin and orthant.  Sizes span several shared-memory
tiles with ragged tails; every kernel path is forced in turn.
"""
import json
import os

import numpy as np
import pytest

import paper_2106_13706_gb300 as pkg
from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2106_13706_gb300 import build as b
    b.build()
    return t


def _ctx(path=pkg.PATH_AUTO):
    return pkg.Context(device=0, path=path)


def _dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _same(got, ref):
    assert (got["num_max"], got["denom"]) == (ref["num_max"], ref["denom"])
    assert got["argmax_origin"] == ref["argmax_origin"]
    assert got["argmax_orthant"] == ref["argmax_orthant"]


PATHS = [pkg.PATH_LANE, pkg.PATH_WARP, pkg.PATH_SORT]


def _paths_for(d, N):
    out = []
    if 2 <= d <= 4:
        out.append(pkg.PATH_REGISTER)
    if d <= 8:
        out.append(pkg.PATH_LANE)
    if d <= 13:
        out.append(pkg.PATH_WARP)
    if N <= 32768:
        out.append(pkg.PATH_SORT)
    return out


def test_hand_cases(torch):
    with _ctx() as c:
        for case in json.load(open(GOLDEN))["cases"]:
            P = np.array(case["P"], dtype=np.float64)
            T = np.array(case["T"], dtype=np.float64)
            r = c.distance(_dev(torch, P), _dev(torch, T))
            assert (r["num_max"], r["denom"]) == (case["num_max"], case["denom"]), case["name"]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_small_random_all_paths(torch, d):
    shapes = [(1, 1), (3, 2), (37, 61), (1000, 1100), (1500, 700)]
    for si, (n_p, n_t) in enumerate(shapes):
        for kind in ("normal", "int"):
            for dt in (np.float32, np.float64):
                P, T = wl.random_pair(1000 * d + 10 * si + (kind == "int"), n_p, n_t, d, kind=kind,
                                      dtype=dt)
                ref = orc.ddks(P, T)
                for path in _paths_for(d, n_p + n_t):
                    with _ctx(path) as c:
                        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


@pytest.mark.parametrize("d", [9, 10, 11, 12, 13])
def test_mid_d_warp_and_sort(torch, d):
    for n_p, n_t in [(5, 9), (700, 513)]:
        P, T = wl.random_pair(d, n_p, n_t, d, kind="normal", dtype=np.float32)
        ref = orc.ddks(P, T)
        for path in (pkg.PATH_WARP, pkg.PATH_SORT):
            with _ctx(path) as c:
                _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)
        with _ctx() as c:
            _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


@pytest.mark.parametrize("d", [14, 17, 22, 30])
def test_high_d_sort(torch, d):
    P, T = wl.random_pair(d, 300, 257, d, kind="int", dtype=np.float64)
    ref = orc.ddks(P, T)
    with _ctx() as c:
        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


def test_degenerate_inputs(torch):
    with _ctx() as c:
        for d in (1, 3, 9, 15):
            P, T = wl.random_pair(1, 40, 33, d, kind="const")
            r = c.distance(_dev(torch, P), _dev(torch, T))
            assert r["num_max"] == 0 and r["argmax_origin"] == 0 and r["argmax_orthant"] == 0
            P, T = wl.random_pair(2, 40, 33, d, kind="shifted")
            r = c.distance(_dev(torch, P), _dev(torch, T))
            assert r["num_max"] == r["denom"] == 40 * 33
            # identical samples
            r = c.distance(_dev(torch, P), _dev(torch, P.copy()))
            assert r["num_max"] == 0


def test_special_values(torch):
    P = np.array([[0.0, -np.inf], [1.0, 2.0], [-0.0, 5.0]])
    T = np.array([[-0.0, np.inf], [1.0, -1.0], [np.inf, 0.0], [0.0, 0.0]])
    ref = orc.ddks(P, T)
    with _ctx() as c:
        for dt in (np.float32, np.float64):
            _same(c.distance(_dev(torch, P.astype(dt)), _dev(torch, T.astype(dt))), ref)
        bad = P.copy()
        bad[1, 1] = np.nan
        with pytest.raises(pkg.DdksError) as e:
            c.distance(_dev(torch, bad), _dev(torch, T))
        assert e.value.code == -2
        # the context stays usable after an error
        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


def test_argument_errors(torch):
    with _ctx() as c:
        P = np.zeros((4, 31), dtype=np.float32)
        with pytest.raises(pkg.DdksError) as e:
            c.distance(_dev(torch, P), _dev(torch, P))
        assert e.value.code == -1
        with pytest.raises(pkg.DdksError) as e:
            c.distance(_dev(torch, np.zeros((0, 3), np.float32)), _dev(torch, np.zeros((2, 3), np.float32)))
        assert e.value.code == -1


def test_host_and_device_inputs_agree(torch):
    P, T = wl.gaussian_pair(seed=5, n_p=3000, n_t=2500, d=4)
    ref = orc.ddks(P, T)
    with _ctx() as c:
        _same(c.distance(P, T), ref)                                   # pageable host
        _same(c.distance(torch.from_numpy(P).pin_memory(), torch.from_numpy(T).pin_memory()), ref)
        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)         # device


def test_origin_range_shards(torch):
    P, T = wl.random_pair(8, 900, 1300, 3, kind="int", dtype=np.float32)
    ref = orc.ddks(P, T, per_origin=True)
    N = 2200
    cuts = [0, 1, 333, 1024, 2199, N]
    with _ctx() as c:
        parts = [c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
                 for a, b in zip(cuts[:-1], cuts[1:])]
    assert max(p["num_max"] for p in parts) == ref["num_max"]
    po = np.concatenate([p["per_origin"] for p in parts])
    assert np.array_equal(po, ref["per_origin"])
    best = min((p["argmax_origin"] for p in parts if p["num_max"] == ref["num_max"]))
    assert best == ref["argmax_origin"]
    with _ctx() as c:
        e = c.distance_range(_dev(torch, P), _dev(torch, T), 5, 5)
        assert e["num_max"] == 0 and e["argmax_origin"] == -1


def test_wide_counters_sampled(torch):
    # NP > 65535 switches to two 32-bit histograms; check a sample of origins
    rng = np.random.default_rng(3)
    P = rng.standard_normal((70000, 2)).astype(np.float32)
    T = (rng.standard_normal((3000, 2)) + 0.1).astype(np.float32)
    ranges = [(0, 64), (69990, 70060), (72936, 73000)]
    for path in (pkg.PATH_REGISTER, pkg.PATH_LANE, pkg.PATH_WARP):
        with _ctx(path) as c:
            for a, b in ranges:
                got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
                ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
                assert np.array_equal(got["per_origin"], ref["per_origin"])
                _same(got, ref)


def test_config1_full(torch):
    P, T = wl.CONFIGS["cfg1_d3_200x200_f32"]()
    ref = orc.ddks(P, T)
    for path in (pkg.PATH_AUTO, pkg.PATH_REGISTER, pkg.PATH_LANE, pkg.PATH_WARP, pkg.PATH_SORT):
        with _ctx(path) as c:
            _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


def test_config3_full(torch):
    P, T = wl.CONFIGS["cfg3_d12_4096x4096_f64"]()
    ref = orc.ddks(P, T)
    for path in (pkg.PATH_AUTO, pkg.PATH_WARP, pkg.PATH_SORT):
        with _ctx(path) as c:
            _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)


def test_config2_full(torch):
    P, T = wl.CONFIGS["cfg2_d4_20000x20000_f32_ties"]()
    ref = orc.ddks(P, T, per_origin=True)
    for path in (pkg.PATH_AUTO, pkg.PATH_REGISTER, pkg.PATH_LANE):
        with _ctx(path) as c:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, 40000, per_origin=True)
        assert np.array_equal(got["per_origin"], ref["per_origin"])
        _same(got, ref)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_register_path_rerank_tiles(torch, d):
    # N > 32768 re-ranks dims 1..d-1 per tile of origins; ties in every
    # dimension (small integer grid) stress the window between phases
    rng = np.random.default_rng(40 + d)
    P = rng.integers(0, 50, size=(20000, d)).astype(np.float32)
    T = (rng.integers(0, 50, size=(17000, d)) + (rng.random((17000, d)) < 0.3)).astype(np.float32)
    ranges = [(0, 2000), (19000, 23000), (36000, 37000)]
    with _ctx(pkg.PATH_REGISTER) as c:
        for a, b in ranges:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"])
            _same(got, ref)


@pytest.mark.parametrize("d,n_p,n_t", [(4, 40000, 25000), (3, 60000, 41000), (2, 100000, 50000)])
def test_register_path_large_n(torch, d, n_p, n_t):
    # large re-rank tables; at 150k points the list chunks of a work unit hit
    # their 16-bit cap; sampled origins, ties in every dimension
    rng = np.random.default_rng(70 + d)
    P = rng.integers(0, 3000, size=(n_p, d)).astype(np.float32)
    T = (rng.integers(0, 3000, size=(n_t, d)) + (rng.random((n_t, d)) < 0.3)).astype(np.float32)
    N = n_p + n_t
    ranges = [(0, 150), (n_p - 70, n_p + 90), (N - 130, N)]
    with _ctx(pkg.PATH_REGISTER) as c:
        for a, b in ranges:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"])
            _same(got, ref)


@pytest.mark.parametrize("d", [2, 4, 6])
def test_autotune_picks_an_agreeing_path(torch, d):
    P, T = wl.random_pair(60 + d, 3000, 2500, d, kind="normal")
    ref = orc.ddks(P, T)
    with _ctx() as c:
        path, ms = c.autotune(_dev(torch, P), _dev(torch, T))
        assert path in (pkg.PATH_REGISTER, pkg.PATH_LANE, pkg.PATH_WARP, pkg.PATH_SORT, pkg.PATH_DOMINANCE)
        assert ms > 0
        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)
