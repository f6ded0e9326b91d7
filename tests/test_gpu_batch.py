"""Many uneven problems in one persistent launch (ddks_batch_distance): each
result equals the oracle's, and equals the same problem computed alone."""
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


def _key(r):
    return (r["num_max"], r["denom"], r["argmax_origin"], r["argmax_orthant"])


def test_uneven_problems_match_oracle(torch):
    probs = wl.uneven_problems(seed=0, count=64, n_lo=16, n_hi=1500, dims=tuple(range(1, 12)))
    with pkg.Context(device=0) as c:
        got = c.batch_distance([(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs])
        alone = [c.distance(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs]
    for (P, T), g, a in zip(probs, got, alone):
        ref = orc.ddks(P, T)
        assert _key(g) == _key(ref)
        assert _key(a) == _key(ref)


def test_host_inputs_and_large_members(torch):
    probs = wl.uneven_problems(seed=3, count=6, n_lo=50, n_hi=400, dims=(2, 7, 12))
    P, T = wl.gaussian_pair(seed=9, n_p=9000, n_t=8000, d=3)  # N > 16384: single path
    probs.append((P, T))
    with pkg.Context(device=0) as c:
        got = c.batch_distance(probs)  # numpy (host) inputs
    for (P, T), g in zip(probs, got):
        assert _key(g) == _key(orc.ddks(P, T))


def test_config4_256_uneven(torch):
    probs = wl.uneven_problems(seed=0, count=256)
    with pkg.Context(device=0) as c:
        got = c.batch_distance([(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs])
    # the oracle on a seeded sample of 24 problems (all 256 take minutes on the host)
    rng = np.random.default_rng(0)
    for i in rng.choice(256, size=24, replace=False):
        P, T = probs[i]
        assert _key(got[i]) == _key(orc.ddks(P, T))


SHAPES = [(ot, pt) for ot in (32, 64, 128) for pt in (256, 512, 1024)]
BITS_SHAPES = [(127, pt) for pt in (256, 512, 1024, 2048)]  # bit-sliced unit, 2 <= d <= 6
BYTE_SHAPES = [(ot, pt) for ot in (31, 63, 127) for pt in (256, 2048)]  # byte unit, d = 7, 8


def _shape_ok(d, ot, pt):
    if ot == 127:  # the bit-sliced unit for d <= 6, the byte unit for d = 7, 8
        return 2 <= d <= 8
    if ot in (31, 63):
        return d in (7, 8)
    return True


def test_every_tile_shape_matches_oracle(torch):
    # the batched units' tile shapes (origins per unit, points per staged
    # tile) change the work split, never the result; ragged tails everywhere
    probs = wl.uneven_problems(seed=5, count=22, n_lo=20, n_hi=1300, dims=tuple(range(1, 12)))
    refs = [orc.ddks(P, T) for P, T in probs]
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs]
    with pkg.Context(device=0) as c:
        for ot, pt in SHAPES + BITS_SHAPES + BYTE_SHAPES:
            for d in range(1, 12):
                if _shape_ok(d, ot, pt):
                    c.set_batch_shape(d, ot, pt)
            got = c.batch_distance(dev)
            for g, r in zip(got, refs):
                assert _key(g) == _key(r), (ot, pt)
        for d, ot, pt in [(3, 48, 512), (9, 127, 1024), (1, 127, 1024), (3, 64, 2048), (4, 127, 128),
                          (6, 63, 1024), (9, 31, 512), (8, 63, 128)]:
            with pytest.raises(pkg.DdksError):
                c.set_batch_shape(d, ot, pt)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_bit_sliced_unit_edges(torch, d):
    # the bit-sliced unit against the oracle: one-point samples, samples of
    # exactly 32k points, ragged tails, heavy ties (integer grids, so origins
    # share values inside a block and splits land on group boundaries), and
    # the largest batched size (16,384 pooled points)
    rng = np.random.default_rng(40 + d)
    shapes = [(1, 1), (1, 40), (33, 1), (32, 64), (127, 128), (200, 55), (700, 901), (64, 4000)]
    probs = []
    for i, (n_p, n_t) in enumerate(shapes):
        kind = "int" if i % 2 else "normal"
        probs.append(wl.random_pair(500 + 10 * d + i, n_p, n_t, d, kind=kind))
    P = rng.integers(0, 6, size=(300, d)).astype(np.float32)  # very few distinct values
    T = rng.integers(0, 6, size=(260, d)).astype(np.float32)
    probs.append((P, T))
    refs = [orc.ddks(P, T) for P, T in probs]
    big = wl.random_pair(77 + d, 8192, 8192, d, kind="int")
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs + [big]]
    with pkg.Context(device=0) as c:
        for pt in (256, 2048):
            c.set_batch_shape(d, 127, pt)
            got = c.batch_distance(dev)
            for g, r in zip(got, refs):
                assert _key(g) == _key(r), (pt, g, r)
            # the largest problem: against the histogram unit and the
            # single-problem path (the oracle over 16,384^2 pairs takes too long)
            c.set_batch_shape(d, 64, 512)
            hist = c.batch_distance(dev[-1:])[0]
            alone = c.distance(*dev[-1])
            assert _key(got[-1]) == _key(hist) == _key(alone)


def test_autotuned_shapes_and_results(torch):
    probs = wl.uneven_problems(seed=6, count=40, n_lo=64, n_hi=3000, dims=(2, 3, 5, 8))
    refs = [orc.ddks(P, T) for P, T in probs]
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs]
    with pkg.Context(device=0) as c:
        shapes = c.autotune_batch(dev)
        for d in (2, 3, 5, 8):
            ot, pt = shapes[d]
            if ot == 127:
                assert 2 <= d <= 8 and pt in (256, 512, 1024, 2048)
            elif ot in (31, 63):
                assert d in (7, 8) and pt in (256, 512, 1024, 2048)
            else:
                assert ot in (32, 64, 128) and pt in (256, 512, 1024)
        for _ in range(2):  # direct, then captured
            got = c.batch_distance(dev)
            assert [_key(g) for g in got] == [_key(r) for r in refs]


@pytest.mark.parametrize("d", [7, 8])
def test_byte_unit_edges(torch, d):
    # the byte unit against the oracle: one-point samples, ragged tails, unit
    # boundaries (31 and 63 origins), heavy ties, and 16,384 pooled points
    rng = np.random.default_rng(60 + d)
    shapes = [(1, 1), (1, 40), (33, 1), (31, 32), (63, 64), (200, 55), (700, 901), (64, 3000)]
    probs = []
    for i, (n_p, n_t) in enumerate(shapes):
        probs.append(wl.random_pair(600 + 10 * d + i, n_p, n_t, d, kind="int" if i % 2 else "normal"))
    P = rng.integers(0, 3, size=(300, d)).astype(np.float32)  # three values per dimension
    T = rng.integers(0, 3, size=(260, d)).astype(np.float32)
    probs.append((P, T))
    refs = [orc.ddks(P, T) for P, T in probs]
    big = wl.random_pair(88 + d, 8192, 8192, d, kind="int")
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs + [big]]
    with pkg.Context(device=0) as c:
        c.set_batch_shape(d, 64, 512)
        hist = c.batch_distance(dev[-1:])[0]
        alone = c.distance(*dev[-1])
        assert _key(hist) == _key(alone)
        for ot, pt in [(31, 256), (63, 2048), (63, 512), (127, 512), (127, 2048)]:
            c.set_batch_shape(d, ot, pt)
            got = c.batch_distance(dev)
            for g, r in zip(got, refs):
                assert _key(g) == _key(r), (ot, pt, g, r)
            assert _key(got[-1]) == _key(hist)


def test_float64_both_rank_classes(torch):
    # K0 of the batch sorts each (problem, dimension) in one CTA; problems
    # above 4,096 pooled points take the 1,024-thread class, up to the
    # 16,384-point limit where a float64 row fills the CTA's shared memory
    rng = np.random.default_rng(12)
    probs = [wl.random_pair(81, 8192, 8192, 3, kind="int", dtype=np.float64),
             wl.random_pair(82, 3000, 2100, 2, kind="normal", dtype=np.float64),
             wl.random_pair(83, 40, 9, 5, kind="int", dtype=np.float64),
             wl.random_pair(84, 1, 1, 4, kind="normal", dtype=np.float64)]
    P = rng.standard_normal((700, 6))
    P[:100, 1] = -0.0  # signed zeros tie with +0.0
    T = rng.standard_normal((650, 6))
    T[:50, 1] = 0.0
    T[60:70, 2] = np.inf
    probs.append((P, T))
    dev = [(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()) for P, T in probs]
    with pkg.Context(device=0) as c:
        for shapes in ((64, 512), (127, 1024)):
            for d in range(2, 7):
                c.set_batch_shape(d, *shapes)
            got = c.batch_distance(dev)
            for i, ((P, T), g) in enumerate(zip(probs, got)):
                if i == 0:  # 16,384 points: against the single-problem path
                    assert _key(g) == _key(c.distance(*dev[0]))
                else:
                    assert _key(g) == _key(orc.ddks(P, T)), (i, shapes)
        bad = [(x.clone(), y.clone()) for x, y in dev[1:3]]
        bad[1][1][3, 0] = float("nan")
        with pytest.raises(pkg.DdksError) as e:
            c.batch_distance(bad)
        assert e.value.code == -2
