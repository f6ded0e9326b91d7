"""Parity of the CUDA vdKS and rdKS (Alg. vdKS, Alg. rdKS of Sec. 2.2) with
the CPU oracle, through the C ABI.

Both statistics are integers (numerator over NP*NT) computed from the same
IEEE double normalisation, so the bar is bit-exact: num_max, the arg-max
voxel and orthant for vdKS, every corner's numerator for rdKS.  Sizes span
several CTAs and sort chunks with ragged tails; the cases cover ties, constant
dimensions, one voxel, one dimension, the thread and warp distance kernels of
rdKS and the paper's 1000-dimensional DVU case.
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


@pytest.fixture(scope="module")
def ctx(torch):
    with pkg.Context(device=0) as c:
        yield c


def _dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _vdks_same(got, ref):
    assert got["num_max"] == ref["num_max"]
    assert got["denom"] == ref["denom"]
    assert got["argmax_origin"] == ref["argmax_voxel"]
    assert got["argmax_orthant"] == ref["argmax_orthant"]


def _rdks_same(got, ref):
    assert got["num_max"] == ref["num_max"]
    assert got["denom"] == ref["denom"]
    assert np.array_equal(got["per_corner"], ref["per_corner"])
    assert got["argmax_origin"] == int(np.argmax(ref["per_corner"] == ref["num_max"]))


VDKS_CASES = [
    (1, 500, 400, 7, "normal"), (1, 300, 333, 1000, "int"), (2, 3000, 2500, 16, "normal"),
    (2, 900, 700, 64, "int"), (3, 2000, 2100, 9, "normal"), (3, 1500, 1400, 32, "int"),
    (4, 700, 650, 5, "normal"), (5, 300, 280, 4, "normal"), (6, 200, 150, 3, "int"),
    (7, 120, 130, 3, "normal"), (8, 100, 90, 2, "normal"), (10, 60, 70, 2, "normal"),
    (3, 400, 300, 6, "shifted"), (2, 50, 40, 8, "const"),
    # many voxels per dimension for the points: the double rescaling of
    # every coordinate instead of the thresholds
    (3, 300, 300, 40, "normal"), (2, 400, 300, 200, "int"), (1, 2000, 1500, 100000, "normal"),
    # many points per voxel: CTA-private shared-memory histograms (with the
    # thresholds for d <= 4 and d > 4, and with the double rescaling)
    (4, 6000, 5000, 5, "normal"), (6, 3000, 3000, 2, "int"), (1, 2000, 1500, 100, "normal"),
    (2, 9000, 200, 7, "normal"),
]


@pytest.mark.parametrize("d,n_p,n_t,V,kind", VDKS_CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_vdks_matches_oracle(torch, ctx, d, n_p, n_t, V, kind, dtype):
    P, T = wl.random_pair(100 + d * 7 + V, n_p, n_t, d, kind=kind, dtype=dtype)
    ref = orc.vdks(P, T, V)
    _vdks_same(ctx.vdks(_dev(torch, P), _dev(torch, T), V), ref)
    _vdks_same(ctx.vdks(P, T, V), ref)  # host inputs


def test_vdks_single_voxel_and_duplicates(torch, ctx):
    P, T = wl.random_pair(3, 777, 501, 3, kind="normal")
    r = ctx.vdks(_dev(torch, P), _dev(torch, T), 1)
    assert r["num_max"] == 0 and r["argmax_origin"] == 0
    P2, T2 = np.concatenate([P, P]), np.concatenate([T, T])
    a = ctx.vdks(_dev(torch, P), _dev(torch, T), 11)
    b = ctx.vdks(_dev(torch, P2), _dev(torch, T2), 11)
    assert b["num_max"] == 4 * a["num_max"]


def test_vdks_dvu_and_mixture(torch, ctx):
    for P, T, V in [wl.dvu_pair(1, 3000, 2800, 3) + (20,),
                    wl.mixture_pair(2, 5000, 4000, 3, shift=0.2) + (32,),
                    wl.gaussian_pair(4, 2000, 2000, 6) + (4,)]:
        _vdks_same(ctx.vdks(_dev(torch, P), _dev(torch, T), V), orc.vdks(P, T, V))


@pytest.mark.parametrize("d,V", [(3, 6), (6, 2)])
def test_vdks_unaligned_rows(torch, ctx, d, V):
    # rows that start off a 16-byte boundary: the shared-memory histogram
    # path without bulk copies
    P, T = wl.random_pair(77 + d, 6000, 5500, d, kind="normal")
    Pb = torch.zeros((len(P) + 1, d), dtype=torch.float32, device="cuda")
    Tb = torch.zeros((len(T) + 1, d), dtype=torch.float32, device="cuda")
    Pb[1:] = _dev(torch, P)
    Tb[1:] = _dev(torch, T)
    Pv, Tv = Pb[1:], Tb[1:]
    assert Pv.is_contiguous() and Pv.data_ptr() % 16 != 0
    _vdks_same(ctx.vdks(Pv, Tv, V), orc.vdks(P, T, V))


@pytest.mark.parametrize("n", [200_000, 300_000])
def test_vdks_large_full_grid(torch, ctx, n):
    # the bench's grid (32^3 voxels, float32 Gaussian pair): at 400k points
    # the voxel counts go to global memory, at 600k (16 points per voxel) to
    # CTA-private shared-memory histograms like the bench's 16M points
    P, T = wl.gaussian_pair(0, n, n, 3, shift=0.2)
    _vdks_same(ctx.vdks(_dev(torch, P), _dev(torch, T), 32), orc.vdks(P, T, 32))


RDKS_CASES = [
    (1, 500, 400, "normal"), (1, 3000, 2000, "int"), (2, 3000, 2900, "normal"),
    (3, 5000, 4000, "normal"), (3, 2500, 2600, "int"), (7, 1000, 1100, "normal"),
    (16, 700, 500, "normal"), (17, 300, 200, "normal"), (40, 100, 90, "int"),
    (5, 60, 40, "const"), (4, 1200, 900, "shifted"),
]


@pytest.mark.parametrize("d,n_p,n_t,kind", RDKS_CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rdks_matches_oracle(torch, ctx, d, n_p, n_t, kind, dtype):
    P, T = wl.random_pair(200 + d, n_p, n_t, d, kind=kind, dtype=dtype)
    ref = orc.rdks(P, T)
    _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), ref)
    _rdks_same(ctx.rdks(P, T), ref)


def test_rdks_dvu_1000_dimensions(torch, ctx):
    # the paper's high-dimensional rdKS case: 100 points per sample in d = 1000
    for seed in (0, 1):
        P, T = wl.dvu_pair(seed, 100, 100, 1000)
        _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), orc.rdks(P, T))


def test_rdks_large_n(torch, ctx):
    # many sort chunks and merge passes (N = 300k, 4 corners)
    P, T = wl.gaussian_pair(5, 150_000, 150_000, 3, shift=0.05)
    _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), orc.rdks(P, T))


def test_replay_and_new_values(torch):
    P, T = wl.random_pair(9, 2000, 1800, 3, kind="normal")
    P2, T2 = wl.random_pair(10, 2000, 1800, 3, kind="int")
    Pd, Td = _dev(torch, P), _dev(torch, T)
    with pkg.Context(device=0) as c:
        rv, rr = orc.vdks(P, T, 12), orc.rdks(P, T)
        for _ in range(4):
            _vdks_same(c.vdks(Pd, Td, 12), rv)
            _rdks_same(c.rdks(Pd, Td), rr)
        assert c.stats()["graph_replays"] >= 4
        Pd.copy_(_dev(torch, P2))
        Td.copy_(_dev(torch, T2))
        _vdks_same(c.vdks(Pd, Td, 12), orc.vdks(P2, T2, 12))
        _rdks_same(c.rdks(Pd, Td), orc.rdks(P2, T2))


def test_errors(torch, ctx):
    P, T = wl.random_pair(1, 50, 40, 3)
    calls = [lambda A, B: ctx.vdks(_dev(torch, A), _dev(torch, B), 4),
             lambda A, B: ctx.rdks(_dev(torch, A), _dev(torch, B))]
    nan, inf = T.copy(), T.copy()
    nan[3, 1] = np.nan
    inf[0, 0] = np.inf
    huge = T.astype(np.float64)
    huge[0, 0], huge[1, 0] = -1.5e308, 1.5e308  # the range overflows
    for f in calls:
        for A, B, code in [(P, nan, -2), (P, inf, -1), (P.astype(np.float64), huge, -1)]:
            with pytest.raises(pkg.DdksError) as e:
                f(A, B)
            assert e.value.code == code
    with pytest.raises(pkg.DdksError) as e:
        ctx.vdks(_dev(torch, P), _dev(torch, T), 0)
    assert e.value.code == -1
    P11, T11 = wl.random_pair(1, 20, 20, 11)
    with pytest.raises(pkg.DdksError) as e:
        ctx.vdks(_dev(torch, P11), _dev(torch, T11), 2)
    assert e.value.code == -8
    P3, T3 = wl.random_pair(1, 20, 20, 3)
    with pytest.raises(pkg.DdksError) as e:
        ctx.vdks(_dev(torch, P3), _dev(torch, T3), 1000)  # 10^9 voxels
    assert e.value.code == -8
    # the context stays usable after the errors
    _vdks_same(ctx.vdks(_dev(torch, P), _dev(torch, T), 4), orc.vdks(P, T, 4))
    _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), orc.rdks(P, T))


def test_vdks_bench_workload_full_size(torch, ctx):
    # the bench's vdKS workload itself (8M + 8M float32, 32 voxels per
    # dimension: bulk-copy voxel pass, CTA-private histograms), checked whole
    P, T = wl.gaussian_pair(0, 8_000_000, 8_000_000, 3, shift=0.2)
    _vdks_same(ctx.vdks(_dev(torch, P), _dev(torch, T), 32), orc.vdks(P, T, 32))


def test_rdks_bench_workload_full_size(torch, ctx):
    # the bench's large rdKS workload (1M + 1M float32, d = 3), checked whole
    P, T = wl.gaussian_pair(0, 1_000_000, 1_000_000, 3, shift=0.05)
    _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), orc.rdks(P, T))



def _ieee_rescale(v, lo, span):
    # NormalizeData in plain IEEE double: numpy's subtraction and division round to nearest
    if span == 0.0:
        return np.zeros_like(v)
    return (v - lo) / span


@pytest.mark.parametrize("lo,span", [(0.0, 1.0), (-3.25, 7.5), (1.0, 3.0), (-1e-3, 2.0 ** -20 * 3),
                                     (12345.678, 0.1), (-2.0 ** 40, 2.0 ** 41 + 1.0), (0.5, 2.0 ** -1000),
                                     (-7.0, 2.0 ** 60 * 1.75), (3.0, 0.0)])
def test_rescale_is_ieee_division(torch, ctx, lo, span):
    # the FMA quotient with its remainder certificate against the IEEE expression, bit for bit
    rng = np.random.default_rng(abs(hash((lo, span))) % 2 ** 32)
    n = 1 << 20
    u = rng.random(n)
    v = lo + u * span
    v = np.minimum(np.maximum(v, lo), lo + span)
    # values whose quotients sit at binade edges, tiny offsets, the ends of the range
    ks = rng.integers(1, 60, 4096)
    edge = lo + span * np.ldexp(1.0, -ks) * (1.0 + rng.integers(-3, 4, 4096) * 2.0 ** -52)
    tiny = lo + np.ldexp(rng.random(4096), -rng.integers(900, 1074, 4096))
    v = np.concatenate([v, edge, tiny, [lo, lo + span, np.nextafter(lo, np.inf)]])
    v = v[(v >= lo) & (v <= lo + span) & np.isfinite(v)]
    ref = _ieee_rescale(v, lo, span)
    got = ctx.rescale(_dev(torch, v), lo, span).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    got_h = ctx.rescale(v, lo, span)
    assert np.array_equal(got_h.view(np.uint64), ref.view(np.uint64))


def test_rescale_random_operands(torch, ctx):
    # random doubles of every magnitude as (v - lo, span) pairs, many per call
    rng = np.random.default_rng(11)
    for _ in range(8):
        span = float(np.ldexp(1.0 + rng.random(), int(rng.integers(-1000, 1000))))
        e = rng.integers(-1074, 1, 1 << 18)
        v = np.ldexp(rng.random(1 << 18), e) * span
        v = np.minimum(v, span)
        ref = _ieee_rescale(v, 0.0, span)
        got = ctx.rescale(_dev(torch, v), 0.0, span).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rdks_histogram_path(torch, ctx, dtype):
    # N >= 8192 takes the histogram path: bucket ends exact, mixed buckets
    # that could beat them sorted in shared memory.  Heavy ties (integer
    # grids: buckets of equal keys), continuous data, and shapes whose
    # buckets force the rerun on the sorting path: P = T (every bucket end
    # is 0, more than 1,024 candidates), one tight cluster plus two outliers
    # (more than 8,192 points in one candidate bucket), all points equal.
    rng = np.random.default_rng(77)
    cases = [wl.random_pair(301, 6000, 5000, 3, kind="int", dtype=dtype),
             wl.random_pair(302, 9000, 8000, 2, kind="int", dtype=dtype),
             wl.random_pair(303, 7000, 9000, 5, kind="normal", dtype=dtype)]
    X = rng.standard_normal((20000, 3)).astype(dtype)
    cases.append((X, X.copy()))
    C = (rng.standard_normal((12000, 2)) * 1e-6).astype(dtype)
    C[0], C[1] = -1.0, 1.0
    cases.append((C[:6000], C[6000:]))
    Z = np.ones((5000, 4), dtype=dtype)
    cases.append((Z, Z[:4000].copy()))
    for P, T in cases:
        ref = orc.rdks(P, T)
        _rdks_same(ctx.rdks(_dev(torch, P), _dev(torch, T)), ref)
