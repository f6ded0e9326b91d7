"""Pins of the oracle's vdKS and rdKS (Alg. vdKS, Alg. rdKS) to facts fixed
outside the oracle: special cases that reduce to the exact ddKS or to the
one-dimensional two-sample KS statistic, brute-force restatements on small
inputs, and invariants."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as orc


def _ks_num(a, b):
    """Exact numerator of the 1-D two-sample KS statistic via scipy."""
    st = stats.ks_2samp(a, b, method="asymp").statistic
    return int(round(st * len(a) * len(b)))


@pytest.mark.parametrize("d,R", [(2, 9), (3, 5)])
def test_vdks_with_fine_voxels_is_exact_ddks(d, R):
    # integer coordinates 0..R: with V = 2R voxels per dimension distinct
    # values fall in distinct voxels, so voxel orthants are point orthants
    rng = np.random.default_rng(d)
    P = rng.integers(0, R + 1, size=(40, d)).astype(np.float64)
    T = rng.integers(0, R + 1, size=(33, d)).astype(np.float64)
    P[0, :] = 0
    T[0, :] = R  # the range is [0, R] in every dimension
    assert orc.vdks(P, T, 2 * R)["num_max"] == orc.ddks(P, T)["num_max"]


_GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                     "golden", "hand_cases.json")


def _hand_cases():
    import json
    return json.load(open(_GOLDEN))["cases"]


def test_vdks_hand_cases():
    # the hand-enumerated ddKS cases (small integer grids): with fine voxels
    # vdKS reproduces their exact numerators, the ">=" side convention included
    for case in _hand_cases():
        P = np.array(case["P"], dtype=np.float64)
        T = np.array(case["T"], dtype=np.float64)
        assert orc.vdks(P, T, 64)["num_max"] == case["num_max"], case["name"]


def test_vdks_argmax_is_the_lowest_voxel_and_orthant():
    # brute force over the voxel grid in numpy: orthant sums at every filled
    # voxel, the first (voxel, orthant) in increasing order reaching the max
    rng = np.random.default_rng(12)
    for d, V in [(2, 5), (3, 3)]:
        P, T = rng.normal(size=(60, d)), rng.normal(0.3, 1.0, size=(45, d))
        X = np.concatenate([P, T])
        lo, hi = X.min(axis=0), X.max(axis=0)
        vox = np.minimum(np.floor((X - lo) / (hi - lo) * V), V - 1).astype(np.int64)
        lin = (vox * (V ** np.arange(d))).sum(axis=1)
        w = np.where(np.arange(len(X)) < len(P), -len(T), len(P))
        best, arg = -1, None
        for f in sorted(set(lin.tolist())):
            cf = vox[lin == f][0]
            codes = ((vox >= cf) * (1 << np.arange(d))).sum(axis=1)
            for j in range(1 << d):
                a = abs(int(w[codes == j].sum()))
                if a > best:
                    best, arg = a, (f, j)
        r = orc.vdks(P, T, V)
        assert (r["num_max"], r["argmax_voxel"], r["argmax_orthant"]) == (best, arg[0], arg[1])


def test_vdks_single_voxel_is_zero():
    rng = np.random.default_rng(1)
    P, T = rng.random((30, 3)), rng.random((20, 3)) + 0.5
    assert orc.vdks(P, T, 1)["num_max"] == 0


@pytest.mark.parametrize("V", [1, 3, 16, 1000])
def test_vdks_one_dimension_is_binned_ks(V):
    rng = np.random.default_rng(V)
    P, T = rng.normal(size=(70, 1)), rng.normal(0.4, 1.0, size=(55, 1))
    allv = np.concatenate([P[:, 0], T[:, 0]])
    lo, hi = allv.min(), allv.max()
    binp = np.minimum(np.floor((P[:, 0] - lo) / (hi - lo) * V), V - 1)
    bint = np.minimum(np.floor((T[:, 0] - lo) / (hi - lo) * V), V - 1)
    assert orc.vdks(P, T, V)["num_max"] == _ks_num(binp, bint)


def test_vdks_invariants():
    rng = np.random.default_rng(5)
    P, T = rng.random((25, 2)), rng.random((31, 2)) ** 2
    a, b = orc.vdks(P, T, 7), orc.vdks(T, P, 7)
    assert a["num_max"] == b["num_max"]
    assert 0.0 <= a["D"] <= 1.0
    assert orc.vdks(P, P, 7)["num_max"] == 0


def test_rdks_one_dimension_is_ks():
    rng = np.random.default_rng(7)
    P, T = rng.normal(size=(80, 1)), rng.normal(0.3, 1.2, size=(64, 1))
    r = orc.rdks(P, T)
    want = _ks_num(P[:, 0], T[:, 0])
    assert r["num_max"] == want
    assert list(r["per_corner"]) == [want, want]


def _brute_corner(P, T, corner):
    """sup over pooled distances r of |#P(dist <= r)*NT - #T(dist <= r)*NP|."""
    X = np.concatenate([P, T]).astype(np.float64)
    lo, hi = X.min(axis=0), X.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    Xn = np.where(hi > lo, (X - lo) / span, 0.0)
    c = np.zeros(X.shape[1])
    if corner > 0:
        c[corner - 1] = 1.0
    dist = ((Xn - c) ** 2).sum(axis=1)
    NP, NT = len(P), len(T)
    best = 0
    for r in dist:
        cp = int((dist[:NP] <= r).sum())
        ct = int((dist[NP:] <= r).sum())
        best = max(best, abs(cp * NT - ct * NP))
    return best


@pytest.mark.parametrize("d", [2, 3, 5])
def test_rdks_matches_brute_force(d):
    rng = np.random.default_rng(10 + d)
    P, T = rng.random((37, d)), rng.beta(2, 2, size=(29, d))
    r = orc.rdks(P, T)
    for c in range(d + 1):
        assert int(r["per_corner"][c]) == _brute_corner(P, T, c)
    assert r["num_max"] == max(int(v) for v in r["per_corner"])


def test_rdks_invariants():
    rng = np.random.default_rng(3)
    P, T = rng.random((40, 4)), rng.random((50, 4))
    assert orc.rdks(P, T)["num_max"] == orc.rdks(T, P)["num_max"]
    assert orc.rdks(P, P)["num_max"] == 0
    # a monotone rescale of the whole sample space changes nothing
    assert orc.rdks(P * 3.0 + 1.0, T * 3.0 + 1.0)["num_max"] == orc.rdks(P, T)["num_max"]


def test_rdks_one_dimension_with_ties():
    rng = np.random.default_rng(8)
    P = rng.integers(0, 6, size=(45, 1)).astype(np.float64)
    T = rng.integers(1, 7, size=(38, 1)).astype(np.float64)
    assert orc.rdks(P, T)["num_max"] == _ks_num(P[:, 0], T[:, 0])


def test_rdks_high_dimension_matches_brute_force():
    # rdKS is not limited to ddKS's 30 dimensions (linear in d, Sec. 4's
    # 1000-dimensional study); a few corners of a 40-dimensional case
    rng = np.random.default_rng(40)
    P, T = rng.random((12, 40)), rng.random((9, 40)) ** 1.5
    r = orc.rdks(P, T)
    for c in (0, 1, 17, 40):
        assert int(r["per_corner"][c]) == _brute_corner(P, T, c)
    assert r["num_max"] == max(int(v) for v in r["per_corner"])


@pytest.mark.parametrize("bad", [np.inf, -np.inf, "overflow"])
def test_normalisation_needs_a_finite_range(bad):
    # NormalizeData rescales every dimension by its range: an infinite
    # coordinate, or a range that overflows, has no normalised image
    P = np.array([[0.0, 1.0], [2.0, 3.0]])
    T = np.array([[1.0, 1.0], [0.5, 2.5]])
    if bad == "overflow":
        P[0, 1], T[0, 1] = -1.5e308, 1.5e308
    else:
        T[1, 0] = bad
    for f in (lambda: orc.vdks(P, T, 4), lambda: orc.rdks(P, T)):
        with pytest.raises(orc.OracleError):
            f()
    assert orc.ddks(P, T)["denom"] == 4  # the exact statistic takes them


# ------------------------------------------------------------- planted mistakes
import ctypes  # noqa: E402
import os  # noqa: E402
import subprocess  # noqa: E402

_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ddks_oracle.c")

APPROX_MUTATIONS = [
    ("vdks_strict_side", "if (ccur[m] >= coord[m]) code |= 1 << m;", "if (ccur[m] > coord[m]) code |= 1 << m;"),
    ("vdks_no_abs", "const uint64_t a = (uint64_t)(osum[j] < 0 ? -osum[j] : osum[j]);",
     "const uint64_t a = (uint64_t)(osum[j] > 0 ? osum[j] : 0);"),
    ("vdks_swapped_weights", "diff[idx] += i < NP ? -(int64_t)NT : (int64_t)NP;",
     "diff[idx] += i < NP ? -(int64_t)NP : (int64_t)NT;"),
    ("rdks_inside_ties", "if (i + 1 < N && list[i + 1].r == list[i].r) continue;", ""),
    ("rdks_wrong_corner", "const double x = xn[i * d + corner - 1];", "const double x = xn[i * d + corner % d];"),
    ("rdks_wrong_expansion", "const double t = r - 2.0 * x;", "const double t = r - x;"),
    ("rdks_unnormalised", "out[i * d + m] = span > 0.0 ? (v - lo) / span : 0.0;", "out[i * d + m] = v;"),
]


def _mutant(tmp_path, name, old, new):
    src = open(_SRC).read()
    assert old in src, f"mutation {name}: target text not found in the oracle"
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", str(so), str(c),
                    "-lm"], check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    i64, i32, u64, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
    lib.oracle_vdks.argtypes = [vp, i64, vp, i64, i32, i32, i32, ctypes.POINTER(u64), vp, vp]
    lib.oracle_vdks.restype = i32
    lib.oracle_rdks.argtypes = [vp, i64, vp, i64, i32, i32, ctypes.POINTER(u64), vp]
    lib.oracle_rdks.restype = i32
    lib.oracle_ddks.argtypes = [vp, i64, vp, i64, i32, i32, i64, i64, i32, ctypes.POINTER(u64),
                                ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32), vp]
    lib.oracle_ddks.restype = i32
    return lib


def _m_vdks(lib, P, T, V):
    P, T = np.ascontiguousarray(P, np.float64), np.ascontiguousarray(T, np.float64)
    n = ctypes.c_uint64(0)
    assert lib.oracle_vdks(P.ctypes.data, len(P), T.ctypes.data, len(T), P.shape[1], 1, V, ctypes.byref(n), None,
                           None) == 0
    return n.value


def _m_rdks(lib, P, T):
    P, T = np.ascontiguousarray(P, np.float64), np.ascontiguousarray(T, np.float64)
    n = ctypes.c_uint64(0)
    pc = np.zeros(P.shape[1] + 1, dtype=np.uint64)
    assert lib.oracle_rdks(P.ctypes.data, len(P), T.ctypes.data, len(T), P.shape[1], 1, ctypes.byref(n),
                           pc.ctypes.data) == 0
    return n.value, [int(v) for v in pc]


def _m_ddks(lib, P, T):
    P, T = np.ascontiguousarray(P, np.float64), np.ascontiguousarray(T, np.float64)
    n, k, j = ctypes.c_uint64(0), ctypes.c_int64(0), ctypes.c_int32(0)
    assert lib.oracle_ddks(P.ctypes.data, len(P), T.ctypes.data, len(T), P.shape[1], 1, 0, len(P) + len(T), 1,
                           ctypes.byref(n), ctypes.byref(k), ctypes.byref(j), None) == 0
    return n.value


def _pins_hold(lib):
    """The pins above, run against a (possibly mutated) library."""
    for case in _hand_cases():
        P = np.array(case["P"], dtype=np.float64)
        T = np.array(case["T"], dtype=np.float64)
        if _m_vdks(lib, P, T, 64) != case["num_max"]:
            return False
    rng = np.random.default_rng(0)
    P = rng.integers(0, 6, size=(40, 2)).astype(np.float64)
    T = rng.integers(0, 6, size=(33, 2)).astype(np.float64)
    P[0], T[0] = 0, 5
    if _m_vdks(lib, P, T, 10) != _m_ddks(lib, P, T):
        return False
    P1, T1 = rng.normal(size=(70, 1)), rng.normal(0.4, 1.0, size=(55, 1))
    allv = np.concatenate([P1[:, 0], T1[:, 0]])
    lo, hi = allv.min(), allv.max()
    binp = np.minimum(np.floor((P1[:, 0] - lo) / (hi - lo) * 16), 15)
    bint = np.minimum(np.floor((T1[:, 0] - lo) / (hi - lo) * 16), 15)
    if _m_vdks(lib, P1, T1, 16) != _ks_num(binp, bint):
        return False
    Pi = rng.integers(0, 6, size=(45, 1)).astype(np.float64)
    Ti = rng.integers(1, 7, size=(38, 1)).astype(np.float64)
    if _m_rdks(lib, Pi, Ti)[0] != _ks_num(Pi[:, 0], Ti[:, 0]):
        return False
    P3, T3 = rng.random((37, 3)), rng.beta(2, 2, size=(29, 3))
    num, pc = _m_rdks(lib, P3, T3)
    return all(pc[c] == _brute_corner(P3, T3, c) for c in range(4))


def test_pins_hold_for_the_oracle(tmp_path):
    assert _pins_hold(_mutant(tmp_path, "unchanged", "", ""))


@pytest.mark.parametrize("name,old,new", APPROX_MUTATIONS, ids=[m[0] for m in APPROX_MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    assert not _pins_hold(_mutant(tmp_path, name, old, new))


def _ks_num_sorted(dp, dt):
    """sup over r of |#P(dist <= r)*NT - #T(dist <= r)*NP| by one sorted sweep."""
    NP, NT = len(dp), len(dt)
    allv = np.concatenate([dp, dt])
    is_p = np.concatenate([np.ones(NP, dtype=np.int64), np.zeros(NT, dtype=np.int64)])
    order = np.argsort(allv, kind="stable")
    v = allv[order]
    cp = np.cumsum(is_p[order])
    ct = np.cumsum(1 - is_p[order])
    last = np.r_[v[1:] != v[:-1], True]  # evaluate after every distance equal to r
    return int(np.abs(cp[last] * NT - ct[last] * NP).max())


def test_rdks_expanded_distance_agrees_with_euclidean():
    # The oracle (and the kernel) compute the squared distance to e_m as
    # (|x'|^2 - 2 x'_m) + 1 (rdKS linear in d, Sec. 2.2 / Sec. 4) instead of
    # sum_j (x'_j - e_j)^2.  Over many seeds and value structures -- continuous
    # data, heavy tails, and dyadic grids whose distances tie exactly -- the two
    # forms give the same per-corner statistic, and the pairs of distances the
    # two forms put in a different order are rare (near-ties within rounding).
    rng = np.random.default_rng(2024)
    inversions = pairs = 0
    for case in range(60):
        d = int(rng.integers(2, 11))
        n_p, n_t = int(rng.integers(20, 300)), int(rng.integers(20, 300))
        kind = case % 4
        if kind == 0:
            P, T = rng.random((n_p, d)), rng.random((n_t, d)) ** 1.3
        elif kind == 1:
            P, T = rng.standard_cauchy((n_p, d)), rng.standard_cauchy((n_t, d)) + 0.2
        elif kind == 2:  # dyadic grid: normalised coordinates k/16, exact ties
            P = rng.integers(0, 17, size=(n_p, d)) / 16.0
            T = rng.integers(0, 17, size=(n_t, d)) / 16.0
            P[0], T[0] = 0.0, 1.0  # the range is exactly [0, 1]
        else:
            P, T = rng.standard_normal((n_p, d)), rng.standard_normal((n_t, d)) * 1.1
        r = orc.rdks(P, T)
        X = np.concatenate([P, T]).astype(np.float64)
        lo, hi = X.min(axis=0), X.max(axis=0)
        span = np.where(hi > lo, hi - lo, 1.0)
        Xn = np.where(hi > lo, (X - lo) / span, 0.0)
        s = np.zeros(len(Xn))
        for j in range(d):  # the oracle's order: dimension by dimension
            s = s + Xn[:, j] * Xn[:, j]
        for c in range(d + 1):
            e = np.zeros(d)
            if c > 0:
                e[c - 1] = 1.0
            euclid = ((Xn - e) ** 2).sum(axis=1)
            expanded = s if c == 0 else (s - 2.0 * Xn[:, c - 1]) + 1.0
            assert int(r["per_corner"][c]) == _ks_num_sorted(euclid[:n_p], euclid[n_p:]), (case, c)
            assert _ks_num_sorted(expanded[:n_p], expanded[n_p:]) == int(r["per_corner"][c]), (case, c)
            if case % 6 == 0 and c < 3:
                a = np.sign(euclid[:, None] - euclid[None, :])
                b = np.sign(expanded[:, None] - expanded[None, :])
                inversions += int((a != b).sum()) // 2
                pairs += len(euclid) * (len(euclid) - 1) // 2
    assert pairs > 100000
    assert inversions <= pairs * 1e-4, (inversions, pairs)
