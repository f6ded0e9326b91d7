"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-enumerated tiny cases (tests/golden/hand_cases.json);
* a second, independent restatement of the definition (orthant membership by
  matching all d bits, pure Python) on small random inputs with many ties;
* d = 1 reduces to the textbook two-sample KS statistic (scipy's ks_2samp and a
  sorted merge written here);
* closed forms (samples separated in every coordinate give D = 1) and the
  invariants the paper states (App. A: identity, symmetry) plus ones that
  follow from the definition (row/coordinate order, strictly increasing maps,
  duplication, 0 <= num <= NP*NT, the per-dimension KS lower bound);
* Philox4x64-10 against numpy's independent implementation;
* the significance cell probability against scipy's binomial/Poisson pmfs.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def test_hand_cases():
    cases = json.load(open(GOLDEN))["cases"]
    assert len(cases) >= 5
    for c in cases:
        r = orc.ddks(c["P"], c["T"])
        assert (r["num_max"], r["denom"]) == (c["num_max"], c["denom"]), c["name"]
        assert orc.brute_force_ddks(c["P"], c["T"]) == (c["num_max"], c["denom"]), c["name"]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["normal", "int"])
def test_against_membership_restatement(d, kind):
    for seed in range(4):
        n_p, n_t = 5 + seed, 7 - seed // 2
        P, T = wl.random_pair(seed, n_p, n_t, d, kind=kind, dtype=np.float64)
        r = orc.ddks(P, T)
        assert (r["num_max"], r["denom"]) == orc.brute_force_ddks(P, T)


def ks_sorted_merge(x, y):
    """Two-sample KS numerator sup|F_x - F_y| * nx * ny by a sorted merge,
    advancing all tied values together."""
    x = np.sort(np.asarray(x, dtype=np.float64))
    y = np.sort(np.asarray(y, dtype=np.float64))
    nx, ny = len(x), len(y)
    i = j = 0
    best = 0
    while i < nx or j < ny:
        v = min(x[i] if i < nx else np.inf, y[j] if j < ny else np.inf)
        while i < nx and x[i] == v:
            i += 1
        while j < ny and y[j] == v:
            j += 1
        best = max(best, abs(i * ny - j * nx))
    return best


@pytest.mark.parametrize("kind", ["normal", "int"])
def test_d1_is_two_sample_ks(kind):
    scipy_stats = pytest.importorskip("scipy.stats")
    for seed in range(12):
        n_p, n_t = 20 + 3 * seed, 31 - seed
        P, T = wl.random_pair(100 + seed, n_p, n_t, 1, kind=kind, dtype=np.float64)
        r = orc.ddks(P, T)
        assert r["num_max"] == ks_sorted_merge(P[:, 0], T[:, 0])
        ks = scipy_stats.ks_2samp(P[:, 0], T[:, 0]).statistic
        assert round(ks * n_p * n_t) == r["num_max"]


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_separated_samples_give_one(d):
    P, T = wl.random_pair(7, 13, 9, d, kind="shifted", dtype=np.float64)
    r = orc.ddks(P, T)
    assert r["num_max"] == r["denom"] == 13 * 9
    r = orc.ddks(T, P)
    assert r["num_max"] == r["denom"]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_invariants(d):
    rng = np.random.default_rng(d)
    for kind in ("normal", "int"):
        P, T = wl.random_pair(d * 10 + 1, 23, 17, d, kind=kind, dtype=np.float64)
        r = orc.ddks(P, T)
        num, den = r["num_max"], r["denom"]
        assert 0 <= num <= den
        # identity (App. A)
        assert orc.ddks(P, P)["num_max"] == 0
        assert orc.ddks(T, T.copy())["num_max"] == 0
        # symmetry (App. A)
        assert orc.ddks(T, P)["num_max"] == num
        # order of rows and of coordinates
        assert orc.ddks(P[rng.permutation(len(P))], T[rng.permutation(len(T))])["num_max"] == num
        perm = rng.permutation(d)
        assert orc.ddks(P[:, perm], T[:, perm])["num_max"] == num
        # strictly increasing per-coordinate maps (exact in floating point)
        assert orc.ddks(P * 8.0 + 0.0, T * 8.0)["num_max"] == num
        assert orc.ddks(np.exp(P / 4.0), np.exp(T / 4.0))["num_max"] == num
        # duplicating both samples scales numerator and denominator by 4
        r2 = orc.ddks(np.concatenate([P, P]), np.concatenate([T, T]))
        assert (r2["num_max"], r2["denom"]) == (4 * num, 4 * den)
        # the per-dimension KS statistics bound D from below
        ks = max(ks_sorted_merge(P[:, m], T[:, m]) for m in range(d))
        assert num * 2 ** (d - 1) >= ks


def test_float32_and_float64_agree_on_same_values():
    P, T = wl.gaussian_pair(seed=3, n_p=40, n_t=50, d=3)
    r32 = orc.ddks(P, T)
    r64 = orc.ddks(P.astype(np.float64), T.astype(np.float64))
    assert r32 == r64


def test_negative_zero_and_infinities():
    P = np.array([[0.0, -np.inf], [1.0, 2.0]])
    T = np.array([[-0.0, np.inf], [1.0, -1.0], [np.inf, 0.0]])
    r = orc.ddks(P, T)
    assert (r["num_max"], r["denom"]) == orc.brute_force_ddks(P, T)
    # -0.0 and +0.0 compare equal: swapping them changes nothing
    P2 = P.copy(); P2[0, 0] = -0.0
    T2 = T.copy(); T2[0, 0] = 0.0
    assert orc.ddks(P2, T2)["num_max"] == r["num_max"]


def test_nan_rejected():
    P = np.array([[0.0, np.nan]])
    T = np.array([[1.0, 1.0]])
    with pytest.raises(orc.OracleError) as e:
        orc.ddks(P, T)
    assert e.value.code == -2


def test_high_d_sort_path_matches_dense_path():
    # a constant extra coordinate puts every point on the >= side of every
    # origin in that dimension, so the partition (and the statistic) is unchanged
    P, T = wl.random_pair(5, 30, 25, 16, kind="int", dtype=np.float64)
    r16 = orc.ddks(P, T)
    P17 = np.concatenate([P, np.ones((30, 1))], axis=1)
    T17 = np.concatenate([T, np.ones((25, 1))], axis=1)
    r17 = orc.ddks(P17, T17)
    assert r17["num_max"] == r16["num_max"]
    assert r17["argmax_origin"] == r16["argmax_origin"]
    assert r17["argmax_orthant"] == r16["argmax_orthant"] | (1 << 16)
    # and a random high-d case against the membership restatement (d = 18 is
    # too large for it, so compare against the 16-d projection plus constants)
    P20 = np.concatenate([P, np.zeros((30, 4))], axis=1)
    T20 = np.concatenate([T, np.zeros((25, 4))], axis=1)
    assert orc.ddks(P20, T20)["num_max"] == r16["num_max"]


def test_origin_range_and_per_origin():
    P, T = wl.random_pair(9, 31, 29, 3, kind="int", dtype=np.float64)
    full = orc.ddks(P, T, per_origin=True)
    N = 60
    parts = [orc.ddks(P, T, origins=(a, b), per_origin=True) for a, b in [(0, 17), (17, 40), (40, N)]]
    assert max(p["num_max"] for p in parts) == full["num_max"]
    assert np.array_equal(np.concatenate([p["per_origin"] for p in parts]), full["per_origin"])
    assert full["per_origin"][full["argmax_origin"]] == full["num_max"]
    assert np.all(full["per_origin"][: full["argmax_origin"]] < full["num_max"])


def test_threads_do_not_change_result():
    P, T = wl.gaussian_pair(seed=11, n_p=150, n_t=120, d=4)
    assert orc.ddks(P, T, nthreads=1) == orc.ddks(P, T, nthreads=4)


# ---------------------------------------------------------------- Philox / perms
def test_philox_matches_numpy():
    for key, ctr in [((0, 0), (0, 0, 0, 0)), ((5, 7), (2**64 - 1, 3, 0, 0)),
                     ((0xDEADBEEF, 1 << 40), (123, 456, 789, 1011))]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
        ref = bg.random_raw(4)
        # numpy advances the counter before it draws a block
        c = list(ctr)
        c[0] = (c[0] + 1) % 2**64
        if c[0] == 0:
            c[1] = (c[1] + 1) % 2**64
        assert np.array_equal(orc.philox4x64_10(c, key), ref)


def test_perm_labels():
    NP, NT = 37, 23
    seen = set()
    freq = np.zeros(NP + NT)
    for b in range(200):
        lab = orc.perm_labels(42, b, NP, NT)
        assert lab.sum() == NP
        seen.add(lab.tobytes())
        freq += lab
    assert len(seen) == 200
    # every point lands in P with frequency NP/N (loose binomial check)
    p = NP / (NP + NT)
    sd = np.sqrt(200 * p * (1 - p))
    assert np.all(np.abs(freq - 200 * p) < 5 * sd)
    # key k(b, i) is word i%4 of Philox(ctr=(i//4, b, 0, 0), key=(seed, 0))
    w = orc.philox4x64_10([2, 5, 0, 0], [42, 0])
    assert orc.perm_key(42, 5, 9) == int(w[1])


def test_permutation_test_definition():
    P, T = wl.gaussian_pair(seed=1, n_p=12, n_t=9, d=2, shift=0.4, dtype=np.float64)
    B = 30
    r = orc.permutation_test(P, T, B, seed=7)
    X = np.concatenate([P, T])
    nums = []
    for b in range(B):
        lab = orc.perm_labels(7, b, 12, 9).astype(bool)
        nums.append(orc.brute_force_ddks(X[lab], X[~lab])[0])
    assert list(r["perm_num_max"]) == nums
    assert r["num_obs"] == orc.brute_force_ddks(P, T)[0]
    assert r["p_value"] == (1 + sum(n >= r["num_obs"] for n in nums)) / (1 + B)
    assert orc.permutation_test(P, T, 0, seed=7)["p_value"] == 1.0


# ---------------------------------------------------------------- significance
def test_cell_probability_against_scipy():
    st = pytest.importorskip("scipy.stats")
    for NP, NT, num, lam in [(5, 7, 6, 0.3), (4, 4, 0, 0.5), (9, 3, 10, 0.05), (6, 6, 36, 0.8)]:
        ref = 0.0
        for a in range(NP + 1):
            for b in range(NT + 1):
                if abs(a * NT - b * NP) <= num:
                    ref += st.binom.pmf(a, NP, lam) * st.binom.pmf(b, NT, lam)
        assert orc.cell_p_le(NP, NT, num, lam, 0) == pytest.approx(ref, rel=1e-12, abs=1e-15)
        refp = 0.0
        for a in range(NP + 1):
            for b in range(NT + 1):
                if abs(a * NT - b * NP) <= num:
                    refp += st.poisson.pmf(a, NP * lam) * st.poisson.pmf(b, NT * lam)
        assert orc.cell_p_le(NP, NT, num, lam, 1) == pytest.approx(refp, rel=1e-12, abs=1e-15)


def test_cell_probability_closed_forms():
    lam = 0.37
    # one point per sample, D = 0: both succeed or both fail
    assert orc.cell_p_le(1, 1, 0, lam, 0) == pytest.approx(lam**2 + (1 - lam) ** 2, rel=1e-14)
    # the largest possible difference is never exceeded
    assert orc.cell_p_le(7, 5, 35, lam, 0) == pytest.approx(1.0, rel=1e-13)
    assert orc.cell_p_le(7, 5, 0, 0.0, 0) == 1.0


def test_significance_against_direct_sum():
    st = pytest.importorskip("scipy.stats")
    P, T = wl.random_pair(3, 6, 5, 2, kind="int", dtype=np.float64)
    num = orc.ddks(P, T)["num_max"]
    S, lp = orc.significance(P, T, num, estimator=1, model=0)
    NP, NT, d = 6, 5, 2
    X = np.concatenate([P, T])
    acc = 0.0
    for o in X:
        for j in range(2 ** d):
            inside = lambda x: all((x[m] >= o[m]) == bool((j >> m) & 1) for m in range(d))
            mt = sum(1 for x in T if inside(x))
            lam = (mt + 1) / (NT + 2)
            p = sum(st.binom.pmf(a, NP, lam) * st.binom.pmf(b, NT, lam)
                    for a in range(NP + 1) for b in range(NT + 1) if abs(a * NT - b * NP) <= num)
            acc += np.log(p)
    assert lp == pytest.approx(acc, rel=1e-10)
    assert S == pytest.approx(1 - np.exp(acc), rel=1e-10, abs=1e-14)
    # at the largest possible D every cell probability is 1, so S = 0
    assert orc.significance(P, T, NP * NT)[0] == pytest.approx(0.0, abs=1e-12)
