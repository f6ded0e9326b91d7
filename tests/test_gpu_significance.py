"""Analytic significance (Sec. 3, Eq. ddks_significance) on the GPU against the
oracle's direct double sum.

Tolerance: both sides work in float64.  The oracle sums the pmf products of
every admissible (nP, nT) pair directly, so each cell probability p carries a
rounding error of up to about (NP+1)(NT+1) * 2^-53 absolute, and log(p) the
same absolute error (p is close to 1).  The kernel sums pmf(nP) times the T
mass outside the admissible interval and takes log1p of minus that mass, which
is more accurate near p = 1.  The log of the product adds N * 2^d cells, so the
test allows  N * 2^d * (NP+1) * (NT+1) * 2^-52  absolute on log(prod) (and on
S = 1 - exp(log prod)), plus 1e-12 relative.
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


def _cmp(torch, P, T, est, model, num=None):
    if num is None:
        num = orc.ddks(P, T)["num_max"]
    S_ref, lp_ref = orc.significance(P, T, num, estimator=est, model=model)
    with pkg.Context(device=0) as c:
        S, lp = c.significance(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), num,
                               estimator=est, model=model)
    NP, d = P.shape
    NT = T.shape[0]
    tol = (NP + NT) * 2 ** d * (NP + 1) * (NT + 1) * 2.0 ** -52
    assert lp == pytest.approx(lp_ref, rel=1e-12, abs=tol)
    assert S == pytest.approx(S_ref, rel=1e-12, abs=tol)
    return S


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("est,model", [(1, 0), (0, 0), (1, 1)])
def test_small(torch, d, est, model):
    P, T = wl.random_pair(10 + d, 17, 23, d, kind="int")
    _cmp(torch, P, T, est, model)
    P, T = wl.random_pair(20 + d, 40, 31, d, kind="normal", dtype=np.float64)
    _cmp(torch, P, T, est, model)


def test_extremes(torch):
    P, T = wl.random_pair(1, 12, 9, 2)
    # the largest possible statistic: every cell probability is 1
    assert _cmp(torch, P, T, 1, 0, num=12 * 9) == pytest.approx(0.0, abs=1e-12)
    # statistic 0: only exact ties in every cell count as "as or less extreme"
    _cmp(torch, P, T, 1, 0, num=0)


def test_config1(torch):
    P, T = wl.CONFIGS["cfg1_d3_200x200_f32"]()
    S = _cmp(torch, P, T, 1, 0)
    assert 0.0 <= S <= 1.0


def test_rejects_unsupported(torch):
    P = np.zeros((5, 14), np.float32)
    with pkg.Context(device=0) as c:
        with pytest.raises(pkg.DdksError) as e:
            c.significance(torch.from_numpy(P).cuda(), torch.from_numpy(P).cuda(), 0)
        assert e.value.code == -8


def test_analytic_significance_and_permutation_p_agree_in_direction(torch):
    # Sec. 3 compares the analytic significance with the permutation test on
    # DVU in 3 dimensions (type I with both samples diagonal, power with
    # diagonal versus uniform, 50 points per sample).  Over 20 seeds: under
    # the alternative both reject at alpha = 0.05 every time; under the null
    # S never rejects (the product over cells treats correlated cells as
    # independent, which makes S conservative) and the permutation p rejects
    # at most a quarter of the time (its type I rate is alpha).
    alpha, seeds = 0.05, 20
    with pkg.Context(device=0) as c:
        for hyp in ("null", "alt"):
            rej_S = rej_p = 0
            for s in range(seeds):
                P, T = (wl.dvu_null_pair if hyp == "null" else wl.dvu_pair)(s, 50, 50, 3)
                Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
                pr = c.permutation_test(Pd, Td, 1000, 500 + s, want_perm=False)
                S, _ = c.significance(Pd, Td, pr["observed"]["num_max"], 1, 0)
                rej_S += S < alpha
                rej_p += pr["p_value"] < alpha
            if hyp == "alt":
                assert rej_S == seeds and rej_p == seeds
            else:
                assert rej_S == 0 and rej_p <= seeds // 4
