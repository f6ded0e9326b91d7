"""The bit-sliced relabelling counter (N up to about 4000, d <= 5) against the
oracle: every relabelling's numerator, across pass boundaries (B not a
multiple of 256), bins of every size and all-equal inputs."""
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


@pytest.mark.parametrize("d,n_p,n_t,B", [(1, 40, 50, 300), (2, 700, 600, 513), (3, 1200, 900, 257),
                                         (4, 2000, 1999, 64), (5, 333, 777, 1000)])
def test_bits_match_oracle(torch, d, n_p, n_t, B):
    P, T = wl.random_pair(d * 7 + 1, n_p, n_t, d, kind="normal")
    ref = orc.permutation_test(P, T, B, seed=d)
    with pkg.Context(device=0) as c:
        got = c.permutation_test(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), B, d)
    assert np.array_equal(got["perm_num_max"], ref["perm_num_max"])
    assert got["p_value"] == ref["p_value"]


def test_bits_ties_and_constants(torch):
    P, T = wl.random_pair(3, 300, 200, 3, kind="int")
    ref = orc.permutation_test(P, T, 100, seed=4)
    with pkg.Context(device=0) as c:
        got = c.permutation_test(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), 100, 4)
    assert np.array_equal(got["perm_num_max"], ref["perm_num_max"])
    P, T = wl.random_pair(3, 100, 60, 2, kind="const")
    with pkg.Context(device=0) as c:
        got = c.permutation_test(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), 40, 4)
    assert np.all(got["perm_num_max"] == 0) and got["p_value"] == 1.0
