"""Bounded device-side waits: a wait that runs out reports DDKS_ETIMEOUT, the
CTA drains its own copies in flight, and the same context then computes
bit-exact results.  Nothing here faults, traps or hangs a GPU: the self-test
waits on a phase that simply never completes, and the streamed kernels are
given a wait bound short enough to run out while their copies still land."""
import numpy as np
import pytest

import paper_2106_13706_gb300 as pkg
from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ETIMEOUT = -6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2106_13706_gb300 import build as b
    b.build()
    return t


def _dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _exact(got, ref):
    assert (got["num_max"], got["denom"]) == (ref["num_max"], ref["denom"])
    assert (got["argmax_origin"], got["argmax_orthant"]) == (ref["argmax_origin"], ref["argmax_orthant"])


def test_wait_selftest_times_out_then_context_is_usable(torch):
    P, T = wl.gaussian_pair(seed=0, n_p=200, n_t=200, d=3)
    ref = orc.ddks(P, T)
    with pkg.Context(device=0) as c:
        c.set_device_wait_limit(1_000_000)  # 1 ms
        for _ in range(2):
            rc, waited = c.wait_selftest()
            assert rc == ETIMEOUT
            assert 1_000_000 <= waited < 1_000_000_000, waited
        c.set_device_wait_limit(0)
        _exact(c.distance(_dev(torch, P), _dev(torch, T)), ref)


def test_config_wait_limit_reaches_the_device(torch):
    with pkg.Context(device=0, wait_limit_ms=2) as c:
        rc, waited = c.wait_selftest()
        assert rc == ETIMEOUT and 2_000_000 <= waited < 1_000_000_000, waited


def _ok_or_timeout(fn):
    try:
        return fn()
    except pkg.DdksError as e:
        assert e.code == ETIMEOUT, e
        return None


@pytest.mark.parametrize("d,n", [(4, 6000), (3, 20000)])
def test_register_path_with_a_one_ns_bound(torch, d, n):
    # the count kernel streams its bit planes by bulk copies; with a 1 ns
    # bound most waits give up, and each CTA drains its copies before exiting
    rng = np.random.default_rng(d * 1000 + n)
    P = rng.standard_normal((n, d)).astype(np.float32)
    T = (rng.standard_normal((n + 37, d)) + 0.1).astype(np.float32)
    ref = orc.ddks(P, T)
    with pkg.Context(device=0, path=pkg.PATH_REGISTER, graphs=False) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        c.set_device_wait_limit(1)
        for _ in range(3):
            got = _ok_or_timeout(lambda: c.distance(Pd, Td))
            if got is not None:
                _exact(got, ref)
        c.set_device_wait_limit(0)
        for _ in range(2):
            _exact(c.distance(Pd, Td), ref)


def test_vdks_voxel_pass_with_a_one_ns_bound(torch):
    P, T = wl.gaussian_pair(seed=3, n_p=300000, n_t=300000, d=3)
    ref = orc.vdks(P, T, 16)
    with pkg.Context(device=0, graphs=False) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        c.set_device_wait_limit(1)
        got = _ok_or_timeout(lambda: c.vdks(Pd, Td, 16))
        if got is not None:
            assert got["num_max"] == ref["num_max"]
        c.set_device_wait_limit(0)
        assert c.vdks(Pd, Td, 16)["num_max"] == ref["num_max"]
