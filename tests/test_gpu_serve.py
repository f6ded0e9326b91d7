"""Serving loop: requests of different N and d submitted while others run are
batched on the GPU; each result is the same as the request computed alone and
as the oracle's.  Host-side failure cases: oversized requests, bad arguments,
unknown tickets, bounded polls."""
import threading
import time

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


def _wait(c, tk, limit_s=60.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        rc, r = c.poll(tk, 20000)
        if rc == pkg.DDKS_OK:
            return r
    raise TimeoutError(tk)


def test_mixed_stream_alone_vs_mixed(torch):
    reqs = wl.serving_requests(seed=1, count=40, n_lo=30, n_hi=3000)
    with pkg.Context(device=0) as c:
        alone = [c.distance(P, T) for _, P, T in reqs]
        tickets = []

        def producer():
            t0 = time.time()
            for arr, P, T in reqs:
                # compressed arrival times: requests keep arriving while batches run
                dt = arr / 20.0 - (time.time() - t0)
                if dt > 0:
                    time.sleep(dt)
                tickets.append(c.submit(P, T))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        mixed = [_wait(c, tk) for tk in tickets]
        st = c.stats()
    assert st["submitted"] == st["completed"] == 40
    assert st["batches"] >= 2
    assert st["bytes_resident"] == 0
    for (_, P, T), a, m in zip(reqs, alone, mixed):
        assert _key(m) == _key(a)
    for i in range(0, 40, 7):
        _, P, T = reqs[i]
        assert _key(mixed[i]) == _key(orc.ddks(P, T))


def test_admission_budget_and_refusal(torch):
    P, T = wl.gaussian_pair(seed=2, n_p=3000, n_t=2000, d=3)
    with pkg.Context(device=0, hbm_budget_bytes=2_000_000, max_batch=4) as c:
        # larger than the whole budget: refused at submit
        big_P, big_T = wl.gaussian_pair(seed=3, n_p=20000, n_t=20000, d=4)
        with pytest.raises(pkg.DdksError) as e:
            c.submit(big_P, big_T)
        assert e.value.code == -4
        # each fits alone but not all at once: they queue and all complete
        tks = [c.submit(P, T) for _ in range(6)]
        res = [_wait(c, t) for t in tks]
        st = c.stats()
        assert st["rejected"] == 1 and st["completed"] == 6
        assert st["bytes_resident_peak"] <= 2_000_000
    ref = orc.ddks(P, T)
    assert all(_key(r) == _key(ref) for r in res)


def test_bad_requests_and_tickets(torch):
    with pkg.Context(device=0) as c:
        with pytest.raises(pkg.DdksError) as e:
            c.submit(np.zeros((3, 31), np.float32), np.zeros((3, 31), np.float32))
        assert e.value.code == -1
        with pytest.raises(pkg.DdksError) as e:
            c.poll(12345, 0)
        assert e.value.code == -7
        P, T = wl.random_pair(4, 100, 80, 2)
        bad = P.copy()
        bad[5, 1] = np.nan
        tk_bad = c.submit(bad, T)
        tk_ok = c.submit(P, T)
        t0 = time.time()
        while True:
            try:
                rc, r = c.poll(tk_bad, 20000)
            except pkg.DdksError as err:
                assert err.code == -2
                break
            assert time.time() - t0 < 60
        assert _key(_wait(c, tk_ok)) == _key(orc.ddks(P, T))
        # a result is released once read
        with pytest.raises(pkg.DdksError):
            c.poll(tk_ok, 0)


def test_poll_without_wait_and_shutdown_with_queue(torch):
    P, T = wl.gaussian_pair(seed=5, n_p=8000, n_t=8000, d=4)
    c = pkg.Context(device=0)
    tks = [c.submit(P, T) for _ in range(8)]
    rc, r = c.poll(tks[-1], 0)
    assert rc in (pkg.DDKS_OK, pkg.DDKS_PENDING)
    c.close()  # joins the workers with requests possibly still queued


def test_submit_inputs_reusable_on_return(torch):
    # submit returns before the device copy of pageable host inputs has
    # landed (the worker waits on an event); the caller may still overwrite
    # its buffers at once: every result must be that of the original data
    rng = np.random.default_rng(12)
    probs = [wl.random_pair(70 + i, int(rng.integers(50, 3000)), int(rng.integers(50, 3000)), 2 + i % 3)
             for i in range(12)]
    refs = [orc.ddks(P, T) for P, T in probs]
    with pkg.Context(device=0, max_batch=8) as c:
        tickets = []
        for P, T in probs:
            Pb, Tb = P.copy(), T.copy()
            tickets.append(c.submit(Pb, Tb))
            Pb[:] = 1e6  # reused by the caller right after submit
            Tb[:] = -1e6
            del Pb, Tb
        for tk, ref in zip(tickets, refs):
            rc, r = c.poll(tk, 10_000_000)
            assert rc == pkg.DDKS_OK
            assert (r["num_max"], r["argmax_origin"], r["argmax_orthant"]) == (
                ref["num_max"], ref["argmax_origin"], ref["argmax_orthant"])
