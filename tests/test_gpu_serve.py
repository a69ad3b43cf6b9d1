"""Continuously batched impurity-solve service.

A served solve must be bit-for-bit the solve the context path computes for the same site,
chains, seed and bath (the context path is checked against the oracle elsewhere), warm starts
included, and must not depend on which other requests shared its launch; admission must respect
the device memory it was given.
"""
import numpy as np
import pytest

from paper_1006_2716_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1006_2716_gb300 import build as B

    B.build()
    from paper_1006_2716_gb300 import hf as H

    return H


def _params(hf, **over):
    p = hf.hf_srv_params()
    d = dict(chains_per_request=8, n_warmup=10, n_measure=40, refresh_every=10, bin_size=10,
             precision=2, team_warps=0, max_L=64, max_inflight=64, max_keys=256, n_streams=4,
             requests_per_launch=16)
    d.update(over)
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _req(hf, run, site, L, seed=99, U=8.0):
    beta = 0.25 * L
    bath = wl.random_baths(1000 * run + site, 1, beta, L)[0]
    return hf.make_request(run, site, L, beta, U, seed + run, bath), bath


def test_same_result_alone_and_in_the_mix(hf):
    x, _ = _req(hf, 0, 7, 40)
    a = hf.Server(_params(hf))
    ra = hf.hf_srv_wait(a.handle, hf.hf_srv_submit(a.handle, x))
    a.close()
    b = hf.Server(_params(hf))
    tickets = []
    for k in range(30):
        r, _ = _req(hf, 1 + k % 3, k, (32, 40, 64)[k % 3])
        tickets.append(hf.hf_srv_submit(b.handle, r))
        if k == 13:
            tx = hf.hf_srv_submit(b.handle, x)
    rb = hf.hf_srv_wait(b.handle, tx)
    for t in tickets:
        assert hf.hf_srv_wait(b.handle, t)["status"] == 0
    st = hf.hf_srv_stats(b.handle)
    assert st["peak_inflight"] > 1          # the mix really shared the device
    b.close()
    for k in ("gtau", "n", "err"):
        assert np.array_equal(ra[k], rb[k])
    assert ra["d"] == rb["d"] and ra["m"] == rb["m"] and ra["warm"] == rb["warm"] == 0


@pytest.mark.parametrize("precision,L,stagger", [(0, 32, 0), (2, 32, 0), (0, 32, 1), (2, 64, 1)])
def test_served_solve_equals_context_path_with_warm_start(hf, precision, L, stagger):
    cps, nw, nm, bs, seed, site = 8, 10, 40, 10, 123, 0
    beta = 0.25 * L
    srv = hf.Server(_params(hf, precision=precision, chains_per_request=cps, n_warmup=nw,
                            n_measure=nm, bin_size=bs, refresh_stagger=stagger))
    cfg = dict(wl.CONFIGS["square6"], Lx=1, Ly=1, beta=beta, dtau=0.25, U=8.0, precision=precision,
               chains_per_site=cps, bin_size=bs, max_bins=nm // bs, seed=seed, n_matsubara=4,
               refresh_stagger=stagger)
    ctx = hf.Context(hf.make_params(cfg))
    for it in range(2):                      # cold start, then warm start with a new bath
        bath = wl.random_baths(50 + it, 1, beta, L)[0]
        r = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(
            srv.handle, hf.make_request(3, site, L, beta, 8.0, seed, bath)))
        hf.hf_set_g0(ctx.handle, 0, 0, bath[0])
        hf.hf_set_g0(ctx.handle, 0, 1, bath[1])
        hf.hf_clear_measurements(ctx.handle)
        hf.hf_sweep(ctx.handle, nw, nm, 1)
        gtau, n, d, m, errs = hf.hf_measure(ctx.handle, 0, L)
        assert r["warm"] == it
        assert r["sweeps_done"] == (it + 1) * (nw + nm)
        assert np.array_equal(r["gtau"].ravel(), gtau)
        assert np.array_equal(r["n"], n) and r["d"] == d and r["m"] == m
        assert np.array_equal(r["err"], errs)
    ctx.close()
    srv.close()


def test_admission_limited_by_device_memory(hf):
    p = _params(hf, max_inflight=3, n_streams=8, requests_per_launch=2)
    srv = hf.Server(p)                       # pool sized for 3 requests at L = 64
    tickets = [hf.hf_srv_submit(srv.handle, _req(hf, 5, k, 64)[0]) for k in range(10)]
    for t in tickets:
        assert hf.hf_srv_wait(srv.handle, t)["status"] == 0
    st = hf.hf_srv_stats(srv.handle)
    assert st["completed"] == 10 and st["queued"] == 0 and st["inflight"] == 0
    assert 1 <= st["peak_inflight"] <= 3
    assert 0 < st["peak_bytes"] <= st["arena_bytes"]
    srv.close()


def test_warm_keys_evicted_least_recently_used(hf):
    srv = hf.Server(_params(hf, max_keys=2))
    res = []
    for site in (1, 2, 3, 1):                # the 4th request's key was evicted by site 3
        res.append(hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, _req(hf, 0, site, 32)[0])))
    assert [r["warm"] for r in res] == [0, 0, 0, 0]
    r = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, _req(hf, 0, 1, 32)[0]))
    assert r["warm"] == 1                    # site 1 is resident again
    srv.close()


def test_invalid_requests_rejected(hf):
    srv = hf.Server(_params(hf, max_L=32))
    r, _ = _req(hf, 0, 0, 64)
    with pytest.raises(hf.HFError) as e:
        hf.hf_srv_submit(srv.handle, r)
    assert e.value.status == hf.HF_EINVAL
    with pytest.raises(hf.HFError):
        hf.hf_srv_poll(srv.handle, 12345)
    srv.close()


def test_key_with_a_new_L_starts_cold(hf):
    # fields kept for a key at one L are not a state of chains at another L: a request of the
    # same (run, site) with a different L starts cold, and its own fields become the kept ones
    srv = hf.Server(_params(hf, precision=0))
    r16, _ = _req(hf, 3, 5, 16)
    r32, _ = _req(hf, 3, 5, 32)
    first = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, r16))
    assert first["status"] == hf.HF_OK and first["warm"] == 0
    again16 = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, r16))
    assert again16["warm"] == 1
    switched = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, r32))
    assert switched["status"] == hf.HF_OK and switched["warm"] == 0
    # a cold L = 32 solve of this key is the solve of a fresh service
    fresh = hf.Server(_params(hf, precision=0))
    ref = hf.hf_srv_wait(fresh.handle, hf.hf_srv_submit(fresh.handle, r32))
    fresh.close()
    assert np.array_equal(switched["gtau"], ref["gtau"]) and switched["d"] == ref["d"]
    again32 = hf.hf_srv_wait(srv.handle, hf.hf_srv_submit(srv.handle, r32))
    assert again32["warm"] == 1
    srv.close()
