"""Served form: continuous batching of independent chains.

A mix of requests (S=1/2 and S=1, different sizes, temperatures and update
counts) submitted together, with fewer slots than requests so that chains
join and leave between ticks, must give every request exactly the result of
the same chain run alone, and the result of the CPU oracle's chain with the
same parameters and seed."""
import time

import numpy as np
import pytest

from oracle import orc

pytestmark = pytest.mark.gpu

MIX = [dict(L=8, beta=4.0, S=0.5, seed=1, n=17), dict(L=64, beta=30.0, S=0.5, seed=2, n=12),
       dict(L=6, beta=2.0, S=1.0, seed=3, n=25), dict(L=200, beta=9.0, S=0.5, seed=4, n=8),
       dict(L=32, beta=48.0, S=1.0, seed=5, n=11), dict(L=10, beta=0.01, S=0.5, seed=6, n=30),
       dict(L=130, beta=70.0, S=0.5, seed=7, n=14), dict(L=2, beta=5.0, S=1.0, seed=8, n=9)]


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.005)
    return out


def _check_against_oracle(r, m):
    # the oracle's chain: the same records, summed in update order
    p = orc.params(m["L"], m["beta"], Q=int(2 * m["S"]), seed=m["seed"])
    recs = orc.keyed_run(p, 0, m["n"], orc.neel(p))
    fields = ("energy", "chi_s", "chi_q", "n", "n_off_new", "n_seg", "n_clusters", None)
    for k, f in enumerate(fields):
        v = [float(x) for x in (recs["n_seg"] + 2 * recs["n"] if f is None else recs[f])]
        s1 = s2 = 0.0
        for x in v:
            s1 += x
            s2 += x * x
        if f in ("energy", "chi_s", "chi_q"):  # fp64 from exact sums; 1e-15 per record
            assert r.obs.sum[k] == pytest.approx(s1, rel=1e-13, abs=1e-300), (m, f)
            assert r.obs.sumsq[k] == pytest.approx(s2, rel=1e-13, abs=1e-300), (m, f)
        else:  # integers, exact in fp64
            assert r.obs.sum[k] == s1 and r.obs.sumsq[k] == s2, (m, f)


def test_mix_equals_alone():
    from paper_1810_07485_gb300 import lcqmc
    srv = lcqmc.Server(hbm_budget=8 << 30, max_slots=3)
    tickets = [srv.submit(m["L"], m["beta"], m["n"], S=m["S"], seed=m["seed"]) for m in MIX]
    res = _wait(srv, tickets)
    srv.close()
    for m, t in zip(MIX, tickets):
        r = res[t]
        assert r.status == 0
        assert r.obs.n_updates == m["n"]
        assert r.t_submit <= r.t_admit <= r.t_done
        ch = lcqmc.Chain(m["L"], m["beta"], S=m["S"], seed=m["seed"])
        ch.update(m["n"])
        o = ch.measure()
        assert list(r.obs.sum) == list(o.sum), m
        assert list(r.obs.sumsq) == list(o.sumsq), m
        assert r.vertices_edges == int(o.sum[7])
        ch.close()
        _check_against_oracle(r, m)


def test_admission_rejects_oversized_and_cancels():
    from paper_1810_07485_gb300 import lcqmc
    srv = lcqmc.Server(hbm_budget=64 << 20, max_slots=1)
    with pytest.raises(lcqmc.LcqmcError) as e:
        srv.submit(4096, 4096.0, 5)
    assert e.value.code == -3  # E_TOO_LARGE
    a = srv.submit(256, 64.0, 200, seed=1)
    b = srv.submit(16, 4.0, 5, seed=2)  # waits for the only slot
    srv.cancel(b)
    res = _wait(srv, [a, b])
    assert res[a].status == 0 and res[b].status == -9  # E_CANCELLED
    srv.close()


def test_failing_chain_fails_only_its_request(monkeypatch):
    # One resident chain's bounded wait runs out: the tick is run again chain
    # by chain, that chain's request fails with LCQMC_E_DEVICE_TIMEOUT and
    # the others finish with the oracle's results.  Tiles above 64 vertices
    # unite their edges in the global forest, whose walks get a bound of one
    # step; the small chains (one tile of a few vertices) never walk it.
    monkeypatch.setenv("LCQMC_LOCAL_CAP", "64")
    monkeypatch.setenv("LCQMC_WAIT_LIMIT", "1")
    from paper_1810_07485_gb300 import lcqmc
    # the small chains run 200 updates (at least 20 ticks), so they are still
    # resident when the large one joins and fails
    small = [dict(L=8, beta=0.5, S=0.5, seed=11, n=200), dict(L=4, beta=1.0, S=0.5, seed=12, n=210),
             dict(L=2, beta=0.5, S=1.0, seed=13, n=205)]
    big = dict(L=1024, beta=40.0, S=0.5, seed=9, n=6)
    srv = lcqmc.Server(hbm_budget=8 << 30, max_slots=4)
    tickets = [srv.submit(m["L"], m["beta"], m["n"], S=m["S"], seed=m["seed"]) for m in small + [big]]
    res = _wait(srv, tickets)
    srv.close()
    assert res[tickets[-1]].status == -5  # LCQMC_E_DEVICE_TIMEOUT
    for m, t in zip(small, tickets):
        r = res[t]
        assert r.status == 0, (m, r.status)
        assert r.obs.n_updates == m["n"]
        _check_against_oracle(r, m)
