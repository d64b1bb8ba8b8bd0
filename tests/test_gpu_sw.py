"""Swendsen-Wang update (Sec. 4.1 benchmark): CUDA path through the C ABI
against the CPU oracle.

Both sides start from the same seeded spins with the same seed and sweep.
Spins, the cluster name of every site and every integer of the record must
agree exactly; energy and chi are the same IEEE expression of those integers
on both sides and must agree exactly too.
"""
import math

import numpy as np
import pytest

from oracle import orc
from paper_1810_07485_gb300 import workloads

pytestmark = pytest.mark.gpu

KC = math.log(1.0 + math.sqrt(2.0)) / 2.0
INT_FIELDS = ("n_eq", "n_act", "n_clusters", "max_cluster", "sum_c2", "mag")


def gpu():
    from paper_1810_07485_gb300 import lcqmc
    return lcqmc


def assert_rec(rg, ro, ctx):
    for f in INT_FIELDS:
        assert int(rg[f]) == int(ro[f]), (ctx, f, int(rg[f]), int(ro[f]))
    for f in ("energy", "chi"):
        assert float(rg[f]) == float(ro[f]), (ctx, f, float(rg[f]), float(ro[f]))


def run_parity(L, K, seed, n, spins=None, roots_every=1, sweep0=0):
    lc = gpu()
    s = np.zeros(L * L, np.uint8) if spins is None else spins.copy()
    h = lc.SWIsing(L, K, seed=seed)
    try:
        if spins is not None or sweep0:
            h.set_spins(s, sweep0)
        for t in range(n):
            ro, roots_o, _ = orc.sw_update(L, K, seed, sweep0 + t, s, roots=(t % roots_every == 0))
            h.update(1)
            rg = h.records()
            assert len(rg) == 1 and int(rg[0]["sweep"]) == sweep0 + t
            ctx = f"L={L} K={K} sweep={sweep0 + t}"
            assert_rec(rg[0], ro, ctx)
            if roots_o is not None:
                assert np.array_equal(h.roots().astype(np.int64), roots_o), ctx
            assert np.array_equal(h.spins(), s), ctx
    finally:
        h.close()


# sizes: one partial tile, exactly one tile row, several tiles with ragged
# right and bottom edges, a lattice narrower than a tile; L = 2 has two bonds
# between each horizontal and vertical pair
CASES = [
    (2, 0.3), (3, KC), (5, 0.8), (17, KC), (32, 0.25), (64, KC), (65, KC), (100, 0.5),
    (130, KC), (257, KC), (96, 0.0), (96, 50.0),
]


@pytest.mark.parametrize("L,K", CASES)
def test_sw_parity_random_start(L, K):
    run_parity(L, K, seed=100 + L, n=6, spins=workloads.ising_spins(L, seed=L))


@pytest.mark.parametrize("L,K", [(64, KC), (100, 0.6), (300, KC)])
def test_sw_parity_ordered_start(L, K):
    run_parity(L, K, seed=7, n=6)


def test_sw_long_chain():
    # 300 chained updates at K_c: every record and the final spins agree.
    L, K, seed = 48, KC, 5
    lc = gpu()
    s = np.zeros(L * L, np.uint8)
    ro = orc.sw_run(L, K, seed, 0, 300, s)
    h = lc.SWIsing(L, K, seed=seed)
    h.update(300)
    rg = h.records()
    assert len(rg) == 300
    for t in range(300):
        assert_rec(rg[t], ro[t], t)
    assert np.array_equal(h.spins(), s)
    o = h.measure()
    assert o.n_updates == 300
    assert o.sum[0] == pytest.approx(ro["energy"].sum(), rel=1e-12)
    assert o.sum[1] == pytest.approx(ro["chi"].sum(), rel=1e-12)
    m = ro["mag"].astype(np.float64)
    assert o.sum[2] == pytest.approx((m * m / (L * L)).sum(), rel=1e-12)
    h.close()


def test_sw_sweep_offset_and_seed():
    run_parity(40, KC, seed=2**40 + 3, n=3, spins=workloads.ising_spins(40, 9), sweep0=1000)


def test_sw_full_size_kc():
    # The paper's lattice, L = 8192 at K_c, from the ordered and from a random
    # start: two updates each, compared in full (67M sites).
    L = 8192
    run_parity(L, KC, seed=1, n=2)
    run_parity(L, KC, seed=3, n=2, spins=workloads.ising_spins(L, seed=8192))


def test_sw_invalid_arguments():
    lc = gpu()
    for L, K in ((1, 0.4), (46341, 0.4), (8, -0.1), (8, float("nan")), (8, float("inf"))):
        with pytest.raises(lc.LcqmcError):
            lc.SWIsing(L, K)
    h = lc.SWIsing(8, KC)
    with pytest.raises(lc.LcqmcError):
        h.roots()  # no update yet
    bad = np.zeros(64, np.uint8)
    bad[3] = 2
    with pytest.raises(lc.LcqmcError):
        h.set_spins(bad)
    h.close()


def test_sw_phase_timing_and_ring():
    lc = gpu()
    h = lc.SWIsing(256, KC, seed=4)
    h.set_phase_timing(True)
    h.update(5)
    ph = h.phase_times()
    assert all(v > 0 for v in ph.values()), ph
    h.set_phase_timing(False)
    h.update(5000)  # more than the ring holds: the oldest records are dropped
    r = h.records(max_n=10000)
    assert len(r) == 4096 and int(r[-1]["sweep"]) == 5004 and int(r[0]["sweep"]) == 5004 - 4095
    h.close()
