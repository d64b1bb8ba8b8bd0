"""Parity of the CUDA update (through the C ABI) with the CPU oracle.

Both sides start from the same state with the same seed and sweep; every
integer output (vertex list, predecessor links, loop roots, new spins and
operators, counts, 128-bit loop sums) must agree exactly, and so must the
fp64 imaginary times, which both sides compute with one IEEE rounding per
operation.  The floating-point estimators are derived from the exact sums by
the same expression on both sides and must agree to 1e-15 relative.
"""
import numpy as np
import pytest

from oracle import ed, orc, stats

pytestmark = pytest.mark.gpu

REL_TOL = 1e-15


def gpu():
    from paper_1810_07485_gb300 import lcqmc
    return lcqmc


def gpu_state(ch):
    s0, ptr, tau = ch.export_config()
    return orc.State(s0, ptr.astype(np.int64), tau)


def assert_records_equal(rg, ro, ctx=""):
    for f in ("n", "n_off_old", "n_off_new", "n_free", "n_clusters", "n_seg", "F", "sw2_lo",
              "sw2_hi", "sf2_lo", "sf2_hi", "sz2_lo", "sz2_hi"):
        assert int(rg[f]) == int(ro[f]), (ctx, f, int(rg[f]), int(ro[f]))
    for f in ("energy", "chi_s", "chi_q", "chi_w"):
        a, b = float(rg[f]), float(ro[f])
        assert abs(a - b) <= REL_TOL * max(abs(a), abs(b), 1e-300), (ctx, f, a, b)


def assert_graph_equal(gg, go, ctx=""):
    assert np.array_equal(gg["tau"], go["tau"]), ctx
    assert np.array_equal(gg["flag"], go["flag"]), ctx
    assert np.array_equal(gg["pl"].astype(np.int64), go["pl"]), ctx
    assert np.array_equal(gg["pr"].astype(np.int64), go["pr"]), ctx
    assert np.array_equal(gg["root"].astype(np.int64), go["root"]), ctx


def assert_state_equal(sg, so, ctx=""):
    assert np.array_equal(sg.s0, so.s0), ctx
    assert np.array_equal(sg.op_ptr, so.op_ptr), ctx
    assert np.array_equal(sg.op_tau, so.op_tau), ctx


def run_parity(L, beta, Q=1, J=1.0, seed=1, nup=12, graph_every=1):
    lc = gpu()
    p = orc.params(L, beta, J=J, Q=Q, seed=seed)
    st = orc.neel(p)
    ch = lc.Chain(L, beta, S=Q / 2, J=J, seed=seed)
    ch.set_temporal(True)
    try:
        for t in range(nup):
            new, ro, go = orc.keyed_update(p, t, st, graph=(t % graph_every == 0))
            ch.update(1)
            rg = ch.records()
            assert len(rg) == 1
            ctx = f"L={L} beta={beta} Q={Q} J={J} sweep={t}"
            assert_records_equal(rg[0], ro, ctx)
            if go is not None:
                assert_graph_equal(ch.export_graph(), go, ctx)
            assert_state_equal(gpu_state(ch), new, ctx)
            st = new
        return st
    finally:
        ch.close()


# (L, beta, Q, J): window edges, partial last window and time block, tiny and
# empty chains, several tiles with a ragged tail, two-site chains, S=1.
CASES = [
    (2, 3.0, 1, 1.0),
    (2, 200.0, 1, 1.0),      # 13 windows: time blocks 4+4+4+1
    (4, 16.0, 1, 1.0),       # exactly one full window
    (8, 16.0000001, 1, 1.0), # a sliver of a last window
    (8, 15.99, 1, 1.0),
    (16, 5.0, 1, 0.37),      # J != 1: window width 16/J
    (64, 16.0, 1, 1.0),
    (250, 70.0, 1, 1.0),     # 1250 cells: 9 full tiles + a ragged one
    (1024, 40.0, 1, 1.0),    # 96 tiles
    (4, 3.0, 2, 1.0),
    (2, 10.0, 2, 1.0),
    (16, 20.0, 2, 1.0),
    (64, 8.0, 2, 0.5),
    (4, 3.0, 3, 1.0),        # S = 3/2: 9 sub-bonds per bond, shuffled tau = 0 joins
    (6, 5.0, 3, 1.0),
    (34, 10.0, 3, 1.0),      # 306 cells: 3 tiles
    (2, 4.0, 4, 1.0),        # S = 2
    (8, 6.0, 4, 0.7),
    (20, 40.0, 4, 1.0),      # 960 cells: 8 tiles
]


@pytest.mark.parametrize("L,beta,Q,J", CASES)
def test_update_parity(L, beta, Q, J):
    run_parity(L, beta, Q=Q, J=J, seed=1000 + L, nup=10)


@pytest.mark.parametrize("L,beta,Q", [(250, 70.0, 1), (1024, 40.0, 1), (16, 20.0, 2)])
def test_update_parity_grouped_insertion(monkeypatch, L, beta, Q):
    # Candidate staging in groups of 256 slots: every tile (about 1024
    # candidates) counts group by group, then draws each group again to write.
    monkeypatch.setenv("LCQMC_INSERT_GROUP_SLOTS", "256")
    run_parity(L, beta, Q=Q, seed=77 + L, nup=6)


def test_long_run_parity():
    # 300 chained updates: states stay identical throughout.
    run_parity(32, 24.0, nup=300, graph_every=50, seed=5)


def test_empty_and_tiny_beta():
    # beta << 1/J: most updates have no vertex at all (every site a free loop).
    lc = gpu()
    p = orc.params(16, 1e-6, seed=3)
    st = orc.neel(p)
    ch = lc.Chain(16, 1e-6, seed=3)
    ch.set_temporal(True)
    orc_recs = orc.keyed_run(p, 0, 40, st)
    ch.update(40)
    rg = ch.records()
    for a, b in zip(rg, orc_recs):
        assert_records_equal(a, b)
    assert (rg["n"] == 0).sum() > 30
    assert_state_equal(gpu_state(ch), st)


def test_import_thermalized_state():
    # A state thermalized by the oracle is imported; the next updates agree.
    lc = gpu()
    L, beta = 48, 30.0
    p = orc.params(L, beta, seed=11)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 40, st)
    ch = lc.Chain(L, beta, seed=11)
    ch.set_temporal(True)
    ch.import_config(st.s0, st.op_ptr.astype(np.int32), st.op_tau, 40)
    assert_state_equal(gpu_state(ch), st)
    for t in range(40, 50):
        new, ro, go = orc.keyed_update(p, t, st, graph=True)
        ch.update(1)
        assert_records_equal(ch.records()[0], ro)
        assert_graph_equal(ch.export_graph(), go)
        st = new
    assert_state_equal(gpu_state(ch), st)


def test_import_rejects_invalid_state():
    lc = gpu()
    p = orc.params(8, 10.0, seed=2)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 5, st)
    ch = lc.Chain(8, 10.0, seed=2)
    bad = st.s0.copy()
    bad[0] ^= 1  # breaks periodicity / antiparallel constraint
    with pytest.raises(lc.LcqmcError):
        ch.import_config(bad, st.op_ptr.astype(np.int32), st.op_tau, 0)


def test_checkpoint_restore_bit_exact():
    lc = gpu()
    a = lc.Chain(40, 12.0, seed=9)
    a.update(20)
    blob = a.checkpoint()
    a.update(15)
    ra = a.records()[-15:]
    b = lc.Chain(40, 12.0, seed=9)
    b.restore(blob)
    b.update(15)
    rb = b.records()
    assert np.array_equal(ra, rb)
    sa, sb = gpu_state(a), gpu_state(b)
    assert_state_equal(sa, sb)


def test_update_paths_identical():
    # The graph of eight updates, the one-update graph and the direct launches
    # of the phase-timed path give the same records and state: 21 updates as
    # one call (two blocks of eight and five single graphs), one by one, and
    # timed.
    lc = gpu()
    chains = [lc.Chain(300, 40.0, seed=12) for _ in range(3)]
    chains[0].update(21)
    for _ in range(21):
        chains[1].update(1)
    chains[2].set_phase_timing(True)
    chains[2].update(21)
    recs = [c.records() for c in chains]
    assert len(recs[0]) == 21
    for r in recs[1:]:
        assert np.array_equal(recs[0], r)
    s0 = gpu_state(chains[0])
    for c in chains[1:]:
        assert_state_equal(gpu_state(c), s0)
    p = orc.params(300, 40.0, seed=12)
    st = orc.neel(p)
    ro = orc.keyed_run(p, 0, 21, st)
    # the temporal moment is off (sz2 and chi_w are 0 on the device)
    for f in ("n", "n_off_old", "n_off_new", "n_free", "n_clusters", "n_seg", "F", "sw2_lo", "sw2_hi",
              "sf2_lo", "sf2_hi"):
        assert np.array_equal(recs[0][f].astype(np.int64), ro[f].astype(np.int64)), f
    for f in ("energy", "chi_s", "chi_q"):
        assert np.allclose(recs[0][f], ro[f], rtol=REL_TOL, atol=0), f
    assert_state_equal(s0, st)


def test_capacity_growth_replays_identically():
    # A chain started from a hot state needs more room than the first estimate
    # at low temperature for S=1; growth replays the update with the same keys.
    lc = gpu()
    p = orc.params(12, 60.0, Q=2, seed=4)
    st = orc.neel(p)
    recs = orc.keyed_run(p, 0, 30, st)
    ch = lc.Chain(12, 60.0, S=1.0, seed=4)
    ch.set_temporal(True)
    ch.update(30)
    rg = ch.records()
    for a, b in zip(rg, recs):
        assert_records_equal(a, b)
    assert_state_equal(gpu_state(ch), st)


def test_records_and_measure_consistent():
    lc = gpu()
    ch = lc.Chain(16, 8.0, seed=21)
    ch.set_temporal(True)
    ch.update(100)
    r = ch.records()
    o = ch.measure()
    assert o.n_updates == 100
    assert o.sum[0] == pytest.approx(r["energy"].sum(), rel=1e-12)
    assert o.sum[1] == pytest.approx(r["chi_s"].sum(), rel=1e-12)
    assert o.sum[3] == pytest.approx(r["n"].sum(), rel=1e-12)
    assert o.sum[8] == pytest.approx(r["chi_w"].sum(), rel=1e-12)
    # imaginary-time second moment and the gap derived from the means
    xt = 8.0 / (2 * np.pi) * np.sqrt(r["chi_s"].mean() / r["chi_w"].mean() - 1)
    assert o.xi_tau == pytest.approx(xt, rel=1e-10)
    assert o.gap == pytest.approx(1 / xt, rel=1e-10)


# beta = 16 at L = 8 and 12 is the low-temperature point of the L = 64,
# beta = 16 accuracy configuration, at sizes exact diagonalization reaches.
@pytest.mark.parametrize("L,beta,Q", [(8, 4.0, 1), (12, 1.0, 1), (8, 16.0, 1), (12, 16.0, 1), (12, 4.0, 1),
                                      (4, 1.0, 2), (4, 0.7, 3), (2, 0.8, 4), (4, 0.5, 4)])
def test_gpu_vs_ed(L, beta, Q):
    # Estimators within 3 standard errors of exact diagonalization.
    lc = gpu()
    ch = lc.Chain(L, beta, S=Q / 2, seed=77)
    ch.set_temporal(True)
    ch.update(1000)
    ch.records()
    parts = []
    for _ in range(50):
        ch.update(4000)
        parts.append(ch.records())
    r = np.concatenate(parts)
    ex = ed.thermal(L, beta, S=Q / 2)
    for name in ("energy", "chi_s", "chi_q", "chi_w"):
        m, e = stats.mean_err(r[name], 100)
        assert stats.within_sigma(m, e, ex[name], 3.0), (name, m, e, ex[name])


def test_batch_matches_single_chains():
    # Chains updated together in one batch give the same records as alone.
    lc = gpu()
    specs = [dict(L=8, beta=4.0, seed=1), dict(L=34, beta=51.0, seed=2), dict(L=4, beta=2.0, S=1.0, seed=3),
             dict(L=128, beta=16.0, seed=4), dict(L=10, beta=0.001, seed=5), dict(L=6, beta=5.0, S=1.5, seed=6),
             dict(L=10, beta=12.0, S=2.0, seed=7)]
    b = lc.Batch(specs)
    b.update(25)
    for i, s in enumerate(specs):
        ch = lc.Chain(s["L"], s["beta"], S=s.get("S", 0.5), seed=s["seed"])
        ch.update(25)
        assert np.array_equal(b.records(i), ch.records()), i


def test_temporal_switch_leaves_standard_results_unchanged():
    # The temporal moment is measured only when switched on; with it off the
    # record's sz2 and chi_w are 0 and every other field and the state are
    # bit-identical.  Switching mid-run takes effect at the next update.
    lc = gpu()
    a = lc.Chain(96, 30.0, seed=13)
    b = lc.Chain(96, 30.0, seed=13)
    b.set_temporal(True)
    a.update(8)
    b.update(8)
    a.set_temporal(True)   # on from update 8
    b.set_temporal(False)  # off from update 8
    a.update(4)
    b.update(4)
    ra, rb = a.records(), b.records()
    std = [f for f in ra.dtype.names if f not in ("sz2_lo", "sz2_hi", "chi_w")]
    for f in std:
        assert np.array_equal(ra[f], rb[f]), f
    assert (ra["chi_w"][:8] == 0).all() and (ra["sz2_lo"][:8] == 0).all() and (ra["sz2_hi"][:8] == 0).all()
    assert (rb["chi_w"][8:] == 0).all() and (rb["sz2_lo"][8:] == 0).all()
    assert (ra["chi_w"][8:] > 0).all() and (rb["chi_w"][:8] > 0).all()
    assert_state_equal(gpu_state(a), gpu_state(b))
    # the measured half agrees with the oracle at the same updates
    p = orc.params(96, 30.0, seed=13)
    st = orc.neel(p)
    ro = orc.keyed_run(p, 0, 12, st)
    for t in range(12):
        assert_records_equal(ra[t] if t >= 8 else rb[t], ro[t], f"sweep={t}")
    oa, ob = a.measure(), b.measure()
    assert oa.sum[0] == ob.sum[0]
    assert oa.sum[8] == pytest.approx(ra["chi_w"].sum(), rel=1e-12)
    a.close()
    b.close()


def test_batch_temporal_switch():
    lc = gpu()
    specs = [dict(L=8, beta=4.0, seed=1), dict(L=40, beta=20.0, S=1.0, seed=2)]
    b = lc.Batch(specs)
    b.set_temporal(True)
    b.update(5)
    for i, s in enumerate(specs):
        p = orc.params(s["L"], s["beta"], Q=int(round(2 * s.get("S", 0.5))), seed=s["seed"])
        ro = orc.keyed_run(p, 0, 5, orc.neel(p))
        rg = b.records(i)
        for t in range(5):
            assert_records_equal(rg[t], ro[t], (i, t))
    b.close()


def test_tuning_gives_identical_results():
    # The block sizes of the union-find phases change no result.
    lc = gpu()
    L, beta = 1024, 40.0
    a = lc.Chain(L, beta, seed=3)
    b = lc.Chain(L, beta, seed=3)
    assert a.tuning() == {"link_threads": 256, "link_x_warps": 8, "compress_threads": 128}
    b.set_tuning(link_threads=128, link_x_warps=2, compress_threads=64)
    assert b.tuning() == {"link_threads": 128, "link_x_warps": 2, "compress_threads": 64}
    a.update(10)
    b.update(10)
    assert np.array_equal(a.records(), b.records())
    assert_state_equal(gpu_state(a), gpu_state(b))
    with pytest.raises(lc.LcqmcError):
        b.set_tuning(link_threads=192)
    with pytest.raises(lc.LcqmcError):
        b.set_tuning(compress_threads=160)
    # autotune: 8 trials of 2 ordinary updates; the chain goes on as an
    # untuned chain advanced by the same 16 updates
    c = lc.Chain(L, beta, seed=3)
    t = c.autotune(2)
    assert t["link_threads"] in (128, 256) and t["link_x_warps"] in (2, 4, 8) and t["compress_threads"] in (64, 128)
    d = lc.Chain(L, beta, seed=3)
    d.update(16)
    c.update(5)
    d.update(5)
    rc, rd = c.records(), d.records()
    assert len(rc) == len(rd) == 21 and np.array_equal(rc, rd)
    assert_state_equal(gpu_state(c), gpu_state(d))
    for h in (a, b, c, d):
        h.close()


def test_batch_autotune_identical():
    lc = gpu()
    specs = [dict(L=64, beta=16.0, seed=1), dict(L=200, beta=30.0, S=1.0, seed=2)]
    b1, b2 = lc.Batch(specs), lc.Batch(specs)
    b1.autotune(1)
    b2.update(8)
    b1.update(3)
    b2.update(3)
    for i in range(len(specs)):
        assert np.array_equal(b1.records(i), b2.records(i))
    b1.close()
    b2.close()


def _tile_sizes(ch):
    vp = ch.export_cells().astype(np.int64)
    ends = np.minimum(np.arange(0, len(vp) - 1 + 128, 128), len(vp) - 1)
    return np.diff(vp[np.unique(ends)])


@pytest.mark.parametrize("cap,slots", [(64, 0), ("mid", 0), (0, 4), (64, 1)])
@pytest.mark.parametrize("L,beta,Q", [(250, 70.0, 1), (1024, 40.0, 1), (40, 40.0, 2), (34, 10.0, 3)])
def test_update_parity_global_fallbacks(monkeypatch, cap, slots, L, beta, Q):
    # Tiles with more vertices than a tile keeps in shared memory (cap) take
    # the global-memory paths: every edge united in the global forest,
    # compression walks in global memory, ticks computed on the fly, every
    # root treated as leaving the tile.  A per-tile loop table of `slots`
    # entries spills the loops that do not fit to their global records.  The
    # results must not change.
    if cap == "mid":  # about two thirds of a thermalized tile: both paths in one chain
        cap = {1: 1000, 2: 800, 3: 500}[Q]
    if cap:
        monkeypatch.setenv("LCQMC_LOCAL_CAP", str(cap))
    if slots:
        monkeypatch.setenv("LCQMC_LOOP_SLOTS", str(slots))
    lc = gpu()
    p = orc.params(L, beta, Q=Q, seed=300 + L + cap + slots)
    st = orc.neel(p)
    ch = lc.Chain(L, beta, S=Q / 2, seed=300 + L + cap + slots)
    ch.set_temporal(True)
    biggest = 0
    try:
        for t in range(6):
            new, ro, go = orc.keyed_update(p, t, st, graph=True)
            ch.update(1)
            ctx = f"L={L} beta={beta} Q={Q} cap={cap} slots={slots} sweep={t}"
            assert_records_equal(ch.records()[0], ro, ctx)
            assert_graph_equal(ch.export_graph(), go, ctx)
            assert_state_equal(gpu_state(ch), new, ctx)
            sizes = _tile_sizes(ch)
            biggest = max(biggest, int(sizes.max()))
            if slots:
                # more distinct multi-node loops in a tile than the table holds
                m = sizes[0]  # the first tile's vertices
                r, pl, pr = go["root"][:m], go["pl"][:m], go["pr"][:m]
                assert len(np.unique(r[pl != pr])) > slots, ctx
            st = new
        if cap:
            # the fallback is reached: some tile held more vertices than the cap
            assert biggest > cap, (L, beta, Q, cap, biggest)
    finally:
        ch.close()
