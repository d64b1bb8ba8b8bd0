"""Failure handling on the GPU without a GPU fault.

* Device allocation failure, injected on the host: a caller-supplied
  allocator (lcqmc_create_ex) that refuses the k-th request.  Creation must
  fail cleanly with LCQMC_E_NOMEM, free whatever it had taken, and leave the
  process able to create and run chains.
* The opt-in forest check (LCQMC_CHECK_FOREST=1) verifies after every
  compression that each node's word is its root; on a correct update it
  stays silent and changes nothing.
* A bounded device wait that runs out: the union-find walks of a correct
  chain get a bound of one step (lcqmc_set_wait_limit), so the update stops
  on the device.  The call reports LCQMC_E_DEVICE_TIMEOUT, the chain's state
  is untouched, and the next update at the default bound is the oracle's.
  No kernel faults or hangs: every wait returns once its bound is reached.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC), ("free", FREE), ("ctx", ctypes.c_void_p)]


class Pool:
    """torch's caching allocator behind the library's allocator hooks, refusing
    the request numbered fail_at (0-based); counts what is outstanding."""

    def __init__(self, fail_at=None):
        import torch
        self.torch = torch
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        self._a = ALLOC(self._alloc)
        self._f = FREE(self._free)
        self.struct = Allocator(self._a, self._f, None)

    def _alloc(self, nbytes, ctx):
        k = self.calls
        self.calls += 1
        if self.fail_at is not None and k >= self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(max(int(nbytes), 1))
        self.live[p] = nbytes
        return p

    def _free(self, ptr, ctx):
        if ptr:
            self.torch.cuda.caching_allocator_delete(ptr)
            self.live.pop(ptr, None)


def create(lc, pool, L=64, beta=8.0, seed=5):
    h = ctypes.c_void_p()
    rc = lc.lib().lcqmc_create_ex(L, 0.5, 1.0, beta, seed, None, ctypes.byref(pool.struct), ctypes.byref(h))
    return rc, h


def test_allocation_failure_is_clean():
    from paper_1810_07485_gb300 import lcqmc as lc
    probe = Pool()
    rc, h = create(lc, probe)
    assert rc == 0
    lc.lib().lcqmc_destroy(h)
    n = probe.calls
    assert n > 3 and not probe.live  # every buffer handed back
    for k in sorted(set([0, 1, n // 2, n - 1])):
        pool = Pool(fail_at=k)
        rc, h = create(lc, pool)
        assert rc == -2, (k, rc)  # LCQMC_E_NOMEM
        assert not h.value
        assert not pool.live, k  # partial allocations released
        assert b"alloc" in lc.lib().lcqmc_last_error().lower()
    # the process still works, on the caller's allocator and on the default one
    pool = Pool()
    rc, h = create(lc, pool)
    assert rc == 0
    ch = lc.Chain(64, 8.0, seed=5)
    assert lc.lib().lcqmc_update(h, 20) == 0
    ch.update(20)
    buf = (lc.Record * 64)()
    cnt = ctypes.c_int64()
    assert lc.lib().lcqmc_get_records(h, buf, 64, ctypes.byref(cnt)) == 0
    ra = lc.records_to_numpy(buf, cnt.value)
    assert np.array_equal(ra, ch.records())
    lc.lib().lcqmc_destroy(h)
    ch.close()
    assert not pool.live


def test_forest_check_silent_on_correct_updates(monkeypatch):
    from oracle import orc
    from paper_1810_07485_gb300 import lcqmc as lc
    monkeypatch.setenv("LCQMC_CHECK_FOREST", "1")
    L, beta = 200, 30.0
    p = orc.params(L, beta, seed=8)
    st = orc.neel(p)
    ro = orc.keyed_run(p, 0, 12, st)
    ch = lc.Chain(L, beta, seed=8)
    ch.update(12)
    rg = ch.records()
    for f in ("n", "n_clusters", "sw2_lo", "sw2_hi", "sf2_lo", "sf2_hi"):
        assert np.array_equal(rg[f].astype(np.int64), ro[f].astype(np.int64)), f
    ch.close()


def test_device_timeout_leaves_state_and_recovers(monkeypatch):
    from oracle import orc
    from paper_1810_07485_gb300 import lcqmc as lc
    # every tile keeps at most 64 vertices in shared memory, so that its edges
    # are united in the global forest, whose walks the bound applies to
    monkeypatch.setenv("LCQMC_LOCAL_CAP", "64")
    L, beta, seed = 1024, 40.0, 9
    p = orc.params(L, beta, seed=seed)
    st = orc.neel(p)
    ch = lc.Chain(L, beta, seed=seed)
    try:
        for t in range(3):
            st, ro, _ = orc.keyed_update(p, t, st)
            ch.update(1)
            assert int(ch.records()[0]["n"]) == int(ro["n"])
        s0, ptr, tau = ch.export_config()
        assert ch.geometry().sweep == 3
        ch.set_wait_limit(1)
        ch.update(1)
        with pytest.raises(lc.LcqmcError) as e:
            ch.sync()
        assert e.value.code == -5  # LCQMC_E_DEVICE_TIMEOUT
        s0b, ptrb, taub = ch.export_config()
        assert np.array_equal(s0, s0b) and np.array_equal(ptr, ptrb) and np.array_equal(tau, taub)
        assert ch.geometry().sweep == 3
        assert len(ch.records()) == 0
        with pytest.raises(lc.LcqmcError):
            ch.set_wait_limit(1 << 23)  # above the maximum bound
        ch.set_wait_limit(0)
        new, ro, go = orc.keyed_update(p, 3, st, graph=True)
        ch.update(1)
        rg = ch.records()
        assert len(rg) == 1
        for f in ("n", "n_off_old", "n_off_new", "n_clusters", "sw2_lo", "sw2_hi", "sf2_lo", "sf2_hi"):
            assert int(rg[0][f]) == int(ro[f]), f
        g = ch.export_graph()
        assert np.array_equal(g["root"].astype(np.int64), go["root"])
        s0c, ptrc, tauc = ch.export_config()
        assert np.array_equal(s0c, new.s0) and np.array_equal(ptrc.astype(np.int64), new.op_ptr)
        assert np.array_equal(tauc, new.op_tau)
    finally:
        ch.close()
