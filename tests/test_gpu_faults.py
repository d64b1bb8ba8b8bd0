"""Failure handling on the GPU without a GPU fault.

* Device allocation failure, injected on the host: a caller-supplied
  allocator (lcqmc_create_ex) that refuses the k-th request.  Creation must
  fail cleanly with LCQMC_E_NOMEM, free whatever it had taken, and leave the
  process able to create and run chains.
* The opt-in forest check (LCQMC_CHECK_FOREST=1) verifies after every
  compression that each node's word is its root; on a correct update it
  stays silent and changes nothing.
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
