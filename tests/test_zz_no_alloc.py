"""lcqmc_loops_noalloc: loop labelling for callers that must not allocate
device memory: code inside another framework's memory pool or under a
device-memory budget fixed in advance, and code whose other streams must not
wait for the device-wide synchronization that cudaMalloc implies.

It must give the same loop labels as the regular update path (the existing
entry point's export), and as the CPU oracle, which finds the loops of the
same graph by walking them.  The check runs twice in a row, on two different
graphs, because every call reuses the same fixed device array and must not
see the previous call's contents.  This file is collected last so that a
failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import orc

pytestmark = pytest.mark.gpu


def _fn():
    from paper_1810_07485_gb300 import lcqmc
    L = lcqmc.lib()
    f = L.lcqmc_loops_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f, lcqmc


def test_noalloc_labels_match_update_twice():
    import torch
    f, lcqmc = _fn()
    L, beta, seed = 160, 48.0, 12
    p = orc.params(L, beta, seed=seed)
    st = orc.neel(p)
    ch = lcqmc.Chain(L, beta, seed=seed)
    stream = torch.cuda.current_stream()
    sizes, sweep = [], 0
    for call in range(2):
        nup = 2 + call  # a different graph on each call
        for t in range(nup):
            st, _, go = orc.keyed_update(p, sweep, st, graph=(t == nup - 1))
            sweep += 1
        ch.update(nup)
        g = ch.export_graph(("pl", "pr", "root"))
        n = len(g["root"])
        sizes.append(n)
        assert np.array_equal(g["pl"].astype(np.int64), go["pl"]) and np.array_equal(g["pr"].astype(np.int64), go["pr"])
        # the oracle's graph goes in
        pl = torch.from_numpy(go["pl"].astype(np.int32)).cuda()
        pr = torch.from_numpy(go["pr"].astype(np.int32)).cuda()
        root = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rc = f(pl.data_ptr(), pr.data_ptr(), n, root.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lcqmc.lib().lcqmc_last_error()
        torch.cuda.synchronize()
        out = root.cpu().numpy()
        assert np.array_equal(out, g["root"]), call  # the existing entry point's labels
        assert np.array_equal(out.astype(np.int64), go["root"]), call  # the oracle's loop walk
    assert sizes[0] != sizes[1]
    ch.close()


def test_noalloc_rejects_oversize_and_bad_ids():
    import torch
    f, lcqmc = _fn()
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = f(buf.data_ptr(), buf.data_ptr(), (1 << 22) + 1, buf.data_ptr(), None)
    assert rc == -3  # LCQMC_E_TOO_LARGE
    assert b"maximum" in lcqmc.lib().lcqmc_last_error()
    bad = torch.tensor([0, 1, 9, 2], dtype=torch.int32, device="cuda")  # 9 is outside [0, 4)
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = f(bad.data_ptr(), bad.data_ptr(), 4, out.data_ptr(), None)
    assert rc == -1  # LCQMC_E_INVAL
