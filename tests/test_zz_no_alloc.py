"""lcqmc_loops_noalloc: loop labelling for callers that must not allocate
device memory (cudaMalloc synchronizes the device, is refused while a CUDA
graph is being captured, and can break a memory budget fixed in advance).

It must give the same loop labels as the regular update path.  The check runs
twice in a row, on two different graphs, because every call reuses the same
fixed device array and must not see the previous call's contents.  This file
is collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

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
    ch = lcqmc.Chain(160, 48.0, seed=12)
    stream = torch.cuda.current_stream()
    sizes = []
    for call in range(2):
        ch.update(2 + call)  # a different graph on each call
        g = ch.export_graph(("pl", "pr", "root"))
        n = len(g["root"])
        sizes.append(n)
        pl = torch.from_numpy(g["pl"]).cuda()
        pr = torch.from_numpy(g["pr"]).cuda()
        root = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rc = f(pl.data_ptr(), pr.data_ptr(), n, root.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lcqmc.lib().lcqmc_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(root.cpu().numpy(), g["root"]), call
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
