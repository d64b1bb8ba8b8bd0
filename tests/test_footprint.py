"""Admission footprint model (host only): monotone in size and temperature,
the single-chain benchmark workloads fit one GB300, and the served request mix
has a small rejected fraction at a 200 GB budget."""
import os
import shutil

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lc():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1810_07485_gb300 import build, lcqmc
    build.build()
    return lcqmc


def test_monotone(lc):
    a = lc.footprint(1024, 64.0)
    assert lc.footprint(2048, 64.0) > a and lc.footprint(1024, 128.0) > a
    assert lc.footprint(1024, 64.0, S=1.0) > a


def test_benchmark_workloads_fit(lc):
    hbm = 284208 * 2**20
    assert lc.footprint(1 << 16, 4096.0) < 0.2 * hbm
    assert lc.footprint(1 << 20, 1024.0) < 0.3 * hbm


def test_served_mix_rejection_fraction(lc):
    # L log-uniform in [64, 65536] (even), beta = L*U, U log-uniform in [1/4, 4].
    rng = np.random.default_rng(0)
    budget = 200e9
    rej = {0.5: 0, 1.0: 0}
    tot = {0.5: 0, 1.0: 0}
    for _ in range(2000):
        S = 0.5 if rng.random() < 0.5 else 1.0
        L = int(round(np.exp(rng.uniform(np.log(64), np.log(65536))) / 2)) * 2
        beta = L * float(np.exp(rng.uniform(np.log(0.25), np.log(4.0))))
        tot[S] += 1
        try:
            if lc.footprint(L, beta, S=S) > budget:
                rej[S] += 1
        except lc.LcqmcError:
            rej[S] += 1
    for S in (0.5, 1.0):
        assert rej[S] / tot[S] < 0.2
