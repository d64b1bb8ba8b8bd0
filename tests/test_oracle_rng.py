"""Pins of the oracle's random-number layer: Philox4x32-10 against NVIDIA's
independent implementation (cuRAND's host generator, which runs on the CPU) and
the Poisson thresholds against scipy."""
import ctypes

import numpy as np
import pytest
from scipy import stats as sps


def _curand_host(seed, n):
    try:
        lib = ctypes.CDLL("libcurand.so.10")
    except OSError:
        try:
            lib = ctypes.CDLL("/usr/local/cuda/lib64/libcurand.so")
        except OSError:
            pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    # CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
        pytest.skip("cuRAND host generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    buf = np.zeros(n, dtype=np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return buf


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(orc, seed):
    # cuRAND's host Philox4_32_10 generator emits block i = Philox(ctr=(0,0,i,0), key=seed).
    nblk = 512
    ref = _curand_host(seed, 4 * nblk).reshape(nblk, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(nblk):
        assert list(orc.philox([0, 0, i, 0], key)) == list(ref[i]), i


def test_philox_uniform_bits(orc):
    # Every output bit of the counter-mode stream is a fair coin (all four words,
    # all counter words varied).
    n = 4000
    bits = np.zeros(128)
    for i in range(n):
        out = orc.philox([i, i * 7 + 1, i * 13 + 5, 3], [11, 22])
        for w in range(4):
            bits[w * 32:(w + 1) * 32] += (out[w] >> np.arange(32, dtype=np.uint32)) & 1
    z = (bits - n / 2) / np.sqrt(n / 4)
    assert np.abs(z).max() < 4.5


@pytest.mark.parametrize("mu", [8.0, 3.25, 0.125, 1e-9])
def test_poisson_thresholds_vs_scipy(orc, mu):
    T = orc.poisson_thresholds(mu).astype(np.float64)
    cdf = sps.poisson.cdf(np.arange(orc.KMAX), mu)
    ref = np.minimum(np.ldexp(cdf, 64), np.ldexp(1.0, 64) - 1)
    assert np.all(np.diff(T) >= 0)
    np.testing.assert_allclose(T, ref, rtol=1e-12, atol=2.0 ** 12)


def test_poisson_counts_from_philox(orc):
    # Counts drawn exactly as the insertion step draws them follow Poisson(8).
    T = orc.poisson_thresholds(8.0)
    n = 20000
    K = np.zeros(n, dtype=np.int64)
    for i in range(n):
        o = orc.philox([1 << 24, i, 0, 0], [5, 0])
        U = int(o[0]) | (int(o[1]) << 32)
        K[i] = int(np.searchsorted(T, np.uint64(U), side="right"))
    obs = np.bincount(np.minimum(K, 20), minlength=21)
    p = sps.poisson.pmf(np.arange(21), 8.0)
    p[20] = sps.poisson.sf(19, 8.0)
    chi2 = ((obs - n * p) ** 2 / (n * p)).sum()
    assert chi2 < sps.chi2.ppf(0.9999, 20)
