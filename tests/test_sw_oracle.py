"""Pins of the Swendsen-Wang oracle (Sec. 4.1 benchmark), CPU only.

What fixes each part independently of the oracle's own code:
* the whole transition (bond probability, cluster flip, estimators): exact
  enumeration of every configuration of L = 2, 3, 4 tori, against long runs,
  and the joint (E, M) histogram of L = 2 and 3;
* the cluster partition: scipy's connected components of the exported bonds;
* the limits K = 0 (no bond, every site its own cluster) and K -> infinity
  (every bond between equal spins, one cluster from the ordered state);
* the bond threshold: p = 1/2 at K = ln(2)/2, p(K_c) = 2 - sqrt(2) exactly,
  the paper's printed K_c, and the measured activation frequency;
* invariants of one update: active bonds join equal new spins, every
  cluster flips as a whole.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KC = math.log(1.0 + math.sqrt(2.0)) / 2.0


def bond_list(L):
    """The 2N bonds of the definition: R(i) = (i, right), D(i) = (i, below)."""
    b = []
    for i in range(L * L):
        x, y = i % L, i // L
        b.append((i, y * L + (x + 1) % L))
        b.append((i, ((y + 1) % L) * L + x))
    return np.array(b)


def exact(L, K):
    """<E>/N, <M^2>/N and the joint distribution of (sum sigma sigma, M) by
    enumerating every configuration."""
    N = L * L
    c = np.arange(2 ** N, dtype=np.int64)
    sig = 1 - 2 * ((c[:, None] >> np.arange(N)) & 1)
    b = bond_list(L)
    ss = (sig[:, b[:, 0]] * sig[:, b[:, 1]]).sum(1)
    M = sig.sum(1)
    w = np.exp(K * (ss - ss.max()))
    Z = w.sum()
    e = -(w * ss).sum() / Z / N
    m2 = (w * M * M).sum() / Z / N
    joint = {}
    for k, v in zip(zip(ss.tolist(), M.tolist()), (w / Z).tolist()):
        joint[k] = joint.get(k, 0.0) + v
    return e, m2, joint


def binned(x, nbin=50):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbin * nbin
    b = x[:n].reshape(nbin, -1).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbin)


def test_threshold_closed_forms(orc):
    assert orc.sw_threshold(0.0) == 0
    assert orc.sw_threshold(math.log(2.0) / 2.0) == 2 ** 31  # e^{-2K} = 1/2
    assert orc.sw_threshold(50.0) == 2 ** 32                 # every equal bond
    # e^{-2 K_c} = sqrt(2) - 1, so p(K_c) = 2 - sqrt(2)
    assert orc.sw_threshold(KC) == round((2.0 - math.sqrt(2.0)) * 2 ** 32)


def test_paper_critical_coupling():
    g = json.load(open(os.path.join(GOLDEN, "paper_sec41_sw.json")))
    assert abs(KC - g["K_c_printed"]) < 1e-6
    assert g["L"] == 8192 and g["burn_in_steps"] == 128 and g["timed_steps"] == 128


@pytest.mark.parametrize("L,K", [(2, 0.3), (3, 0.2), (3, KC), (4, KC), (4, 0.7)])
def test_matches_exact_enumeration(orc, L, K):
    e_ex, m2_ex, _ = exact(L, K)
    s = np.zeros(L * L, np.uint8)
    orc.sw_run(L, K, 11, 0, 200, s)
    r = orc.sw_run(L, K, 11, 200, 40000, s)
    N = L * L
    for name, x, ref in (("energy", r["energy"], e_ex), ("chi", r["chi"], m2_ex),
                         ("M^2/N", r["mag"].astype(np.float64) ** 2 / N, m2_ex)):
        m, err = binned(x)
        assert abs(m - ref) < 4 * err + 1e-12, (name, m, err, ref)


@pytest.mark.parametrize("L,K", [(2, 0.4), (3, 0.3)])
def test_joint_energy_magnetization_histogram(orc, L, K):
    # The state after update t has magnetization mag[t] and equal-bond count
    # n_eq[t+1]; thinned by 4 so that the samples are nearly independent.
    N, nb = L * L, 2 * L * L
    _, _, joint = exact(L, K)
    s = np.zeros(N, np.uint8)
    orc.sw_run(L, K, 5, 0, 100, s)
    r = orc.sw_run(L, K, 5, 100, 200001, s)
    ss = 2 * r["n_eq"][1:] - nb
    M = r["mag"][:-1]
    ss, M = ss[::4], M[::4]
    n = len(ss)
    got = {}
    for k in zip(ss.tolist(), M.tolist()):
        got[k] = got.get(k, 0) + 1
    assert set(got) <= {k for k, v in joint.items() if v > 0}
    for k, p in joint.items():
        exp_n = n * p
        if exp_n < 20:
            continue
        z = (got.get(k, 0) - exp_n) / math.sqrt(exp_n * (1 - p))
        assert abs(z) < 5.5, (k, got.get(k, 0), exp_n)


@pytest.mark.parametrize("L,K,seed", [(2, 0.5, 1), (3, 0.9, 2), (7, KC, 3), (16, KC, 4), (16, 1.5, 5)])
def test_partition_is_connected_components(orc, L, K, seed):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(seed)
    N = L * L
    s = rng.integers(0, 2, N).astype(np.uint8)
    s_old = s.copy()
    rec, roots, bonds = orc.sw_update(L, K, seed, 7, s, roots=True, bonds=True)
    b = bond_list(L)[bonds.astype(bool)]
    g = coo_matrix((np.ones(len(b)), (b[:, 0], b[:, 1])), shape=(N, N))
    nc, lab = connected_components(g, directed=False)
    canon = np.full(nc, N)
    np.minimum.at(canon, lab, np.arange(N))
    assert np.array_equal(roots, canon[lab])
    assert rec["n_clusters"] == nc
    sizes = np.bincount(lab)
    assert int(rec["sum_c2"]) == int((sizes.astype(np.int64) ** 2).sum())
    assert rec["max_cluster"] == sizes.max()
    assert rec["n_act"] == len(b)
    # bonds only between equal spins; every cluster flips as a whole
    eq = s_old[bond_list(L)[:, 0]] == s_old[bond_list(L)[:, 1]]
    assert rec["n_eq"] == eq.sum() and not (bonds.astype(bool) & ~eq).any()
    flip = s ^ s_old
    assert np.array_equal(flip, flip[roots])
    assert (s[b[:, 0]] == s[b[:, 1]]).all()
    assert rec["mag"] == int((1 - 2 * s.astype(np.int64)).sum())


def test_zero_coupling_isolated_sites(orc):
    L = 32
    N = L * L
    s = np.zeros(N, np.uint8)
    flips = 0
    for t in range(40):
        old = s.copy()
        rec, _, _ = orc.sw_update(L, 0.0, 3, t, s)
        assert rec["n_act"] == 0 and rec["n_clusters"] == N and rec["sum_c2"] == N
        assert rec["max_cluster"] == 1
        flips += int((old != s).sum())
    # each site flips with probability 1/2, independently
    n = 40 * N
    assert abs(flips - n / 2) < 5 * math.sqrt(n / 4)


def test_infinite_coupling_one_cluster(orc):
    L = 24
    N = L * L
    s = np.zeros(N, np.uint8)
    seen = set()
    for t in range(30):
        rec, roots, _ = orc.sw_update(L, 50.0, 9, t, s, roots=True)
        assert rec["n_eq"] == 2 * N and rec["n_act"] == 2 * N
        assert rec["n_clusters"] == 1 and rec["sum_c2"] == N * N and rec["max_cluster"] == N
        assert (roots == 0).all() and len(set(s.tolist())) == 1
        seen.add(int(s[0]))
    assert seen == {0, 1}  # the single cluster's coin takes both values


def test_activation_frequency(orc):
    # Given n_eq equal bonds, the active ones are Binomial(n_eq, T / 2^32).
    L = 128
    s = np.zeros(L * L, np.uint8)
    r = orc.sw_run(L, KC, 21, 0, 60, s)
    p = orc.sw_threshold(KC) / 2 ** 32
    ne, na = r["n_eq"].sum(), r["n_act"].sum()
    assert abs(na - p * ne) < 5 * math.sqrt(ne * p * (1 - p))
