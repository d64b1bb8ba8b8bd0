"""Pins of the oracle's loop update (keyed and paper-literal forms).

What pins it, besides itself:
  * exact diagonalization (numpy eigh) within 3 standard errors,
  * the Curie limit beta -> 0 (chi = beta S(S+1)/3),
  * the paper's own numbers: n/(L beta) = 5.64e11/8.14e11 and clusters/(L beta)
    = 3.24e11/8.14e11 (Sec. 4.4), fragments = 2 x operators, and the S=1 row of
    Table 4 (E/L, chi_s, xi),
  * world-line invariants (Sec. 2), and
  * brute-force reconstructions of the predecessor links and of the loop
    partition (union-find over the exported edges) on small inputs.
"""
import json
import os

import numpy as np
import pytest

from oracle import ed, stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bond_ends(L, Q, b):
    i, a, a2 = b // (Q * Q), (b // Q) % Q, b % Q
    return i * Q + a, ((i + 1) % L) * Q + a2


def _ops_by_bond(orc, p, st):
    g = orc.geometry(p)
    out = []
    for b in range(g["nbond"]):
        taus = []
        for j in range(g["nwin"]):
            c = orc.cell_index(p, b, j)
            taus.extend(st.op_tau[st.op_ptr[c]:st.op_ptr[c + 1]])
        out.append(np.array(taus))
    return out


def check_worldlines(orc, p, st):
    """Every off-diagonal operator swaps two antiparallel spins; the world lines
    are periodic in tau (S=1/2) or match up to a subspin permutation (S=1)."""
    L, Q = p.L, p.Q
    g = orc.geometry(p)
    ops = _ops_by_bond(orc, p, st)
    events = [[] for _ in range(g["nsub"])]
    allev = []
    for b, taus in enumerate(ops):
        assert np.all(np.diff(taus) >= 0)
        assert np.all((taus >= 0) & (taus < p.beta))
        for t in taus:
            allev.append((t, b))
    allev.sort()
    s = st.s0.astype(np.int64).copy()
    for t, b in allev:
        ul, ur = _bond_ends(L, Q, b)
        assert s[ul] != s[ur], "off-diagonal operator on parallel spins"
        s[ul] ^= 1
        s[ur] ^= 1
    if Q == 1:
        assert np.array_equal(s, st.s0)
    else:
        for i in range(L):
            assert sorted(s[i * Q:(i + 1) * Q]) == sorted(st.s0[i * Q:(i + 1) * Q])


def brute_predecessors(L, Q, graph):
    """Cyclic predecessor of each vertex on its left / right subsite for Q=1,
    by sorting leg ends by (tau, id)."""
    assert Q == 1
    n = len(graph["tau"])
    legs = [[] for _ in range(L * Q)]
    for v in range(n):
        ul, ur = _bond_ends(L, Q, int(graph["bond"][v]))
        legs[ul].append((graph["tau"][v], v))
        legs[ur].append((graph["tau"][v], v))
    pl = np.empty(n, np.int64)
    pr = np.empty(n, np.int64)
    for u, lst in enumerate(legs):
        lst.sort()
        for k, (_, v) in enumerate(lst):
            prev = lst[k - 1][1]
            ul, ur = _bond_ends(L, Q, int(graph["bond"][v]))
            if ul == u:
                pl[v] = prev
            if ur == u:
                pr[v] = prev
    return pl, pr


def brute_partition(n, pl, pr):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for w in range(n):
        a, b = find(int(pl[w])), find(int(pr[w]))
        if a != b:
            parent[max(a, b)] = min(a, b)
    comp = {}
    for v in range(n):
        r = find(v)
        comp.setdefault(r, []).append(v)
    root = np.empty(n, np.int64)
    for members in comp.values():
        m = min(members)
        for v in members:
            root[v] = m
    return root


@pytest.mark.parametrize("L,beta,Q", [(2, 3.0, 1), (6, 5.0, 1), (10, 40.0, 1), (4, 3.0, 2), (2, 20.0, 2),
                                      (4, 3.0, 3), (2, 6.0, 4)])
def test_keyed_invariants(orc, L, beta, Q):
    p = orc.params(L, beta, Q=Q, seed=101)
    st = orc.neel(p)
    check_worldlines(orc, p, st)
    for t in range(25):
        new, rec, gr = orc.keyed_update(p, t, st, graph=True)
        n = int(rec["n"])
        assert n == len(gr["tau"])
        assert int(rec["n_off_old"]) == int(st.op_ptr[-1])
        assert int(rec["n_off_new"]) == int(new.op_ptr[-1])
        # Fragments = 2 x vertices (+ vertex-free loops); edges = 2 x vertices.
        assert int(rec["n_seg"]) == 2 * n + int(rec["n_free"])
        # Old operators are exactly the flagged vertices, in cell order.
        assert int(gr["flag"].sum()) == int(rec["n_off_old"])
        # Degree 2: every node is the lower end of exactly two fragments.
        cnt = np.bincount(np.concatenate([gr["pl"], gr["pr"]]), minlength=n)
        assert np.all(cnt == 2)
        # The loop labelling equals an independent union-find over the edges.
        assert np.array_equal(brute_partition(n, gr["pl"], gr["pr"]), gr["root"])
        assert int(rec["n_clusters"]) == len(np.unique(gr["root"])) + int(rec["n_free"])
        if Q == 1:
            bpl, bpr = brute_predecessors(L, Q, gr)
            assert np.array_equal(bpl, gr["pl"]) and np.array_equal(bpr, gr["pr"])
        check_worldlines(orc, p, new)
        st = new


def test_keyed_estimator_sums_exact(orc):
    """The 128-bit sum of squared loop lengths equals a brute-force recomputation
    from the exported graph (S=1/2: in ticks q(t) = rint(t 2^F), the fragment
    below w has length q(tau_w) - q(tau_P), plus q(beta) when it wraps through
    tau=0)."""
    L, beta = 8, 6.0
    p = orc.params(L, beta, seed=77)
    st = orc.neel(p)
    F = orc.geometry(p)["F"]
    for t in range(20):
        new, rec, gr = orc.keyed_update(p, t, st, graph=True)
        n = len(gr["tau"])
        W = {}
        touched = np.zeros(L, bool)
        for w in range(n):
            b = int(gr["bond"][w])
            touched[b] = touched[(b + 1) % L] = True
            for P in (int(gr["pl"][w]), int(gr["pr"][w])):
                tw, tp = gr["tau"][w], gr["tau"][P]
                wrapped = (tp > tw) or (tp == tw and P >= w)
                ln = int(np.rint(np.ldexp(tw, F))) - int(np.rint(np.ldexp(tp, F)))
                if wrapped:
                    ln += int(np.rint(np.ldexp(beta, F)))
                r = int(gr["root"][P])
                W[r] = W.get(r, 0) + ln
        sw2 = sum(v * v for v in W.values())
        sw2 += int((~touched).sum()) * int(np.rint(np.ldexp(beta, F))) ** 2
        assert sw2 == orc.u128(rec["sw2_lo"], rec["sw2_hi"])
        # temporal sums: per fragment e(top) - e(bottom), per loop summed
        qb = int(np.rint(np.ldexp(beta, F)))
        Z = {}
        for w in range(n):
            cw = orc.phase(int(np.rint(np.ldexp(gr["tau"][w], F))), qb)
            for P in (int(gr["pl"][w]), int(gr["pr"][w])):
                cp = orc.phase(int(np.rint(np.ldexp(gr["tau"][P], F))), qb)
                r = int(gr["root"][P])
                zr, zi = Z.get(r, (0, 0))
                Z[r] = (zr + cw[0] - cp[0], zi + cw[1] - cp[1])
        sz2 = sum(a * a + b * b for a, b in Z.values())
        assert sz2 == orc.u128(rec["sz2_lo"], rec["sz2_hi"])
        assert int(rec["n_free"]) == int((~touched).sum())
        st = new


def test_keyed_deterministic(orc):
    p = orc.params(12, 7.5, seed=9)
    a = orc.neel(p)
    b = orc.neel(p)
    ra = orc.keyed_run(p, 0, 30, a)
    rb = orc.keyed_run(p, 0, 30, b)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.op_tau, b.op_tau) and np.array_equal(a.s0, b.s0)
    # Resume from the state after 15 updates reproduces the last 15 records.
    c = orc.neel(p)
    orc.keyed_run(p, 0, 15, c)
    rc = orc.keyed_run(p, 15, 15, c)
    assert np.array_equal(rc, ra[15:])


def test_curie_limit_empty(orc):
    # At tiny beta almost every update has no vertex: every site is a free loop of
    # length beta, so chi_s = chi_q = beta/4 exactly for those updates.
    p = orc.params(16, 1e-6, seed=3)
    st = orc.neel(p)
    r = orc.keyed_run(p, 0, 50, st)
    empty = r["n"] == 0
    assert empty.sum() > 40
    assert np.allclose(r["chi_s"][empty], 1e-6 / 4, rtol=1e-12)
    assert np.allclose(r["chi_q"][empty], 1e-6 / 4, rtol=1e-12)
    assert np.all(r["n_clusters"][empty] == 16)


@pytest.mark.parametrize("form", ["keyed", "serial"])
@pytest.mark.parametrize("L,beta,Q,seed", [(2, 1.0, 1, 21), (4, 2.0, 1, 22), (8, 4.0, 1, 23),
                                           (12, 1.0, 1, 24), (4, 1.0, 2, 25), (2, 2.0, 2, 26),
                                           (2, 1.0, 3, 27), (4, 0.7, 3, 28), (2, 0.8, 4, 29),
                                           (4, 0.5, 4, 30)])
def test_vs_ed(orc, form, L, beta, Q, seed):
    p = orc.params(L, beta, Q=Q, seed=seed)
    n = 200000
    if form == "keyed":
        st = orc.neel(p)
        orc.keyed_run(p, 0, 500, st)
        r = orc.keyed_run(p, 500, n, st)
    else:
        r, _, _ = orc.serial_run(p, 0, n + 500)
        r = r[500:]
    ex = ed.thermal(L, beta, S=Q / 2)
    for name in ("energy", "chi_s", "chi_q", "chi_w"):
        m, e = stats.mean_err(r[name], 100)
        assert stats.within_sigma(m, e, ex[name], 3.0), (name, m, e, ex[name])


@pytest.mark.parametrize("Q", [1, 2, 3, 4])
def test_curie_limit_statistics(orc, Q):
    S = Q / 2
    beta = 0.01 * 0.75 / (S * (S + 1))  # the same expansion parameter beta S(S+1) for every S
    L = 8 if Q <= 2 else 4  # exact diagonalization size
    p = orc.params(L, beta, Q=Q, seed=31)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 100, st)
    r = orc.keyed_run(p, 100, 20000, st)
    ex = ed.thermal(L, beta, S=S)
    m, e = stats.mean_err(r["chi_s"], 50)
    assert stats.within_sigma(m, e, ex["chi_s"], 3.0)
    assert ex["chi_s"] == pytest.approx(beta * S * (S + 1) / 3, rel=2e-2)


def test_paper_overall_ratios(orc):
    """Sec. 4.4: operators/(L beta) = 5.64e11/8.14e11, clusters/(L beta) =
    3.24e11/8.14e11, fragments = edges = 2 x operators (large L, low T)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sec44_overall.json")))
    L, beta = 128, 128.0
    p = orc.params(L, beta, seed=3)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 100, st)
    r = orc.keyed_run(p, 100, 300, st)
    Lb = L * beta
    n_ratio = g["operators"] / g["space_time_volume"]
    c_ratio = g["clusters"] / g["space_time_volume"]
    m, e = stats.mean_err(r["n"] / Lb, 30)
    # The paper's ratios carry 3 significant digits (+-0.0005 on 0.69, 0.40).
    assert abs(m - n_ratio) < 3 * e + 0.0006
    m, e = stats.mean_err(r["n_clusters"] / Lb, 30)
    assert abs(m - c_ratio) < 3 * e + 0.0006
    assert np.all(r["n_seg"] == 2 * r["n"] + r["n_free"])
    assert g["fragments"] == pytest.approx(2 * g["operators"], rel=0.01)


def test_paper_table4_s1(orc):
    """Table 4, S=1: E/L, chi_s and the second-moment xi of the Haldane chain,
    at L=64 >> xi and beta=32 >> 1/gap."""
    g = json.load(open(os.path.join(GOLDEN, "paper_table4_s1.json")))
    L = 64
    p = orc.params(L, 32.0, Q=2, seed=5)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 200, st)
    r = orc.keyed_run(p, 200, 4000, st)
    m, e = stats.mean_err(r["energy"], 40)
    assert stats.within_sigma(m, e, g["energy_per_site"], 3.0)
    m, e = stats.mean_err(r["chi_s"], 40)
    assert stats.within_sigma(m, e, g["chi_s"], 3.0, g["chi_s_err"])
    xi, xe = stats.jackknife(stats.xi_second_moment(L), r["chi_s"], r["chi_q"], nbins=40)
    assert stats.within_sigma(xi, xe, g["xi"], 3.0, g["xi_err"])


def test_phase_factor(orc):
    """The integer phase factor against numpy's exp(i 2 pi q / qbeta), within
    the table-and-interpolation bound (2 pi / 2^16)^2 / 8 of the 2^30 unit plus
    the roundings, over tick counts of several magnitudes."""
    rng = np.random.default_rng(5)
    for qbeta in (1000003, 1 << 30, 3 * (1 << 44) + 12345, (1 << 59) + 7):
        qs = list(rng.integers(0, qbeta, 400, dtype=np.int64)) + [0, qbeta - 1, qbeta // 4, qbeta // 2]
        for q in qs:
            c, s = orc.phase(int(q), qbeta)
            ang = 2 * np.pi * (int(q) / qbeta)
            assert abs(c - np.cos(ang) * 2**30) < 4.0 and abs(s - np.sin(ang) * 2**30) < 4.0, (qbeta, q)
