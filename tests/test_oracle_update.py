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
from oracle import orc as _orc

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
                                           (12, 1.0, 1, 24), (8, 16.0, 1, 31), (12, 16.0, 1, 32),
                                           (4, 1.0, 2, 25), (2, 2.0, 2, 26),
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


def cut_permutation_q2(p, sweep, s0, nlegs):
    """tau = 0 joins of an S = 1 chain (2 subspins per site): the top of
    subsite u continues into the bottom of perm[u].  A join must connect equal
    spins (top spin = s0 xor the parity of the subsite's off-diagonal
    operators, nlegs[u]); where both
    joins are allowed, the coin of tag 4 at the site index decides (swap on 1).
    Philox itself is pinned against cuRAND (test_oracle_rng.py)."""
    L, seed = int(p.L), int(p.seed)
    perm = np.arange(2 * L)
    for i in range(L):
        u0, u1 = 2 * i, 2 * i + 1
        t0, t1 = int(s0[u0]) ^ (nlegs[u0] & 1), int(s0[u1]) ^ (nlegs[u1] & 1)
        ok_id = t0 == s0[u0] and t1 == s0[u1]
        ok_sw = t0 == s0[u1] and t1 == s0[u0]
        if ok_id and ok_sw:
            w = _orc.philox([4 << 24, i >> 7, 0, sweep], [seed & 0xFFFFFFFF, seed >> 32])
            swap = (int(w[(i & 127) >> 5]) >> (i & 31)) & 1
        else:
            assert ok_id or ok_sw
            swap = int(ok_sw)
        if swap:
            perm[u0], perm[u1] = u1, u0
    return perm


def plain_loop_moments(p, gr, perm=None):
    """The estimators' plain definitions (Sec. 2 improved estimators, Sec. 5
    moment estimators), in fp64 from the exported vertices, with none of the
    oracle's fixed-point arithmetic: per loop c, W_c = sum of its fragments'
    lengths, C_c + i S_c = sum of len e^{i k x} (k = 2 pi / L, x the fragment's
    site) and Z_c = sum over fragments of e^{i w1 tau_top} - e^{i w1 tau_bottom}
    (w1 = 2 pi / beta, so that Z_c / (i w1) is the loop's integral of
    e^{i w1 tau}).

    The fragments are rebuilt here: on every subsite the legs are ordered by
    (tau, vertex id); a fragment runs from one leg up to the next, and from the
    last leg up through tau = beta into the bottom of perm[u] (the tau = 0
    join; the identity for S = 1/2), on through every empty subspin it meets
    (one more period each), to the next leg.  A fragment belongs to the loop
    of the vertex at its lower end (node = the pair of fragments above a
    vertex).  Cycles of perm through empty subsites only are vertex-free loops
    of m periods.  With perm = None (S >= 3/2 here) the tau = 0 joins are read
    off the exported predecessors, which is exact when no subsite is empty.

    Returns (per-loop W, C, S, Z, fragment counts, total length, free loops)."""
    L, Q, beta = int(p.L), int(p.Q), float(p.beta)
    tau = np.asarray(gr["tau"], np.float64)
    bond = np.asarray(gr["bond"], np.int64)
    root = np.asarray(gr["root"], np.int64)
    n = len(tau)
    ul = (bond // (Q * Q)) * Q + (bond // Q) % Q
    ur = ((bond // (Q * Q) + 1) % L) * Q + bond % Q
    legs = [[] for _ in range(L * Q)]
    for v in range(n):
        legs[int(ul[v])].append((tau[v], v))
        legs[int(ur[v])].append((tau[v], v))
    for lst in legs:
        lst.sort()
    if perm is None:
        assert Q == 1 or all(legs), "perm needed where a subsite is empty"
        perm = np.arange(L * Q)
        if Q > 1:
            first = {lst[0][1]: u for u, lst in enumerate(legs)}  # unique ids per subsite's first leg
            for u, lst in enumerate(legs):
                v = lst[-1][1]
                # the fragment above u's last leg ends at the first leg w of
                # some subsite of the same site whose predecessor there is v
                for w_u in range((u // Q) * Q, (u // Q + 1) * Q):
                    w = legs[w_u][0][1]
                    pred = gr["pl"][w] if int(ul[w]) == w_u else gr["pr"][w]
                    if int(pred) == v and first.get(w) is not None:
                        perm[u] = w_u
                        break
            assert sorted(perm) == list(range(L * Q))
    k, w1 = 2 * np.pi / L, 2 * np.pi / beta
    acc = {}
    total = 0.0

    def add(r, length, x, tb, tt):
        a = acc.setdefault(r, [0.0, 0.0, 0.0, 0j, 0])
        a[0] += length
        a[1] += length * np.cos(k * x)
        a[2] += length * np.sin(k * x)
        a[3] += np.exp(1j * w1 * tt) - np.exp(1j * w1 * tb)
        a[4] += 1

    for u, lst in enumerate(legs):
        x = u // Q
        for (ta, va), (tb_, _) in zip(lst[:-1], lst[1:]):
            add(int(root[va]), tb_ - ta, x, ta, tb_)
            total += tb_ - ta
        if lst:
            t_last, v_last = lst[-1]
            c, nxt = 1, int(perm[u])
            while not legs[nxt]:
                c += 1
                nxt = int(perm[nxt])
                assert c <= Q
            t_first = legs[nxt][0][0]
            add(int(root[v_last]), t_first - t_last + c * beta, x, t_last, t_first)
            total += t_first - t_last + c * beta
    seen = np.zeros(L * Q, bool)
    n_free = 0
    for u in range(L * Q):
        if legs[u] or seen[u]:
            continue
        cyc, y = [], u
        while not seen[y] and not legs[y]:
            seen[y] = True
            cyc.append(y)
            y = int(perm[y])
        if y == u:  # a cycle of empty subsites: one vertex-free loop
            m = len(cyc)
            acc[("free", u)] = [m * beta, m * beta * np.cos(k * (u // Q)), m * beta * np.sin(k * (u // Q)), 0j, 1]
            total += m * beta
            n_free += 1
    vals = list(acc.values())
    W = np.array([a[0] for a in vals])
    C = np.array([a[1] for a in vals])
    S = np.array([a[2] for a in vals])
    Z = np.array([a[3] for a in vals])
    nf = np.array([a[4] for a in vals], np.float64)
    return W, C, S, Z, nf, total, n_free


def _square_sum_bound(X, delta):
    """Largest |sum |X_c|^2 - sum |X_c + e_c|^2| over |e_c| <= delta_c."""
    return float(np.sum(2 * np.abs(X) * delta + delta * delta))


@pytest.mark.parametrize("L,beta,Q", [(2, 3.0, 1), (8, 6.0, 1), (16, 0.5, 1), (64, 16.0, 1),
                                      (250, 70.0, 1), (8, 10.0, 2), (12, 0.4, 2), (4, 8.0, 3),
                                      (4, 8.0, 4)])
def test_estimators_vs_plain_fp64(orc, L, beta, Q):
    """The oracle's estimators (ticks of 2^-F, 32-bit Fourier weights, the
    interpolated phase table, exact integer sums) against their plain fp64
    definitions, within the bound their arithmetic implies:
      * a fragment's length in ticks is off by at most one tick 2^-F (two
        roundings of half a tick);
      * its Fourier term adds at most len 2^-33 (the 32-bit cos/sin weight) and
        half a tick (the rounding of the product);
      * a phase factor is off by at most 4 units of 2^-30 (pinned against numpy
        in test_phase_factor) plus w1 times half a tick (the rounded time);
    summed per loop into delta_c and carried through the squares.  A dropped
    term, a wrong sign, a wrong site or exponent F, or a wrong crossing count
    each miss by orders of magnitude more."""
    p = orc.params(L, beta, Q=Q, seed=4000 + L + Q)
    st = orc.neel(p)
    F = orc.geometry(p)["F"]
    tick = 2.0 ** -F
    w1 = 2 * np.pi / beta
    checked = 0
    saw_free = saw_wrap = False
    for t in range(12):
        new, rec, gr = orc.keyed_update(p, t, st, graph=True)
        perm = None
        if Q == 2:
            ob = gr["bond"][gr["flag"] != 0]  # off-diagonal operators flip spins, diagonal ones do not
            ends = np.concatenate([(ob // 4) * 2 + (ob // 2) % 2, ((ob // 4 + 1) % L) * 2 + ob % 2])
            perm = cut_permutation_q2(p, t, st.s0, np.bincount(ends, minlength=2 * L))
        st = new
        W, C, S, Z, nf, total, n_free = plain_loop_moments(p, gr, perm)
        # crossings: the fragments and free loops cover every subsite's period once
        assert total == pytest.approx(Q * L * beta, rel=1e-12), (t, total)
        assert int(rec["n_free"]) == n_free
        saw_free |= n_free > 0
        saw_wrap |= bool(np.any(nf > 1))
        norm = 4.0 * beta * L
        chi_s, chi_q = np.sum(W * W) / norm, np.sum(C * C + S * S) / norm
        chi_w = np.sum(np.abs(Z) ** 2) / (w1 * w1) / norm
        dW = nf * tick
        dF = nf * (1.5 * tick) + np.abs(W) * 2.0 ** -33
        dZ = nf * 2 * (4 * 2.0 ** -30 + w1 * 0.5 * tick)
        fp = 1e-13  # fp64 rounding of the plain sums
        tol_s = _square_sum_bound(W, dW) / norm + fp * chi_s
        tol_q = (_square_sum_bound(C, dF) + _square_sum_bound(S, dF)) / norm + fp * chi_q
        tol_w = _square_sum_bound(Z, dZ) / (w1 * w1) / norm + fp * chi_w
        assert abs(float(rec["chi_s"]) - chi_s) <= tol_s, (t, rec["chi_s"], chi_s, tol_s)
        assert abs(float(rec["chi_q"]) - chi_q) <= tol_q, (t, rec["chi_q"], chi_q, tol_q)
        assert abs(float(rec["chi_w"]) - chi_w) <= tol_w, (t, rec["chi_w"], chi_w, tol_w)
        # the bounds are tight enough to matter: far below the loop moments
        # themselves (chi_q may vanish: at L = 2, q = 2 pi is the conserved
        # uniform magnetization)
        assert tol_s <= 1e-8 * chi_s and tol_q <= 1e-8 * chi_s
        n = int(rec["n"])
        assert float(rec["energy"]) == pytest.approx(Q * Q * p.J / 4 - n / (beta * L), rel=1e-14, abs=1e-15)
        assert int(rec["n_clusters"]) == len(W)
        checked += 1
    assert checked == 12
    if (L, beta, Q) in ((16, 0.5, 1), (12, 0.4, 2)):
        assert saw_free
