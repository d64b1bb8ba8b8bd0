"""Exact diagonalization of the periodic Heisenberg chain (test infrastructure).

H = J sum_{j=1}^{L} S_j . S_{j+1} with S_{L+1} = S_1 (Eq. 1, Sec. 2), spin S in
{1/2, 1}.  Thermal averages <A> = Tr A e^{-beta H} / Z (Sec. 2) are evaluated
from the full spectrum, block by block in total S^z, with numpy.linalg.eigh.

Dynamic susceptibility at wave number q:
  chi(q) = (1/(beta L)) < |int_0^beta dtau M_q(tau)|^2 >,  M_q = sum_x e^{iqx} S^z_x
         = (1/(L Z)) sum_{m,n} |<m|M_q|n>|^2 (e^{-beta E_n} - e^{-beta E_m}) / (E_m - E_n)
(with beta e^{-beta E_n} for E_m = E_n).  q = pi gives the staggered
susceptibility chi_s; q = pi + 2 pi / L enters the second-moment correlation
length.  Feasible for L <= 12 (S=1/2) and L <= 8 (S=1).
"""
import itertools

import numpy as np


def _basis(L, twoS):
    d = twoS + 1
    m_vals = np.array([twoS / 2.0 - k for k in range(d)])  # S^z values of one site
    states = np.array(list(itertools.product(range(d), repeat=L)), dtype=np.int64)
    sz = m_vals[states]  # (D, L)
    return states, sz, m_vals


def spectrum(L, S=0.5, J=1.0):
    """Returns a list of (energies, eigenvectors, sz_configs) per S^z sector."""
    twoS = int(round(2 * S))
    d = twoS + 1
    states, sz, m_vals = _basis(L, twoS)
    Mtot = sz.sum(axis=1)
    weights = d ** np.arange(L - 1, -1, -1)
    sectors = []
    for M in np.unique(Mtot):
        idx = np.nonzero(Mtot == M)[0]
        sub = states[idx]
        code = sub @ weights
        pos = {int(c): i for i, c in enumerate(code)}
        D = len(idx)
        H = np.zeros((D, D))
        szs = sz[idx]
        for j in range(L):
            k = (j + 1) % L
            H[np.arange(D), np.arange(D)] += J * szs[:, j] * szs[:, k]
            # (J/2) (S+_j S-_k + S-_j S+_k); S+ raises m: index k_site -> k_site-1.
            for a in range(D):
                cj, ck = sub[a, j], sub[a, k]
                m_j, m_k = m_vals[cj], m_vals[ck]
                S_ = twoS / 2.0
                # S+_j S-_k
                if cj > 0 and ck < d - 1:
                    amp = np.sqrt(S_ * (S_ + 1) - m_j * (m_j + 1)) * np.sqrt(S_ * (S_ + 1) - m_k * (m_k - 1))
                    new = sub[a].copy()
                    new[j] -= 1
                    new[k] += 1
                    H[pos[int(new @ weights)], a] += 0.5 * J * amp
                # S-_j S+_k
                if cj < d - 1 and ck > 0:
                    amp = np.sqrt(S_ * (S_ + 1) - m_j * (m_j - 1)) * np.sqrt(S_ * (S_ + 1) - m_k * (m_k + 1))
                    new = sub[a].copy()
                    new[j] += 1
                    new[k] -= 1
                    H[pos[int(new @ weights)], a] += 0.5 * J * amp
        E, V = np.linalg.eigh(H)
        sectors.append((E, V, szs))
    return sectors


def thermal(L, beta, S=0.5, J=1.0, sectors=None):
    """E/L, chi(pi), chi(pi + 2 pi / L) and chi(pi, w1), w1 = 2 pi / beta, at
    inverse temperature beta.

    chi(q, w) = (1/(L Z)) sum_mn |<m|M_q|n>|^2 (e^{-beta E_n} - e^{-beta E_m})
                (E_m - E_n) / ((E_m - E_n)^2 + w^2)
    (the Fourier transform over [0, beta) of <M_q(t) M_q(0)> / L at Matsubara
    frequency w; degenerate pairs contribute beta e^{-beta E_n} at w = 0 and
    nothing otherwise)."""
    if sectors is None:
        sectors = spectrum(L, S, J)
    Emin = min(E.min() for E, _, _ in sectors)
    Z = sum(np.exp(-beta * (E - Emin)).sum() for E, _, _ in sectors)
    Eavg = sum((E * np.exp(-beta * (E - Emin))).sum() for E, _, _ in sectors) / Z
    x = np.arange(L)
    out = {"energy": Eavg / L}
    w1 = 2 * np.pi / beta
    for name, q, w in (("chi_s", np.pi, 0.0), ("chi_q", np.pi + 2 * np.pi / L, 0.0), ("chi_w", np.pi, w1)):
        phase = np.exp(1j * q * x)
        tot = 0.0
        for E, V, szs in sectors:
            Mq = szs @ phase  # diagonal of M_q in this sector
            A = V.conj().T @ (Mq[:, None] * V)
            A2 = np.abs(A) ** 2
            Es = E - Emin
            Em = Es[:, None]
            En = Es[None, :]
            dE = Em - En
            wn = np.exp(-beta * En)
            with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
                if w == 0.0:
                    K = np.where(np.abs(dE) > 1e-12, wn * (-np.expm1(-beta * dE)) / np.where(dE == 0, 1, dE),
                                 beta * wn)
                else:
                    K = np.where(np.abs(dE) > 1e-12, wn * (-np.expm1(-beta * dE)) * dE / (dE * dE + w * w),
                                 0.0)
            tot += float((A2 * K).sum())
        out[name] = tot / (L * Z)
    return out


def dimer_closed_form(beta, J=1.0):
    """L=2 periodic S=1/2 chain: H = 2J S1.S2, singlet -3J/2, triplet +J/2."""
    Z = np.exp(1.5 * beta * J) + 3 * np.exp(-0.5 * beta * J)
    E = (-1.5 * J * np.exp(1.5 * beta * J) + 1.5 * J * np.exp(-0.5 * beta * J)) / Z
    chi_s = (np.exp(1.5 * beta * J) - np.exp(-0.5 * beta * J)) / (2 * Z * J)
    # M_pi = S1z - S2z joins the singlet and the triplet m=0 (matrix element 1,
    # gap 2J): chi(pi, w) = (e^{3 beta J/2} - e^{-beta J/2}) 2J / (Z (4J^2 + w^2)).
    w1 = 2 * np.pi / beta
    chi_w = (np.exp(1.5 * beta * J) - np.exp(-0.5 * beta * J)) * 2 * J / (Z * (4 * J * J + w1 * w1))
    return {"energy": E / 2, "chi_s": chi_s, "chi_w": chi_w}


def ring4_closed_form(beta, J=1.0):
    """L=4 periodic S=1/2 ring: H = J (S1+S3).(S2+S4); levels -2J (x1), -J (x3),
    0 (x7), +J (x5)."""
    lv = np.array([-2.0, -1.0, 0.0, 1.0]) * J
    g = np.array([1, 3, 7, 5])
    w = g * np.exp(-beta * lv)
    return {"energy": float((lv * w).sum() / w.sum()) / 4}


def s1_dimer_closed_form(beta, J=1.0):
    """L=2 periodic S=1 chain: H = 2J S1.S2 = J (T(T+1) - 4), T = 0, 1, 2."""
    lv = np.array([-4.0, -2.0, 2.0]) * J
    g = np.array([1, 3, 5])
    w = g * np.exp(-beta * lv)
    return {"energy": float((lv * w).sum() / w.sum()) / 2}


def spin_dimer_closed_form(beta, S, J=1.0):
    """L=2 periodic spin-S chain: two bonds between the same pair, H = 2J S1.S2
    = J (T(T+1) - 2S(S+1)), total spin T = 0 .. 2S with multiplicity 2T+1.
    Energy per site."""
    T = np.arange(0, int(round(2 * S)) + 1)
    lv = J * (T * (T + 1) - 2 * S * (S + 1))
    g = 2 * T + 1
    w = g * np.exp(-beta * (lv - lv.min()))
    return {"energy": float((lv * w).sum() / w.sum()) / 2}
