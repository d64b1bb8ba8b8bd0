"""Pins of the exact-diagonalization oracle against closed forms."""
import numpy as np
import pytest

from oracle import ed


@pytest.mark.parametrize("beta", [0.25, 1.0, 4.0, 16.0])
def test_dimer(beta):
    t = ed.thermal(2, beta)
    c = ed.dimer_closed_form(beta)
    assert t["energy"] == pytest.approx(c["energy"], rel=1e-12, abs=1e-14)
    assert t["chi_s"] == pytest.approx(c["chi_s"], rel=1e-12)
    assert t["chi_w"] == pytest.approx(c["chi_w"], rel=1e-12)


@pytest.mark.parametrize("L,beta", [(6, 2.0), (8, 8.0)])
def test_chi_w_bounds(L, beta):
    # spectral weights are positive: 0 < chi(pi, w1) < chi(pi, 0); at low T
    # the ratio approaches the single-gap Lorentzian.
    t = ed.thermal(L, beta)
    assert 0 < t["chi_w"] < t["chi_s"]


@pytest.mark.parametrize("beta", [0.5, 2.0, 8.0])
def test_ring4(beta):
    assert ed.thermal(4, beta)["energy"] == pytest.approx(ed.ring4_closed_form(beta)["energy"], rel=1e-12)


@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_s1_dimer(beta):
    assert ed.thermal(2, beta, S=1.0)["energy"] == pytest.approx(ed.s1_dimer_closed_form(beta)["energy"],
                                                                 rel=1e-12)


@pytest.mark.parametrize("S", [0.5, 1.0, 1.5, 2.0])
@pytest.mark.parametrize("beta", [0.3, 1.0, 4.0])
def test_spin_dimer_closed_form(S, beta):
    # the L = 2 spectrum from the total spin of two spins S
    assert ed.thermal(2, beta, S=S)["energy"] == pytest.approx(ed.spin_dimer_closed_form(beta, S)["energy"],
                                                               rel=1e-12)


@pytest.mark.parametrize("L,S", [(8, 0.5), (6, 1.0), (4, 1.5), (4, 2.0)])
def test_curie_limit(L, S):
    # beta -> 0: chi(q) -> beta S(S+1)/3 for every q.
    beta = 1e-4
    t = ed.thermal(L, beta, S=S)
    assert t["chi_s"] == pytest.approx(beta * S * (S + 1) / 3, rel=1e-3)
    assert t["chi_q"] == pytest.approx(beta * S * (S + 1) / 3, rel=1e-3)
    # leading high-temperature term: E/L = -beta <(S_i.S_j)^2> = -beta (S(S+1))^2 / 3
    assert t["energy"] == pytest.approx(-beta * (S * (S + 1)) ** 2 / 3, rel=1e-3)


def test_coupling_scale():
    # E(beta, J) = J E(beta J, 1); chi(beta, J) = chi(beta J, 1) / J.
    a = ed.thermal(6, 2.0, J=0.5)
    b = ed.thermal(6, 1.0, J=1.0)
    assert a["energy"] == pytest.approx(0.5 * b["energy"], rel=1e-12)
    assert a["chi_s"] == pytest.approx(b["chi_s"] / 0.5, rel=1e-12)
