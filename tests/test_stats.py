"""Pins of the error analysis (binning, jackknife) and of the derived
estimators (xi, xi_tau) against exact diagonalization."""
import math

import numpy as np
import pytest

from oracle import ed, stats


def test_jackknife_of_linear_function_is_binned_error():
    # for f(a) = a the jackknife error equals the standard error of the bin means
    x = np.random.default_rng(1).normal(size=10000)
    m, e = stats.mean_err(x, 40)
    v, je = stats.jackknife(lambda a: a, x, nbins=40)
    assert v == pytest.approx(m, rel=1e-12) and je == pytest.approx(e, rel=1e-10)


def test_jackknife_ratio_matches_delta_method():
    # independent X ~ N(2, 1), Y ~ N(4, 1): var(mean X / mean Y) by the delta method
    rng = np.random.default_rng(2)
    n = 200000
    x, y = rng.normal(2.0, 1.0, n), rng.normal(4.0, 1.0, n)
    v, je = stats.jackknife(lambda a, b: a / b, x, y, nbins=100)
    mx, my = 2.0, 4.0
    delta = math.sqrt((1.0 / my) ** 2 / n + (mx / my ** 2) ** 2 / n)
    assert v == pytest.approx(0.5, abs=5 * delta)
    assert je == pytest.approx(delta, rel=0.25)


@pytest.mark.parametrize("L,beta,Q", [(8, 4.0, 1), (4, 2.0, 2)])
def test_xi_and_xi_tau_vs_ed(orc, L, beta, Q):
    # ratio-of-means estimators with jackknife errors, against the same
    # functions of the exact chi(pi), chi(pi + 2 pi / L), chi(pi, 2 pi / beta)
    p = orc.params(L, beta, Q=Q, seed=41)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 500, st)
    r = orc.keyed_run(p, 500, 200000, st)
    ex = ed.thermal(L, beta, S=Q / 2)
    xi, xe = stats.jackknife(stats.xi_second_moment(L), r["chi_s"], r["chi_q"], nbins=100)
    xt, te = stats.jackknife(stats.xi_tau(beta), r["chi_s"], r["chi_w"], nbins=100)
    assert stats.within_sigma(xi, xe, stats.xi_second_moment(L)(ex["chi_s"], ex["chi_q"]), 3.0)
    assert stats.within_sigma(xt, te, stats.xi_tau(beta)(ex["chi_s"], ex["chi_w"]), 3.0)
