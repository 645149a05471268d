"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle on the CPU (a flipped sign, a
dropped term, a wrong convention, a missing factor) and checks that at least
one of the pins of the other test files then fails.  Nothing here touches
the GPU path; the mistakes live only for the duration of a test.
"""
import numpy as np
import pytest

from oracle import bias, dft, filters, lambertw, plc, stats
from tests import (test_oracle_bias as tb, test_oracle_dft as td, test_oracle_filters as tf,
                   test_oracle_lambertw as tl, test_oracle_map as tm,
                   test_oracle_operators as to, test_oracle_stats as ts)


def _fails(check):
    with pytest.raises(AssertionError):
        check()


def test_forward_dft_with_the_inverse_sign(monkeypatch):
    good = dft.dft_axis
    monkeypatch.setattr(dft, "dft_axis", lambda x, axis, sign: good(x, axis, -sign))
    _fails(lambda: td.test_separable_dft_matches_bruteforce((4, 4, 4)))


def test_eigenvalues_with_the_box_and_grid_swapped(monkeypatch):
    # lambda = P L^3 / n^3 instead of P n^3 / L^3
    good = plc.inverse_eigenvalues

    def bad(n, box, k_tab, P_tab, inv_lambda_dc=0.0):
        return good(n, box, k_tab, P_tab, inv_lambda_dc) * (box ** 3 / n ** 3) ** -2
    monkeypatch.setattr(plc, "inverse_eigenvalues", bad)
    _fails(lambda: to.test_single_mode_eigenvalue(8, (2, 3, 1)))


def test_gradient_without_the_prior_term(monkeypatch):
    monkeypatch.setattr(plc, "gradient", lambda s, p: plc.diagonal(s, p) - p.N)
    _fails(lambda: to.test_gradient_matches_finite_differences(True))


def test_gradient_with_the_count_term_of_the_wrong_sign(monkeypatch):
    good = plc.gradient
    monkeypatch.setattr(plc, "gradient", lambda s, p: good(s, p) + 2.0 * p.N)
    _fails(lambda: to.test_gradient_matches_finite_differences(False))
    # and the MAP built on it misses the closed form
    _fails(lambda: tm.test_diagonal_prior_matches_lambert_w(8, 1.5, False))


def test_hessian_without_its_likelihood_diagonal(monkeypatch):
    monkeypatch.setattr(plc, "hessvec", lambda s, v, p: plc.apply_Sinv(v, p.inv_lam))
    _fails(to.test_hessvec_matches_finite_differences_of_gradient)


def test_likelihood_with_a_dropped_selection(monkeypatch):
    # nbar e^s instead of nbar w e^s in the objective only
    good = plc.neg_log_posterior

    def bad(s, p):
        return good(s, p) - float(np.sum(p.wn * np.exp(s))) + float(np.sum(p.nbar * np.exp(s)))
    monkeypatch.setattr(plc, "neg_log_posterior", bad)
    _fails(lambda: to.test_gradient_matches_finite_differences(True))


def test_lambert_w_one_percent_off(monkeypatch):
    good = lambertw.lambertw_from_log
    monkeypatch.setattr(tl, "lambertw_from_log", lambda lx: 1.01 * good(lx))
    _fails(tl.test_log_space_identity_for_huge_arguments)


def test_gaussian_model_with_a_squared_density(monkeypatch):
    # N / (1 + delta)^2 in place of N / (1 + delta) in the gradient
    good = filters.gauss_gradient

    def bad(delta, p):
        u = 1.0 + delta
        occ = p.N > 0
        extra = np.where(occ, p.N / np.where(occ, u, 1.0) - p.N / np.where(occ, u * u, 1.0), 0.0)
        return good(delta, p) + extra
    monkeypatch.setattr(filters, "gauss_gradient", bad)
    _fails(tf.test_gauss_gradient_and_hessian_finite_differences)


def test_bias_applied_as_its_inverse(monkeypatch):
    good = bias.apply_B
    monkeypatch.setattr(bias, "apply_B", lambda x, bk: good(x, 1.0 / bk))
    _fails(lambda: tb.test_constant_bias_diagonal_prior_by_bisection(1.3, 0.7))


def test_correlation_without_the_square_roots(monkeypatch):
    monkeypatch.setattr(stats, "correlation",
                        lambda a, b: float(np.sum(a * b) / (np.sum(a * a) * np.sum(b * b))))
    _fails(ts.test_correlation_and_distance)


def test_bias_hessian_without_its_coupling_term(monkeypatch):
    # drop e^s . B(N/u^2 . B(e^s v)), the term that couples cells through B
    def bad(s, v, q):
        e = np.exp(s)
        u = bias.galaxy_density(s, q)
        return plc.apply_Sinv(v, q.p.inv_lam) + e * bias.apply_B(q.p.wn - q.p.N / u, q.bk) * v
    monkeypatch.setattr(bias, "bias_hessvec", bad)
    _fails(tb.test_gradient_and_hessian_finite_differences)


def _interp_linear_in_k(k, k_tab, P_tab):
    """P linear in k between nodes (instead of linear in (ln k, ln P))."""
    return np.interp(k, k_tab, P_tab)


def _interp_log_p_linear_in_k(k, k_tab, P_tab):
    """ln P linear in k between nodes."""
    return np.exp(np.interp(k, k_tab, np.log(P_tab)))


def _interp_wrong_segment(k, k_tab, P_tab):
    """The right formula on the segment to the left of the right one."""
    k_tab, P_tab, k = (np.asarray(a, dtype=np.float64) for a in (k_tab, P_tab, k))
    j = np.clip(np.searchsorted(k_tab, k, side="right") - 2, 0, k_tab.size - 2)
    t = (np.log(k) - np.log(k_tab[j])) / (np.log(k_tab[j + 1]) - np.log(k_tab[j]))
    return np.exp(np.log(P_tab[j]) + t * (np.log(P_tab[j + 1]) - np.log(P_tab[j])))


@pytest.mark.parametrize("bad", [_interp_linear_in_k, _interp_log_p_linear_in_k, _interp_wrong_segment])
def test_pk_interpolation_mistakes(monkeypatch, bad):
    monkeypatch.setattr(plc, "interp_pk", bad)
    _fails(lambda: to.test_single_mode_between_table_nodes(12, (1, 2, 0), (3, 1, 4), -1.7, 0.6))
