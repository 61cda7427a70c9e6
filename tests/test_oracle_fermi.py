"""Pins of the oracle's scalar and dense-block functions (CPU only).

Each check compares the oracle against something other than itself: a closed
form, a different numerical route (matrix exponential, finite differences,
explicit 2x2 algebra) or a mathematical identity the paper states.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fermi import (dense_density, dense_response, fermi, fermi_divided_difference,
                          fermi_weight, occupation, solve_mu)


def test_fermi_limits_and_symmetry():
    kT = 0.1
    eps = np.array([-1e4, -50.0, -1.0, 0.0, 1.0, 50.0, 1e4])
    f = fermi(eps, 0.0, kT)
    assert np.all(np.isfinite(f))
    assert f[0] == 1.0 and f[-1] == 0.0
    assert f[3] == 0.5
    # particle-hole symmetry f(-x) = 1 - f(x)
    np.testing.assert_allclose(fermi(-eps, 0.0, kT), 1.0 - f, atol=1e-16)
    # closed form where it is safe to evaluate directly
    x = np.linspace(-3, 3, 13)
    np.testing.assert_allclose(fermi(x, 0.2, 0.5), 1.0 / (np.exp((x - 0.2) / 0.5) + 1.0), rtol=1e-14)


def test_fermi_weight_is_f_one_minus_f():
    x = np.linspace(-20, 20, 81)
    # f(1 - f) = f(x) f(-x): both factors evaluated directly, no cancellation
    ref = (1.0 / (np.exp(x) + 1.0)) * (1.0 / (np.exp(-x) + 1.0))
    np.testing.assert_allclose(fermi_weight(x, 0.0, 1.0), ref, rtol=1e-13, atol=1e-300)
    assert np.all(np.isfinite(fermi_weight(np.array([1e5, -1e5]), 0.0, 0.01)))


def test_one_state_chemical_potential_closed_form():
    # one level eps with N_occ in (0, 1): f(eps) = N_occ => mu = eps - kT ln(1/N_occ - 1)
    for eps, nocc, kT in [(-3.0, 0.3, 0.1), (2.5, 0.9, 0.05), (0.0, 0.5, 1.0)]:
        mu, _, resid = solve_mu([np.array([eps])], [np.array([1.0])], nocc, kT)
        assert abs(mu - (eps - kT * np.log(1.0 / nocc - 1.0))) < 1e-12
        assert abs(resid) < 1e-12  # the solver stops at 1e-12 N_occ


def _tanh_2x2(m):
    """tanh of a symmetric 2x2 matrix from its Pauli decomposition (no eigh)."""
    m0 = 0.5 * (m[0, 0] + m[1, 1])
    r = np.hypot(0.5 * (m[0, 0] - m[1, 1]), m[0, 1])
    tp, tm = np.tanh(m0 + r), np.tanh(m0 - r)
    return 0.5 * (tp + tm) * np.eye(2) + 0.5 * (tp - tm) * (m - m0 * np.eye(2)) / r


def test_two_by_two_density_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, c = rng.normal(0, 2, 2)
        b = rng.normal(0, 1)
        H = np.array([[a, b], [b, c]])
        kT, mu = rng.uniform(0.05, 1.0), rng.normal()
        eps, V = np.linalg.eigh(H)
        D = dense_density(eps, V, mu, kT)
        ref = 0.5 * (np.eye(2) - _tanh_2x2((H - mu * np.eye(2)) / (2 * kT)))
        np.testing.assert_allclose(D, ref, atol=1e-14)


def test_density_against_matrix_exponential():
    # D = [exp(beta (H - mu I)) + I]^-1 (Eq. Fermi) through expm and a solve
    rng = np.random.default_rng(2)
    A = rng.normal(size=(7, 7))
    H = 0.5 * (A + A.T)
    kT, mu = 0.7, 0.3
    eps, V = np.linalg.eigh(H)
    ref = np.linalg.inv(sla.expm((H - mu * np.eye(7)) / kT) + np.eye(7))
    np.testing.assert_allclose(dense_density(eps, V, mu, kT), ref, atol=1e-12)


def test_divided_difference_off_diagonal_and_diagonal():
    eps = np.array([-2.0, -1.5, -0.2, 0.01, 0.6, 3.0])
    kT, mu = 0.25, 0.0
    F = fermi_divided_difference(eps, mu, kT)
    f = fermi(eps, mu, kT)
    for k in range(len(eps)):
        for l in range(len(eps)):
            if k != l:
                assert abs(F[k, l] - (f[k] - f[l]) / (eps[k] - eps[l])) < 1e-12
    np.testing.assert_allclose(np.diag(F), -fermi_weight(eps, mu, kT) / kT, rtol=1e-13)
    # continuity through near-degenerate pairs: no threshold, no jump
    e2 = np.array([0.3, 0.3 + 1e-9, 0.3 + 1e-5])
    F2 = fermi_divided_difference(e2, 0.0, kT)
    assert abs(F2[0, 1] - F2[0, 0]) < 1e-7
    # no overflow far from mu
    F3 = fermi_divided_difference(np.array([-500.0, 0.0, 500.0]), 0.0, 0.01)
    assert np.all(np.isfinite(F3))
    assert abs(F3[0, 2] - (1.0 - 0.0) / (-1000.0)) < 1e-15


def test_grand_canonical_response_is_derivative():
    # d1_lambda = d/dlambda Theta(mu - h - lambda h1) at fixed mu (Eq. ddlambda)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(9, 9))
    h = 0.5 * (A + A.T)
    B = rng.normal(size=(9, 9))
    h1 = 0.5 * (B + B.T)
    kT, mu, e = 0.3, 0.1, 1e-5
    eps, V = np.linalg.eigh(h)
    d1lam, d1mu = dense_response(eps, V, h1, mu, kT)

    def dens(m, mu_):
        ee, vv = np.linalg.eigh(m)
        return dense_density(ee, vv, mu_, kT)

    fd = (dens(h + e * h1, mu) - dens(h - e * h1, mu)) / (2 * e)
    np.testing.assert_allclose(d1lam, fd, atol=1e-8)
    # d1_mu = beta d (I - d) = dD/dmu (Eq. dddmu)
    fdmu = (dens(h, mu + e) - dens(h, mu - e)) / (2 * e)
    np.testing.assert_allclose(d1mu, fdmu, atol=1e-8)
    d = dens(h, mu)
    np.testing.assert_allclose(d1mu, d @ (np.eye(9) - d) / kT, atol=1e-12)


def test_newton_converges_quadratically():
    rng = np.random.default_rng(4)
    eps_list = [np.sort(rng.normal(0, 1.0, 30)) for _ in range(5)]
    w_list = [rng.uniform(0.1, 1.0, 30) for _ in range(5)]
    kT, nocc = 0.2, 40.0
    mu_star, _, _ = solve_mu(eps_list, w_list, nocc, kT)
    # Newton-Raphson iterates from a nearby start (Eq. NewtonRaphson)
    mu = mu_star + 0.05
    errs = []
    for _ in range(4):
        n, dn = occupation(mu, eps_list, w_list, kT)
        mu = mu - (n - nocc) / dn
        errs.append(abs(mu - mu_star))
    assert errs[2] < 1e-9
    assert errs[1] < 10.0 * errs[0] ** 2 + 1e-14
