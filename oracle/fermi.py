"""Fermi-Dirac occupations, the chemical potential and the canonical response.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain float64 numpy.

Notation follows the paper: beta = 1 / kT, occupation
f_k = [exp(beta (eps_k - mu)) + 1]^-1 (Eq. Fermi / the occupation factors
after Eq. NewtonRaphson), D = sum_k f_k v_k v_k^T (Eq. DD).
"""

from __future__ import annotations

import numpy as np
from scipy.special import expit


def fermi(eps, mu, kT):
    """f = [exp(beta (eps - mu)) + 1]^-1, evaluated without overflow."""
    return expit(-(np.asarray(eps, dtype=np.float64) - mu) / kT)


def fermi_weight(eps, mu, kT):
    """f (1 - f) = exp(-|x|) / (1 + exp(-|x|))^2 with x = beta (eps - mu).

    This is the factor of the Newton-Raphson denominator and of
    d1_mu = beta d (I - d) (Eq. dddmu), written so it never cancels.
    """
    x = np.abs((np.asarray(eps, dtype=np.float64) - mu) / kT)
    e = np.exp(-x)
    return e / (1.0 + e) ** 2


def fermi_divided_difference(eps, mu, kT):
    """F_kl = (f_k - f_l) / (eps_k - eps_l), F_kk = -beta f_k (1 - f_k).

    This is the kernel of the first derivative of the matrix function
    Theta_beta(mu I - H) along H1 (Eq. ddlambda): in the eigenbasis of H,
    dD/dlambda = V (F o (V^T H1 V)) V^T.  With f = 1/2 - tanh(x/2)/2 and
    tanh(a) - tanh(b) = sinh(a - b) / (cosh a cosh b):

        F_kl = -(beta / 4) sinh(y) / (y cosh(a) cosh(b)),
        a = x_k / 2,  b = x_l / 2,  y = a - b,

    evaluated in the overflow-free form
        sinh(y) / (y cosh a cosh b)
          = [-expm1(-2|y|) / (2|y|)] * 4 exp(|y| - |a| - |b|)
            / ((1 + exp(-2|a|)) (1 + exp(-2|b|))),
    whose y -> 0 limit gives the diagonal -beta f (1 - f) with no
    degeneracy threshold.
    """
    beta = 1.0 / kT
    x = (np.asarray(eps, dtype=np.float64) - mu) * beta
    a = 0.5 * x[:, None]
    b = 0.5 * x[None, :]
    y = np.abs(a - b)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = np.where(y > 0.0, -np.expm1(-2.0 * y) / (2.0 * y), 1.0)
    aa, bb = np.abs(a), np.abs(b)
    core = 4.0 * np.exp(y - aa - bb) / ((1.0 + np.exp(-2.0 * aa)) * (1.0 + np.exp(-2.0 * bb)))
    return -(beta / 4.0) * ratio * core


def occupation(mu, eps_list, w_list, kT):
    """N(mu) = sum_i sum_k f(eps_k^(i)) w_k^(i)  and  dN/dmu = beta sum f(1-f) w."""
    n = 0.0
    dn = 0.0
    for eps, w in zip(eps_list, w_list):
        n += float(np.dot(fermi(eps, mu, kT), w))
        dn += float(np.dot(fermi_weight(eps, mu, kT), w))
    return n, dn / kT


def solve_mu(eps_list, w_list, n_occ, kT, *, mu0=None, tol=1e-12, max_newton=60,
             bracket_width=1e-13):
    """Shared chemical potential from Tr[D_G(mu)] = N_occ (Eq. NewtonRaphson).

    ``eps_list[i]`` are the eigenvalues of subgraph i and ``w_list[i]`` the
    core weights w_k = sum_{j in core} v_kj^2 (the squared core parts of the
    eigenvectors, the terms after Eq. d_Collect).  N(mu) increases with mu, so
    a bisection bracket [eps_min - 40 kT, eps_max + 40 kT] is shrunk until it
    is narrow, then Newton-Raphson steps
        mu <- mu - (N(mu) - N_occ) / (beta sum f (1 - f) w)
    polish the root while they stay inside the bracket.
    Returns (mu, n_newton_steps, N(mu) - N_occ).
    """
    lo = min(float(np.min(e)) for e in eps_list if len(e)) - 40.0 * kT
    hi = max(float(np.max(e)) for e in eps_list if len(e)) + 40.0 * kT
    n_lo, _ = occupation(lo, eps_list, w_list, kT)
    n_hi, _ = occupation(hi, eps_list, w_list, kT)
    if not (n_lo <= n_occ <= n_hi):
        raise ValueError(f"N_occ={n_occ} outside [{n_lo}, {n_hi}]")
    while hi - lo > bracket_width * max(1.0, abs(lo), abs(hi)):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        n_mid, _ = occupation(mid, eps_list, w_list, kT)
        if n_mid < n_occ:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi) if mu0 is None or not (lo <= mu0 <= hi) else mu0
    steps = 0
    n, dn = occupation(mu, eps_list, w_list, kT)
    for _ in range(max_newton):
        if abs(n - n_occ) <= tol * max(1.0, n_occ) or dn <= 0.0:
            break
        nxt = mu - (n - n_occ) / dn
        if not (lo <= nxt <= hi) or nxt == mu:
            break
        mu = nxt
        steps += 1
        n, dn = occupation(mu, eps_list, w_list, kT)
    return mu, steps, n - n_occ


def dense_density(eps, V, mu, kT):
    """d = V diag(f) V^T (Eq. DD before the core restriction)."""
    return (V * fermi(eps, mu, kT)) @ V.T


def dense_response(eps, V, h1, mu, kT):
    """Grand-canonical response and mu-response of one dense block.

    d1_lambda = V (F o (V^T h1 V)) V^T   (Eq. ddlambda, F from
                fermi_divided_difference)
    d1_mu     = beta d (I - d) = V diag(beta f (1 - f)) V^T   (Eq. dddmu)
    """
    h1p = V.T @ h1 @ V
    F = fermi_divided_difference(eps, mu, kT)
    d1lam = V @ (F * h1p) @ V.T
    d1mu = (V * (fermi_weight(eps, mu, kT) / kT)) @ V.T
    return d1lam, d1mu
