"""Full and graph-based FP64 solutions for D, D1, mu and mu_1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

oracle_full -- the whole H diagonalised once: D = V f V^T with Tr D = N_occ,
    D1 = d1_lambda + mu_1 d1_mu with mu_1 = -Tr d1_lambda / Tr d1_mu
    (Eqs. D1_a, D1_b, dddmu and the Tr D1 = 0 condition).
oracle_graph -- the graph method itself: per-subgraph diagonalisation of
    h^(i) = H[S_i, S_i] (Eq. SmallKS), one mu shared by all subgraphs from the
    core-weighted occupation sum (Eq. NewtonRaphson and the terms after it),
    core columns of d^(i) collected (Eqs. DD0, DD), and the graph response of
    Eq. D1 with d1_lambda^(i) (Eq. ddlambda), d1_mu^(i) (Eq. dddmu) and the
    global mu_1 of Eq. dmu_1 (core traces summed over all subgraphs).
"""

from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .fermi import dense_density, dense_response, fermi, fermi_weight, solve_mu
from .graph import Partition, collect_columns, gather


@dataclass
class FullResult:
    D: np.ndarray
    D1: list
    mu: float
    mu1: np.ndarray
    eps: np.ndarray
    d1lam: list
    d1mu: np.ndarray


def oracle_full(H: np.ndarray, h1_list, kT: float, n_occ: float) -> FullResult:
    """D, D1, mu, mu_1 of the whole system by one dense diagonalisation."""
    H = np.asarray(H, dtype=np.float64)
    eps, V = np.linalg.eigh(H)
    mu, _, _ = solve_mu([eps], [np.ones_like(eps)], n_occ, kT)
    D = dense_density(eps, V, mu, kT)
    D1, mu1, d1lams = [], [], []
    d1mu = None
    for h1 in h1_list:
        h1 = np.asarray(h1, dtype=np.float64)
        d1lam, d1mu = dense_response(eps, V, h1, mu, kT)
        m1 = -np.trace(d1lam) / np.trace(d1mu)
        D1.append(d1lam + m1 * d1mu)
        mu1.append(m1)
        d1lams.append(d1lam)
    return FullResult(D, D1, mu, np.array(mu1), eps, d1lams, d1mu)


@dataclass
class GraphResult:
    mu: float
    mu1: np.ndarray
    D: tuple                      # ragged CSC (col_ptr, row_idx, val)
    D1: list                      # one ragged CSC per right-hand side
    trace_core: float             # sum_i Tr_c d^(i)
    trace_core_dd: float          # sum_i Tr_c d^(i)(I - d^(i))
    trace_d1lam: np.ndarray       # sum_i Tr_c d1_lambda^(i), per RHS
    trace_d1mu: float             # sum_i Tr_c d1_mu^(i)
    n_newton: int
    residual: float               # Tr D - N_occ at the returned mu
    spectra: list = field(default_factory=list)   # (eps, w) per subgraph
    blocks: dict = field(default_factory=dict)    # subgraph -> (d_c, [d1_c], d1mu_c)


def _to_csr(m):
    if sp.issparse(m):
        return m.tocsr()
    n, indptr, indices, data = m.n, m.indptr, m.indices, m.data
    return sp.csr_matrix((data, indices, indptr), shape=(n, n))


def _spectrum_task(args):
    h, core_local = args
    eps, V = np.linalg.eigh(h)
    w = np.sum(V[core_local, :] ** 2, axis=0)
    return eps, V, w


def _response_task(args):
    eps, V, h1s, core_local, mu, kT = args
    f = fermi(eps, mu, kT)
    d_c = (V * f) @ V[core_local, :].T
    d1_c, tr1 = [], []
    d1mu_c = None
    for h1 in h1s:
        d1lam, d1mu = dense_response(eps, V, h1, mu, kT)
        d1_c.append(d1lam[:, core_local])
        tr1.append(float(np.trace(d1lam[np.ix_(core_local, core_local)])))
        d1mu_c = d1mu[:, core_local]
    if d1mu_c is None:
        d1mu_c = (V * (fermi_weight(eps, mu, kT) / kT)) @ V[core_local, :].T
    tr_mu = float(np.trace(d1mu_c[core_local, :]))
    return d_c, d1_c, d1mu_c, np.array(tr1), tr_mu


def _map(fn, items, workers):
    if workers and workers > 1 and len(items) > 4 * workers:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(fn, items, chunksize=max(1, len(items) // (8 * workers))))
    return [fn(it) for it in items]


def oracle_graph(H, h1_list, kT: float, n_occ: float, part: Partition, *,
                 keep=None, workers: int = 0, mu0=None) -> GraphResult:
    """The graph-based D, D1, mu and mu_1 (Eqs. DD, NewtonRaphson, D1, dmu_1).

    ``keep``: subgraph indices whose core-column blocks are returned in
    ``blocks``; ``None`` collects every subgraph into global ragged CSC
    matrices, an empty list collects none (mu and mu_1 still use all).
    """
    Hc = _to_csr(H)
    h1c = [_to_csr(h) for h in h1_list]
    subs = [part.sub(i).astype(np.int64) for i in range(part.n_sub)]
    cores = [part.local_core(i).astype(np.int64) for i in range(part.n_sub)]
    spectra = _map(_spectrum_task, [(gather(Hc, s), c) for s, c in zip(subs, cores)], workers)
    eps_list = [e for e, _, _ in spectra]
    w_list = [w for _, _, w in spectra]
    mu, n_newton, resid = solve_mu(eps_list, w_list, n_occ, kT, mu0=mu0)
    tr_d = sum(float(np.dot(fermi(e, mu, kT), w)) for e, w in zip(eps_list, w_list))
    tr_dd = sum(float(np.dot(fermi_weight(e, mu, kT), w)) for e, w in zip(eps_list, w_list))
    items = [(e, V, [gather(h, s) for h in h1c], c, mu, kT)
             for (e, V, _), s, c in zip(spectra, subs, cores)]
    resp = _map(_response_task, items, workers)
    m = len(h1c)
    tr1 = np.zeros(m)
    tr_mu = 0.0
    for r in resp:
        tr1 += r[3]
        tr_mu += r[4]
    mu1 = -tr1 / tr_mu if m else np.zeros(0)
    collect_all = keep is None
    keep_set = set(range(part.n_sub)) if collect_all else set(keep)
    blocks = {}
    for i in keep_set:
        d_c, d1_c, d1mu_c, _, _ = resp[i]
        blocks[i] = (d_c, [d1_c[r] + mu1[r] * d1mu_c for r in range(m)], d1mu_c)
    D = D1 = None
    if collect_all:
        D = collect_columns([blocks[i][0] for i in range(part.n_sub)], part)
        D1 = [collect_columns([blocks[i][1][r] for i in range(part.n_sub)], part)
              for r in range(m)]
    return GraphResult(mu=mu, mu1=mu1, D=D, D1=D1 or [], trace_core=tr_d,
                       trace_core_dd=tr_dd, trace_d1lam=tr1, trace_d1mu=tr_mu,
                       n_newton=n_newton, residual=resid,
                       spectra=list(zip(eps_list, w_list)), blocks=blocks)


def mulliken_charges(diag: np.ndarray, orb_atom: np.ndarray, z_val: np.ndarray) -> np.ndarray:
    """q_I = Z_I - 2 sum_{o in I} D_oo (spin-restricted Mulliken net charge)."""
    pop = np.zeros(len(z_val))
    np.add.at(pop, orb_atom, 2.0 * diag)
    return z_val - pop
