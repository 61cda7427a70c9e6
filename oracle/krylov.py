"""Preconditioned low-rank Krylov approximation of the kernel, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The charge model: a vector n of atomic electron populations acts on the
Hamiltonian through the charge -> potential map C (atoms x atoms),
H[n] = H0 + diag((C (n - Z))_atom(o)), and the ground-state populations are
rho0[n]_I = 2 sum_{o in I} D_oo of D = D_G(H[n]) (the graph method at fixed
electron count).  The residual is f(n) = rho0[n] - n and its Jacobian J.

core_jacobians -- the subgraph preconditioner (Sec. "Preconditioner for a
    partitioned graph"): per subgraph k, the core-atom Jacobian
    j_c = chi + rho_mu mu1^T - I from the canonical responses of the core
    populations to a unit charge on each core atom (d1_lambda, Eq. ddlambda)
    and to mu (d1_mu, Eq. dddmu), with mu1 per column chosen so that every
    column of j_c sums to -1 (charge neutrality of the core), and
    k0 = (j_c - alpha I)^-1 (Eq. PreCond: K0 is their block diagonal).
krylov_update -- the preconditioned Krylov subspace approximation (Sec.
    "Preconditioned Krylov Subspace Approximation for the electronic equations
    of motion", steps 1-5): v_1 = K0 f / |K0 f|; f_v_i = K0 (d rho0 / d lambda
    along v_i - v_i) from the graph response to H1 = diag(C v_i); v_{i+1} from
    f_v_i orthonormalised against v_1..v_i; O = f_v^T f_v, M = O^-1; the update
    dn = -sum_ij v_i M_ij f_v_j^T K0 f (Eqs. LowRankEEOM, Newton_SCF).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fermi import dense_response
from .graph import Partition, gather
from .solve import _to_csr, oracle_graph


def atom_populations(diag: np.ndarray, orb_atom: np.ndarray, n_atoms: int) -> np.ndarray:
    """2 sum_{o in I} D_oo per atom (spin restricted)."""
    return 2.0 * np.bincount(orb_atom, weights=diag, minlength=n_atoms)


def collected_diagonal(csc: tuple) -> np.ndarray:
    """D_jj of a collected matrix (column j holds its own row j)."""
    ptr, idx, val = csc
    col = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    return val[idx == col]


def charge_hamiltonian(H0, C, orb_atom, z, n):
    """H[n] = H0 + diag((C (n - Z))_atom(o))."""
    H0 = _to_csr(H0)
    v = (_to_csr(C) @ (np.asarray(n) - np.asarray(z)))[orb_atom]
    return (H0 + sp.diags(v)).tocsr()


def potential_matrix(C, orb_atom, x):
    """H1[x] = diag((C x)_atom(o)): the perturbation from a charge vector x."""
    return sp.diags((_to_csr(C) @ np.asarray(x))[orb_atom]).tocsr()


def core_atoms(part: Partition, orb_atom: np.ndarray):
    """The atoms of every core (cores hold whole atoms), ascending."""
    return [np.unique(orb_atom[part.core(i)]) for i in range(part.n_sub)]


def core_jacobians(H, part: Partition, kT: float, mu: float, C, orb_atom, alpha: float):
    """[(atoms_k, j_c, k0)] per subgraph at the chemical potential mu."""
    Hc, Cc = _to_csr(H), _to_csr(C).tocsc()
    out = []
    for k in range(part.n_sub):
        S = part.sub(k).astype(np.int64)
        cl = part.local_core(k).astype(np.int64)
        atoms = np.unique(orb_atom[S[cl]])
        eps, V = np.linalg.eigh(gather(Hc, S))
        # responses of the core atoms' populations
        na = len(atoms)
        chi = np.zeros((na, na))
        rho_mu = np.zeros(na)
        owner = np.searchsorted(atoms, orb_atom[S[cl]])      # core orbital -> core atom index
        for b, j in enumerate(atoms):
            u = Cc[:, j].toarray().ravel()[orb_atom[S]]      # potential of a unit charge on atom j
            d1lam, d1mu = dense_response(eps, V, np.diag(u), mu, kT)
            chi[:, b] = 2.0 * np.bincount(owner, weights=np.diag(d1lam)[cl], minlength=na)
        rho_mu = 2.0 * np.bincount(owner, weights=np.diag(d1mu)[cl], minlength=na)
        # mu1 per column: the core populations keep their sum (columns of j_c sum to -1)
        mu1 = -chi.sum(axis=0) / rho_mu.sum()
        jc = chi + np.outer(rho_mu, mu1) - np.eye(na)
        out.append((atoms, jc, np.linalg.inv(jc - alpha * np.eye(na))))
    return out


def apply_preconditioner(blocks, x):
    """K0 x with K0 the block diagonal of the k0 blocks over their core atoms."""
    y = np.zeros_like(np.asarray(x, dtype=np.float64))
    for atoms, _, k0 in blocks:
        y[atoms] = k0 @ np.asarray(x)[atoms]
    return y


def ground_state_populations(H, part, kT, n_occ, orb_atom, n_atoms, workers=0):
    """rho0 of the graph method for H at fixed electron count, and mu."""
    R = oracle_graph(H, [], kT, n_occ, part, workers=workers)
    return atom_populations(collected_diagonal(R.D), orb_atom, n_atoms), R.mu


def krylov_update(H0, part, kT, n_occ, C, orb_atom, z, n, blocks, m, workers=0, breakdown=1e-6):
    """Steps 1-5 of the preconditioned Krylov approximation; see the module doc.

    The expansion stops before m vectors when the subspace is invariant: the
    part of f_v_i orthogonal to v_1..v_i is below `breakdown` times |f_v_i|
    (step 5's "until sufficient convergence")."""
    n = np.asarray(n, dtype=np.float64)
    n_atoms = len(n)
    H = charge_hamiltonian(H0, C, orb_atom, z, n)
    rho0, mu = ground_state_populations(H, part, kT, n_occ, orb_atom, n_atoms, workers)
    f = rho0 - n
    K0f = apply_preconditioner(blocks, f)
    vs, fvs = [], []
    v = K0f / np.linalg.norm(K0f)                                        # step 1
    for i in range(m):
        vs.append(v)
        R = oracle_graph(H, [potential_matrix(C, orb_atom, v)], kT, n_occ, part, workers=workers)   # step 2
        drho = atom_populations(collected_diagonal(R.D1[0]), orb_atom, n_atoms)
        fv = apply_preconditioner(blocks, drho - v)                      # step 3
        fvs.append(fv)
        if i + 1 < m:                                                    # step 4
            # orthonormalised against v_1..v_i: the projection taken twice, so
            # the result is orthogonal to working precision
            w = fv - sum(float(fv @ vj) * vj for vj in vs)
            w = w - sum(float(w @ vj) * vj for vj in vs)
            if np.linalg.norm(w) <= breakdown * np.linalg.norm(fv):
                break
            v = w / np.linalg.norm(w)
    Vm, Fm = np.array(vs), np.array(fvs)
    O = Fm @ Fm.T
    M = np.linalg.inv(O)
    dn = -Vm.T @ (M @ (Fm @ K0f))
    return {"f": f, "rho0": rho0, "mu": mu, "K0f": K0f, "v": Vm, "fv": Fm, "O": O, "M": M, "dn": dn}
