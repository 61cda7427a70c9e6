"""Pins of the oracle's subgraph preconditioner and Krylov kernel
(oracle/krylov.py) against finite differences of the residual itself.

A tiny periodic water box (8 waters, 24 atoms, 48 orbitals) with the softened
Coulomb charge model: H[n] = H0 + diag(C (n - Z)).  The Jacobian of
f(n) = rho0[n] - n is taken by central differences of the full calculation at
fixed electron count, independently of the response formulas.
"""

import numpy as np
import pytest

from oracle import graph_build, partition
from oracle.krylov import (apply_preconditioner, charge_hamiltonian, core_jacobians, ground_state_populations,
                           krylov_update)
from oracle.graph import Partition
from synth import softened_coulomb_matrix, water_box

KT = 0.3


def krylov_model():
    """8 waters with the softened Coulomb charge model and off-neutral populations."""
    system = water_box(8, 77)
    C = softened_coulomb_matrix(system.positions, system.box)
    z = system.z_valence
    rng = np.random.default_rng(3)
    dq = rng.normal(0.0, 0.05, size=system.n_atoms)
    n = z + dq - dq.mean()
    return system, C, z, n


@pytest.fixture(scope="module")
def model():
    return krylov_model()


def residual(system, C, z, part, n):
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    rho, _ = ground_state_populations(H, part, KT, system.n_occ, system.orb_atom, system.n_atoms)
    return rho - n


def fd_jacobian(system, C, z, part, n, eps=1e-4):
    cols = []
    for j in range(len(n)):
        e = np.zeros_like(n)
        e[j] = eps
        cols.append((residual(system, C, z, part, n + e) - residual(system, C, z, part, n - e)) / (2 * eps))
    return np.array(cols).T


def single_part(system):
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, 0.0)
    return partition(adj, np.zeros(H.n, dtype=np.int32))


def molecule_part(system):
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, 1e-5)
    return partition(adj, system.orb_group)


def test_single_core_jacobian_is_the_full_jacobian(model):
    # one core holding every atom: j_c is the Jacobian of the residual
    system, C, z, n = model
    part = single_part(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    _, mu = ground_state_populations(H, part, KT, system.n_occ, system.orb_atom, system.n_atoms)
    (atoms, jc, k0), = core_jacobians(H, part, KT, mu, C, system.orb_atom, 0.0)
    J = fd_jacobian(system, C, z, part, n)
    assert np.array_equal(atoms, np.arange(system.n_atoms))
    assert np.abs(jc - J).max() < 1e-6
    assert np.abs(jc.sum(axis=0) + 1.0).max() < 1e-10


def test_subgraph_blocks_are_charge_neutral_and_inverted(model):
    system, C, z, n = model
    part = molecule_part(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    _, mu = ground_state_populations(H, part, KT, system.n_occ, system.orb_atom, system.n_atoms)
    alpha = 0.3
    blocks = core_jacobians(H, part, KT, mu, C, system.orb_atom, alpha)
    assert len(blocks) == 8 and sorted(np.concatenate([b[0] for b in blocks])) == list(range(system.n_atoms))
    for atoms, jc, k0 in blocks:
        assert len(atoms) == 3
        assert np.abs(jc.sum(axis=0) + 1.0).max() < 1e-10   # the core keeps its charge
        assert np.abs(k0 @ (jc - alpha * np.eye(3)) - np.eye(3)).max() < 1e-12
        # off the diagonal the response is the susceptibility (it does not vanish)
        assert np.abs(jc + np.eye(3)).max() > 1e-3
    # K0 is the block diagonal of the k0 blocks over their core atoms (Eq.
    # PreCond), applied as a matrix: against the assembled dense K0
    K0 = np.zeros((system.n_atoms, system.n_atoms))
    for atoms, _, k0 in blocks:
        K0[np.ix_(atoms, atoms)] = k0
    x = np.random.default_rng(4).normal(size=system.n_atoms)
    assert np.abs(apply_preconditioner(blocks, x) - K0 @ x).max() < 1e-12


def test_krylov_directional_derivatives(model):
    # f_v = K0 J v for the graph method's own Jacobian (finite differences)
    system, C, z, n = model
    part = molecule_part(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    _, mu = ground_state_populations(H, part, KT, system.n_occ, system.orb_atom, system.n_atoms)
    blocks = core_jacobians(H, part, KT, mu, C, system.orb_atom, 0.3)
    out = krylov_update(system.H, part, KT, system.n_occ, C, system.orb_atom, z, n, blocks, 4)
    J = fd_jacobian(system, C, z, part, n)
    for v, fv in zip(out["v"], out["fv"]):
        assert np.abs(fv - apply_preconditioner(blocks, J @ v)).max() < 1e-6
    assert np.abs(out["v"] @ out["v"].T - np.eye(4)).max() < 1e-12
    assert np.abs(out["f"] - residual(system, C, z, part, n)).max() < 1e-12


def test_full_rank_krylov_is_the_newton_step(model):
    # The residual and every Krylov vector sum to zero (the electron count is
    # fixed and the columns of each k0 keep it), so at most N - 1 vectors; the
    # expansion stops when the subspace is invariant under K0 J, where
    # sum v_i M_ij f_v_j^T acts as (K0 J)^-1 and dn = -J^-1 f (Newton step)
    system, C, z, n = model
    part = single_part(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    _, mu = ground_state_populations(H, part, KT, system.n_occ, system.orb_atom, system.n_atoms)
    blocks = core_jacobians(H, part, KT, mu, C, system.orb_atom, 0.2)
    out = krylov_update(system.H, part, KT, system.n_occ, C, system.orb_atom, z, n, blocks, system.n_atoms - 1)
    J = fd_jacobian(system, C, z, part, n)
    newton = -np.linalg.solve(J, out["f"])
    assert abs(out["f"].sum()) < 1e-10 and abs(out["v"].sum(axis=1)).max() < 1e-10
    k = len(out["v"])
    assert 1 < k <= system.n_atoms - 1
    assert np.abs(out["v"] @ out["v"].T - np.eye(k)).max() < 1e-8
    assert np.abs(out["dn"] - newton).max() < 1e-6 * max(1.0, np.abs(newton).max())
