"""Mulliken charges q and their responses q1 on the GPU against the oracle.

q_I = Z_I - 2 sum_{o in I} D_oo and q1_I = -2 sum_{o in I} D1_oo from the
collected matrices (Sec. "Response in observables").  FP64 path within 1e-9;
split precision within 2 x (orbitals per atom) x 1e-5, the bound that D's own
1e-5 tolerance implies.
"""

import numpy as np
import pytest
import torch

from oracle import graph_build as o_graph, oracle_graph, partition as o_part
from oracle.graph import csc_to_dense
from oracle.solve import mulliken_charges
from synth import make_workload
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


def atom_map(orb_atom):
    order = np.argsort(orb_atom, kind="stable").astype(np.int32)
    ptr = np.concatenate([[0], np.cumsum(np.bincount(orb_atom))]).astype(np.int64)
    return torch.as_tensor(ptr), torch.as_tensor(order)


@pytest.mark.parametrize("name,precision", [("water64", "fp64"), ("water64", "fp16x3"), ("water1k", "fp16x3"),
                                            ("chains_small", "fp16x3")])
def test_mulliken_parity(gb, name, precision):
    wl, system, h1 = make_workload(name, n_rhs=2)
    H = system.H
    adj = o_graph(H.n, H.indptr, H.indices, H.data, wl.tau)
    part = o_part(adj, system.orb_group)
    ref = oracle_graph(H, h1, wl.kT, system.n_occ, part, workers=4)
    z = system.z_valence
    dref = np.diag(csc_to_dense(H.n, *ref.D))
    qref = mulliken_charges(dref, system.orb_atom, z)
    q1ref = [mulliken_charges(np.diag(csc_to_dense(H.n, *r)), system.orb_atom, np.zeros_like(z)) for r in ref.D1]
    Hd = to_device(H)
    P = gb.partition(gb.graph_build(Hd, wl.tau), torch.as_tensor(system.orb_group))
    R = gb.density_and_response(Hd, [to_device(h) for h in h1], wl.kT, system.n_electrons, P,
                                precision=precision, mu0=ref.mu)
    aptr, aorb = atom_map(system.orb_atom)
    q, q1 = gb.mulliken_charges(R.D, R.D1, aptr, aorb, torch.as_tensor(z))
    q, q1 = q.cpu().numpy(), [x.cpu().numpy() for x in q1]
    eq = np.abs(q - qref).max()
    eq1 = max(np.abs(a - b).max() for a, b in zip(q1, q1ref))
    per_atom = np.bincount(system.orb_atom).max()
    tol = 1e-9 if precision == "fp64" else 2 * per_atom * 1e-5
    print(f"{name} {precision}: max|dq|={eq:.2e} max|dq1|={eq1:.2e} (bound {tol:.0e}) sum q={q.sum():.2e}")
    assert eq <= tol and eq1 <= tol
    # neutral system: the charges sum to -2 (Tr D - N_occ)
    assert abs(q.sum() + 2 * R.report["occ_residual"]) < 1e-8


def test_mulliken_errors(gb):
    wl, system, h1 = make_workload("water64", n_rhs=0)
    Hd = to_device(system.H)
    P = gb.partition(gb.graph_build(Hd, wl.tau), torch.as_tensor(system.orb_group))
    R = gb.density_and_response(Hd, [], wl.kT, system.n_electrons, P)
    aptr, aorb = atom_map(system.orb_atom)
    bad = aorb.clone()
    bad[3] = system.H.n + 5  # an orbital out of range
    with pytest.raises(gb.GbError) as e:
        gb.mulliken_charges(R.D, [], aptr, bad, torch.as_tensor(system.z_valence))
    assert e.value.status == 1
