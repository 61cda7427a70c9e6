"""The subgraph preconditioner and the preconditioned Krylov kernel on the GPU
against the oracle (oracle/krylov.py), for the softened-Coulomb charge model
H[n] = H0 + diag(C (n - Z)).

FP64 (eigenbasis and recursion) within 1e-9; the split-precision density
solves within the 1e-5 scale of their D and D1.
"""

import numpy as np
import pytest
import torch

from oracle import graph_build as o_graph, partition as o_part
from oracle.krylov import charge_hamiltonian, core_jacobians, ground_state_populations, krylov_update
from synth import make_workload, softened_coulomb_matrix, water_box
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


def model(system, seed=3):
    C = softened_coulomb_matrix(system.positions, system.box)
    z = system.z_valence
    rng = np.random.default_rng(seed)
    dq = rng.normal(0.0, 0.05, size=system.n_atoms)
    return C, z, z + dq - dq.mean()


def atom_map(orb_atom):
    order = np.argsort(orb_atom, kind="stable").astype(np.int32)
    ptr = np.concatenate([[0], np.cumsum(np.bincount(orb_atom))]).astype(np.int64)
    return torch.as_tensor(ptr), torch.as_tensor(order)


def blocks_of(K0):
    ap, at, vp, val = (t.cpu().numpy() for t in (K0.atom_ptr, K0.atoms, K0.val_ptr, K0.val))
    out = []
    for k in range(len(ap) - 1):
        na = ap[k + 1] - ap[k]
        out.append((at[ap[k]:ap[k + 1]], val[vp[k]:vp[k] + na * na].reshape(na, na)))
    return out


@pytest.mark.parametrize("name,kT", [("water64", 0.3), ("chains_small", 0.1)])
def test_preconditioner_blocks(gb, name, kT):
    wl, system, _ = make_workload(name, n_rhs=0)
    C, z, n = model(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    adj = o_graph(H.shape[0], H.indptr, H.indices, H.data, wl.tau)
    part = o_part(adj, system.orb_group)
    _, mu = ground_state_populations(H, part, kT, system.n_occ, system.orb_atom, system.n_atoms, workers=4)
    alpha = 0.3
    ref = core_jacobians(H, part, kT, mu, C, system.orb_atom, alpha)
    Hd = gb.DeviceCSR.from_arrays(H.shape[0], H.indptr, H.indices, H.data)
    Cd = gb.DeviceCSR.from_arrays(C.n, C.indptr, C.indices, C.data)
    P = gb.partition(gb.graph_build(Hd, wl.tau), torch.as_tensor(system.orb_group))
    K0 = gb.preconditioner(Hd, P, kT, system.n_electrons, Cd, torch.as_tensor(system.orb_atom), alpha)
    got = blocks_of(K0)
    assert len(got) == len(ref)
    err = 0.0
    for (atoms, k0), (ratoms, _, rk0) in zip(got, ref):
        assert np.array_equal(atoms, ratoms)
        err = max(err, np.abs(k0 - rk0).max())
    print(f"preconditioner {name}: {len(got)} blocks of {min(len(a) for a, _ in got)}-"
          f"{max(len(a) for a, _ in got)} atoms, max|dk0|={err:.2e}, dmu={K0.mu - mu:.2e}")
    assert err <= 1e-9 and abs(K0.mu - mu) < 1e-9


@pytest.mark.parametrize("name,nw,m,precision,tol", [("tiny", 8, 6, "fp64", 1e-9), ("tiny", 8, 6, "eigen", 1e-9),
                                                     ("water64", 64, 4, "fp64", 1e-9),
                                                     ("water64", 64, 4, "fp16x3", 2e-4)])
def test_krylov_update(gb, name, nw, m, precision, tol):
    system = water_box(nw, 77) if name == "tiny" else make_workload(name, n_rhs=0)[1]
    kT = 0.3
    C, z, n = model(system)
    H = charge_hamiltonian(system.H, C, system.orb_atom, z, n)
    adj = o_graph(system.H.n, system.H.indptr, system.H.indices, system.H.data, 1e-5)
    part = o_part(adj, system.orb_group)
    _, mu = ground_state_populations(H, part, kT, system.n_occ, system.orb_atom, system.n_atoms)
    blocks = core_jacobians(H, part, kT, mu, C, system.orb_atom, 0.3)
    ref = krylov_update(system.H, part, kT, system.n_occ, C, system.orb_atom, z, n, blocks, m)
    H0d = to_device(system.H)
    Cd = gb.DeviceCSR.from_arrays(C.n, C.indptr, C.indices, C.data)
    P = gb.partition(gb.graph_build(H0d, 1e-5), torch.as_tensor(system.orb_group))
    Hn = gb.DeviceCSR.from_arrays(H.shape[0], H.indptr, H.indices, H.data)
    oa = torch.as_tensor(system.orb_atom)
    K0 = gb.preconditioner(Hn, P, kT, system.n_electrons, Cd, oa, 0.3)
    aptr, aorb = atom_map(system.orb_atom)
    out = gb.krylov_update(H0d, P, kT, system.n_electrons, Cd, oa, aptr, aorb, torch.as_tensor(z),
                           torch.as_tensor(n), m, K0=K0, precision=precision)
    r = out["rank"]
    assert r == len(ref["v"])
    ef = np.abs(out["f"].cpu().numpy() - ref["f"]).max()
    ev = np.abs(out["v"].cpu().numpy() - ref["v"]).max()
    efv = np.abs(out["fv"].cpu().numpy() - ref["fv"]).max()
    edn = np.abs(out["dn"].cpu().numpy() - ref["dn"]).max()
    print(f"krylov {name} {precision}: rank {r}, max|df|={ef:.2e} |dv|={ev:.2e} |dfv|={efv:.2e} |ddn|={edn:.2e} "
          f"(|dn|={np.abs(ref['dn']).max():.2e})")
    assert ef <= tol and efv <= tol and edn <= tol * max(1.0, np.abs(ref["dn"]).max())
    assert ev <= tol * 10
