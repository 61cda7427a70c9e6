"""The adaptive graph loop along a trajectory (Sec. "Estimating the
connectivity graph"): at every geometry the graph is estimated again from the
previous step's density matrix and the new H, the partition and the size-class
plan follow it, and D, D1 are solved on it.

Per step: the graph is bit-exact against the oracle's graph built from the same
previous D; D and D1 are within the path's tolerance of the oracle on that
graph; the plan is re-tuned when the subgraph sizes change.
"""

import dataclasses

import numpy as np
import pytest
import torch

from oracle import graph_build as o_graph, oracle_graph, partition as o_part
from synth import make_workload
from synth.water import tb_hamiltonian, thermal_trajectory, water_perturbation
from tests.helpers import max_abs_block_error, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp16x3", 1e-5)])
def test_graph_follows_the_previous_density(gb, precision, tol):
    wl, system, _ = make_workload("water1k", n_rhs=0)
    tau = 1e-5
    groups = torch.as_tensor(system.orb_group)
    h = gb.Handle(device="cuda")
    d_prev = None
    mu = float("nan")
    last_key = None
    for k, pos in enumerate(thermal_trajectory(system, 3, seed=20221204 + 1000)):
        H, _ = tb_hamiltonian(pos, system.species, system.box)
        moved = dataclasses.replace(system, positions=pos, H=H)
        h1 = [water_perturbation(moved, 20221204 + 1000 * (k + 1))]
        Hd = to_device(H)
        G = gb.graph_build(Hd, tau, d_prev=d_prev, handle=h)
        # the oracle's graph from the same H and the same previous D
        dp = None if d_prev is None else (d_prev.ptr.cpu().numpy(), d_prev.idx.cpu().numpy(),
                                          d_prev.val.cpu().numpy())
        adj = o_graph(H.n, H.indptr, H.indices, H.data, tau, d_prev=dp)
        assert np.array_equal(G.ptr.cpu().numpy(), adj.indptr)
        assert np.array_equal(G.idx.cpu().numpy(), adj.indices)
        P = gb.partition(G, groups, handle=h)
        part = o_part(adj, system.orb_group)
        assert np.array_equal(P.sub_idx.cpu().numpy(), part.sub_idx)
        if precision != "fp64":
            plan = gb.plan_autotune(Hd, [to_device(h1[0])], wl.kT, system.n_electrons, P,
                                    mu if mu == mu else -7.5, handle=h)
            key = (P.n_sub, P.sub_nnz)
            assert plan["cached"] == (key == last_key)
            last_key = key
            small = plan["split_small_npad"]
        else:
            small = 0
        ref = oracle_graph(H, h1, wl.kT, system.n_occ, part, workers=4)
        R = gb.density_and_response(Hd, [to_device(h1[0])], wl.kT, system.n_electrons, P, precision=precision,
                                    mu0=mu, split_small_npad=small, handle=h)
        eD, eD1 = max_abs_block_error(R, ref, part)
        print(f"step {k} {precision}: edges {G.nnz} sub_nnz {P.sub_nnz} max_sub {P.max_sub} "
              f"max|dD|={eD:.2e} max|dD1|={eD1:.2e} passes={R.report['passes']}")
        assert eD <= tol and eD1 <= tol
        d_prev, mu = R.D, R.mu
    # the graph grew from the H graph once the density joined the estimate
    assert G.nnz > 0
