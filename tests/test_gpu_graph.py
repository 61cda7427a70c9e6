"""Graph estimate and partition on the GPU: bit-exact against the oracle."""

import numpy as np
import pytest
import torch

from oracle import graph_build as o_graph, oracle_graph, partition as o_part
from oracle.graph import partition_capped as o_part_capped
from synth import CSR, make_workload
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


def _check_graph(G, adj):
    assert np.array_equal(G.ptr.cpu().numpy(), adj.indptr)
    assert np.array_equal(G.idx.cpu().numpy(), adj.indices)


def _check_partition(P, part):
    assert P.n_sub == part.n_sub
    assert np.array_equal(P.core_ptr.cpu().numpy(), part.core_ptr)
    assert np.array_equal(P.core_idx.cpu().numpy(), part.core_idx)
    assert np.array_equal(P.sub_ptr.cpu().numpy(), part.sub_ptr)
    assert np.array_equal(P.sub_idx.cpu().numpy(), part.sub_idx)
    assert np.array_equal(P.core_pos.cpu().numpy(), part.core_pos)
    sizes = np.diff(part.sub_ptr)
    assert P.max_sub == sizes.max()
    assert P.out_nnz == int(np.sum(sizes * np.diff(part.core_ptr)))


@pytest.mark.parametrize("name,paths2", [("water64", False), ("water64", True), ("water1k", False),
                                         ("water1k", True)])
def test_water_graph_and_partition_bit_exact(gb, name, paths2):
    wl, system, _ = make_workload(name, n_rhs=0)
    H = system.H
    G = gb.graph_build(to_device(H), wl.tau, paths2=paths2)
    adj = o_graph(H.n, H.indptr, H.indices, H.data, wl.tau, paths2=paths2)
    _check_graph(G, adj)
    P = gb.partition(G, torch.as_tensor(system.orb_group))
    _check_partition(P, o_part(adj, system.orb_group))
    # deterministic across runs
    G2 = gb.graph_build(to_device(H), wl.tau, paths2=paths2)
    assert torch.equal(G.idx, G2.idx)


def test_graph_with_previous_density(gb):
    # two-pass estimate: |D_prev| > tau joins the thresholded H graph
    wl, system, h1 = make_workload("water64", n_rhs=0)
    H = system.H
    adj0 = o_graph(H.n, H.indptr, H.indices, H.data, wl.tau)
    part0 = o_part(adj0, system.orb_group)
    ref = oracle_graph(H, [], wl.kT, system.n_occ, part0)
    col_ptr, row_idx, val = ref.D
    dprev = gb.CSC(H.n, torch.as_tensor(col_ptr).cuda(), torch.as_tensor(row_idx, dtype=torch.int32).cuda(),
                   torch.as_tensor(val).cuda())
    for tau in (1e-4, 1e-6):
        G = gb.graph_build(to_device(H), tau, d_prev=dprev)
        adj = o_graph(H.n, H.indptr, H.indices, H.data, tau, d_prev=(col_ptr, row_idx, val))
        _check_graph(G, adj)
        P = gb.partition(G, torch.as_tensor(system.orb_group))
        _check_partition(P, o_part(adj, system.orb_group))


def test_capped_partition_bit_exact(gb):
    # adaptive graph of the 1,000-water box (|D_prev| > 1e-6 joins the H graph):
    # a few one-molecule subgraphs exceed 128 orbitals and split into atoms
    wl, system, _ = make_workload("water1k", n_rhs=0)
    H = system.H
    adj0 = o_graph(H.n, H.indptr, H.indices, H.data, 1e-4)
    ref = oracle_graph(H, [], 0.2, system.n_occ, o_part(adj0, system.orb_group), workers=4)
    col_ptr, row_idx, val = ref.D
    dprev = gb.CSC(H.n, torch.as_tensor(col_ptr).cuda(), torch.as_tensor(row_idx, dtype=torch.int32).cuda(),
                   torch.as_tensor(val).cuda())
    G = gb.graph_build(to_device(H), 1e-6, d_prev=dprev)
    adj = o_graph(H.n, H.indptr, H.indices, H.data, 1e-6, d_prev=(col_ptr, row_idx, val))
    _check_graph(G, adj)
    groups = torch.as_tensor(system.orb_group)
    atoms = torch.as_tensor(system.orb_atom)
    assert gb.partition(G, groups).max_sub > 128
    P = gb.partition(G, groups, subgroups=atoms, max_sub=128)
    part = o_part_capped(adj, system.orb_group, system.orb_atom, 128)
    _check_partition(P, part)
    assert P.max_sub <= 128 and part.n_sub > int(system.orb_group.max()) + 1
    # random graph, tight cap: many groups split
    rng = np.random.default_rng(8)
    n = 257
    A = rng.normal(size=(n, n)) * (rng.random((n, n)) < 0.03)
    A = 0.5 * (A + A.T) + np.diag(rng.normal(size=n))
    Ac = CSR.from_dense(A)
    G = gb.graph_build(to_device(Ac), 0.0)
    adj = o_graph(n, Ac.indptr, Ac.indices, Ac.data, 0.0)
    grp = rng.integers(0, 40, size=n).astype(np.int32)
    sub = (grp * 3 + rng.integers(0, 3, size=n)).astype(np.int32)
    for cap in (12, 20, 30, 1000):
        P = gb.partition(G, torch.as_tensor(grp), 40, subgroups=torch.as_tensor(sub), n_subgroups=120, max_sub=cap)
        _check_partition(P, o_part_capped(adj, grp, sub, cap))


def test_random_graph_blocks_and_edge_cases(gb):
    rng = np.random.default_rng(5)
    n = 301
    A = rng.normal(size=(n, n)) * (rng.random((n, n)) < 0.02)
    A = 0.5 * (A + A.T) + np.diag(rng.normal(size=n))
    Ac = CSR.from_dense(A)
    for tau in (0.0, 0.05):
        G = gb.graph_build(to_device(Ac), tau)
        adj = o_graph(n, Ac.indptr, Ac.indices, Ac.data, tau)
        _check_graph(G, adj)
        # no groups: consecutive blocks of 7 (ragged last block)
        P = gb.partition(G, None, target_core_size=7)
        _check_partition(P, o_part(adj, None, target_core_size=7))
        # sparse group ids with empty groups
        groups = rng.integers(0, 500, size=n).astype(np.int32)
        P = gb.partition(G, torch.as_tensor(groups), 500)
        _check_partition(P, o_part(adj, groups))
    # a diagonal matrix: no edges, every subgraph is its core
    Dg = CSR.from_dense(np.diag(np.arange(1.0, 11.0)))
    G = gb.graph_build(to_device(Dg), 0.0)
    assert G.nnz == 0 and torch.all(G.ptr == 0)
    P = gb.partition(G, None, target_core_size=3)
    assert P.n_sub == 4 and P.max_sub == 3


def test_hub_row_and_uneven_cores_in_one_call(gb):
    # a hub vertex of degree ~900 beside rows of ~10 in one graph build, then
    # cores of 1 to 250 vertices (core plus neighbour lists from 9 to ~16,000
    # entries) in one partition, bit-exact against the oracle
    rng = np.random.default_rng(11)
    n = 2000
    A = (rng.random((n, n)) < 0.004) * rng.normal(size=(n, n))
    A[0, rng.choice(n, size=900, replace=False)] = 1.0
    A = 0.5 * (A + A.T)
    np.fill_diagonal(A, 1.0)
    Ac = CSR.from_dense(A)
    G = gb.graph_build(to_device(Ac), 0.0)
    adj = o_graph(n, Ac.indptr, Ac.indices, Ac.data, 0.0)
    _check_graph(G, adj)
    assert np.diff(adj.indptr).max() > 512
    sizes = np.concatenate([rng.integers(1, 6, size=200), [250, 180, 120]])
    groups = np.repeat(np.arange(len(sizes)), sizes)[:n]
    groups = np.concatenate([groups, np.full(n - len(groups), len(sizes))]).astype(np.int32)
    groups = groups[rng.permutation(n)]
    P = gb.partition(G, torch.as_tensor(groups), len(sizes) + 1)
    ref = o_part(adj, groups)
    _check_partition(P, ref)
    deg = np.diff(adj.indptr)
    entries = np.array([len(c) + deg[c].sum() for c in (ref.core_idx[ref.core_ptr[i]:ref.core_ptr[i + 1]]
                                                         for i in range(len(ref.core_ptr) - 1))])
    assert entries.min() < 20 and entries.max() > 10000


def test_argument_errors(gb):
    wl, system, _ = make_workload("water64", n_rhs=0)
    H = to_device(system.H)
    with pytest.raises(gb.GbError):
        gb.graph_build(H, -1.0)
    G = gb.graph_build(H, wl.tau)
    bad = torch.full((H.n,), 7, dtype=torch.int32)
    with pytest.raises(gb.GbError):
        gb.partition(G, bad, 5)       # group id out of range
