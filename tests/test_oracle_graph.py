"""Pins of the oracle's graph estimate, partition, gather and collect (CPU).

* graph_build against an O(N^2) enumeration of pairs and an explicit loop for
  paths of length two;
* partition against a brute-force neighbourhood computed from the dense
  adjacency;
* Eq. sub_f: a matrix polynomial on the graph, masked after every product
  (Fig. 0), equals the collected core columns of the same polynomial of the
  dense principal submatrices -- for single-vertex cores on the symmetric
  graph (the paper's Fig. 1 case) and for multi-vertex cores on the
  column-collect (directed) mask.
"""

import numpy as np
import pytest

from oracle.graph import (collect_columns, column_mask, csc_to_dense, dense_polynomial, gather,
                          graph_build, partition, partition_capped, polynomial_on_graph)
from synth import CSR, make_workload


def _random_sparse_sym(rng, n, density):
    a = rng.normal(size=(n, n)) * (rng.random((n, n)) < density)
    a = 0.5 * (a + a.T)
    a += np.diag(rng.normal(size=n))
    return a


def _brute_graph(A, tau, dprev=None, paths2=False):
    n = A.shape[0]
    E = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for j in range(n):
            if i != j and (abs(A[i, j]) > tau or (dprev is not None and abs(dprev[i, j]) > tau)):
                E[i, j] = E[j, i] = True
    if paths2:
        E2 = E.copy()
        for i in range(n):
            for k in np.nonzero(E[i])[0]:
                for j in np.nonzero(E[k])[0]:
                    if i != j:
                        E2[i, j] = True
        E = E2
    return E


@pytest.mark.parametrize("paths2", [False, True])
def test_graph_build_matches_pair_enumeration(paths2):
    rng = np.random.default_rng(20)
    A = _random_sparse_sym(rng, 60, 0.06)
    A[np.abs(A) < 0.3] *= 1e-3          # values near the threshold
    dprev = _random_sparse_sym(rng, 60, 0.03)
    np.fill_diagonal(dprev, 1.0)
    Ac, Dc = CSR.from_dense(A), CSR.from_dense(dprev)
    for tau in [0.0, 1e-3, 0.2]:
        adj = graph_build(60, Ac.indptr, Ac.indices, Ac.data, tau, paths2=paths2,
                          d_prev=(Dc.indptr, Dc.indices, Dc.data))
        E = _brute_graph(A, tau, dprev, paths2)
        assert np.array_equal(adj.to_dense(), E)
        assert all(np.all(np.diff(adj.neighbours(i)) > 0) for i in range(60))


def test_graph_symmetrises_one_sided_entries():
    # A column-collected D_prev is not symmetric, and an H given as one
    # triangle is not either: an entry above tau on one side alone makes the
    # edge both ways (the graph is undirected).
    rng = np.random.default_rng(23)
    n, tau = 40, 0.1
    A = np.triu(_random_sparse_sym(rng, n, 0.05))
    dprev = rng.normal(size=(n, n)) * (rng.random((n, n)) < 0.04)
    one_sided = (np.abs(dprev) > tau) & ~(np.abs(dprev.T) > tau)
    np.fill_diagonal(one_sided, False)
    assert one_sided.any()
    Ac, Dc = CSR.from_dense(A), CSR.from_dense(dprev)
    for paths2 in (False, True):
        adj = graph_build(n, Ac.indptr, Ac.indices, Ac.data, tau, paths2=paths2,
                          d_prev=(Dc.indptr, Dc.indices, Dc.data))
        E = _brute_graph(A, tau, dprev, paths2)
        assert np.array_equal(E, E.T)
        assert np.array_equal(adj.to_dense(), E)


def test_graph_threshold_is_strict():
    A = np.array([[0.0, 0.5, 0.0], [0.5, 0.0, 0.25], [0.0, 0.25, 0.0]])
    Ac = CSR.from_dense(A + np.eye(3))
    adj = graph_build(3, Ac.indptr, Ac.indices, Ac.data, 0.25)
    assert np.array_equal(adj.to_dense(), np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0]], bool))


def test_water_graph_matches_enumeration():
    wl, system, _ = make_workload("water64")
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, wl.tau)
    Hd = H.to_dense()
    E = (np.abs(Hd) > wl.tau)
    np.fill_diagonal(E, False)
    assert np.array_equal(adj.to_dense(), E | E.T)


def test_partition_matches_brute_force():
    rng = np.random.default_rng(21)
    A = _random_sparse_sym(rng, 50, 0.05)
    Ac = CSR.from_dense(A)
    adj = graph_build(50, Ac.indptr, Ac.indices, Ac.data, 0.0)
    E = adj.to_dense()
    groups = rng.integers(0, 13, size=50).astype(np.int32)
    part = partition(adj, groups)
    seen = np.zeros(50, dtype=int)
    present = sorted(set(groups.tolist()))
    assert part.n_sub == len(present)
    for i, g in enumerate(present):
        core = np.nonzero(groups == g)[0]
        assert np.array_equal(part.core(i), core)
        seen[core] += 1
        halo = np.nonzero(E[core].any(axis=0))[0]
        s = np.union1d(core, halo)
        assert np.array_equal(part.sub(i), s)
        assert np.array_equal(part.sub(i)[part.local_core(i)], core)
    assert np.all(seen == 1)
    # no groups: consecutive blocks
    p2 = partition(adj, None, target_core_size=7)
    assert p2.n_sub == 8 and np.array_equal(p2.core(7), np.arange(49, 50))


def test_partition_capped_rule_by_brute_force():
    # cores whose subgraph exceeds the cap are replaced by their subgroups,
    # and subgroup cores still over the cap by single vertices; order: kept
    # groups, then kept subgroup cores, then vertex cores, each ascending
    rng = np.random.default_rng(33)
    n = 60
    A = _random_sparse_sym(rng, n, 0.04)
    Ac = CSR.from_dense(A)
    adj = graph_build(n, Ac.indptr, Ac.indices, Ac.data, 0.0)
    E = adj.to_dense()
    groups = rng.integers(0, 9, size=n).astype(np.int32)
    # subgroups: pairs of consecutive vertices, never crossing a group
    subgroups = np.array([200 * groups[v] + v // 2 for v in range(n)], dtype=np.int32)

    def nbhd(core):
        return np.union1d(core, np.nonzero(E[core].any(axis=0))[0])

    gsizes = {g: len(nbhd(np.nonzero(groups == g)[0])) for g in sorted(set(groups.tolist()))}
    levels_seen = set()
    for cap in sorted(set(gsizes.values()))[:-1] + [3]:
        kept, subs, verts = [], [], []
        for g in sorted(gsizes):
            core = np.nonzero(groups == g)[0]
            if len(nbhd(core)) <= cap:
                kept.append(core)
                continue
            for sg in sorted(set(subgroups[core].tolist())):
                sc = np.nonzero(subgroups == sg)[0]
                if len(nbhd(sc)) <= cap:
                    subs.append(sc)
                else:
                    verts.extend(np.array([v]) for v in sc)
        verts.sort(key=lambda c: int(c[0]))
        expected = kept + subs + verts
        levels_seen.update(k for k, lst in enumerate((kept, subs, verts)) if lst)
        part = partition_capped(adj, groups, subgroups, cap)
        assert part.n_sub == len(expected)
        for i, core in enumerate(expected):
            assert np.array_equal(part.core(i), core)
            assert np.array_equal(part.sub(i), nbhd(core))
    assert levels_seen == {0, 1, 2}
    # a cap above every subgraph leaves the partition unchanged
    same = partition_capped(adj, groups, subgroups, max(gsizes.values()))
    ref = partition(adj, groups)
    assert np.array_equal(same.sub_idx, ref.sub_idx) and np.array_equal(same.core_idx, ref.core_idx)


def test_sub_f_single_vertex_cores():
    # Fig. 1: one core vertex per subgraph, halo = neighbours, symmetric graph
    rng = np.random.default_rng(22)
    X = _random_sparse_sym(rng, 30, 0.1)
    Xc = CSR.from_dense(X)
    adj = graph_build(30, Xc.indptr, Xc.indices, Xc.data, 0.0)
    part = partition(adj, np.arange(30, dtype=np.int32))
    coeffs = [0.3, -1.1, 0.7, 0.25, -0.05]
    mask = adj.to_dense() | np.eye(30, dtype=bool)
    ref = polynomial_on_graph(X, mask, coeffs)
    blocks = []
    for i in range(part.n_sub):
        p = dense_polynomial(gather(X, part.sub(i)), coeffs)
        blocks.append(p[:, part.local_core(i)])
    got = csc_to_dense(30, *collect_columns(blocks, part))
    np.testing.assert_allclose(got, ref, atol=1e-12)
    assert np.abs(ref).max() > 0.1


def test_sub_f_multi_vertex_cores_column_collect():
    # multi-vertex cores: the collected result is the polynomial on the
    # directed column mask M[r, j] = (r in S_part(j)), left multiplication
    wl, system, _ = make_workload("water64")
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, wl.tau)
    part = partition(adj, system.orb_group)
    X = H.to_dense() / 30.0
    coeffs = [1.0, 0.5, -0.3, 0.2, 0.1, -0.05]
    ref = polynomial_on_graph(X, column_mask(part), coeffs)
    blocks = [dense_polynomial(gather(X, part.sub(i)), coeffs)[:, part.local_core(i)]
              for i in range(part.n_sub)]
    got = csc_to_dense(H.n, *collect_columns(blocks, part))
    np.testing.assert_allclose(got, ref, atol=1e-13)
    # a mask that is one vertex short breaks the equality (the pin is sharp)
    m2 = column_mask(part)
    s0 = part.sub(0)
    m2[s0[-1], part.core(0)] = False
    assert np.abs(polynomial_on_graph(X, m2, coeffs) - got).max() > 1e-6
