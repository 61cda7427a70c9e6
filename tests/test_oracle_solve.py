"""Pins of oracle_full and oracle_graph (CPU only).

What the paper fixes and what mathematics fixes: Tr D = N_occ; D symmetric;
D idempotent as kT -> 0 across a gap; Tr D1 = 0 at fixed N_occ; D1 equals the
central finite difference of D(H + eps H1) with mu re-solved; one subgraph
holding everything reproduces the full calculation; disconnected blocks are
solved exactly by the graph method.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import graph_build, oracle_full, oracle_graph, partition
from oracle.graph import Partition, csc_to_dense
from oracle.solve import mulliken_charges
from synth import CSR, make_workload


def _random_sym(rng, n, scale=1.0):
    a = rng.normal(size=(n, n)) * scale
    return 0.5 * (a + a.T)


@pytest.fixture(scope="module")
def water64():
    wl, system, h1 = make_workload("water64")
    return wl, system, h1


def test_full_trace_symmetry_and_occupation():
    rng = np.random.default_rng(10)
    H = _random_sym(rng, 40, 2.0)
    h1 = _random_sym(rng, 40, 0.3)
    res = oracle_full(H, [h1], 0.2, 17.0)
    assert abs(np.trace(res.D) - 17.0) < 1e-10
    np.testing.assert_allclose(res.D, res.D.T, atol=1e-14)
    assert abs(np.trace(res.D1[0])) < 1e-12
    w = np.linalg.eigvalsh(res.D)
    assert w.min() > -1e-14 and w.max() < 1 + 1e-14


def test_full_idempotent_at_low_temperature():
    # block-diagonal gapped H: eigenvalues well separated around mu
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.normal(size=(30, 30)))
    eps = np.concatenate([rng.uniform(-6, -3, 12), rng.uniform(3, 6, 18)])
    H = (Q * eps) @ Q.T
    res = oracle_full(H, [], 0.05, 12.0)
    gap = 6.0
    err = np.abs(res.D @ res.D - res.D).max()
    assert err < 12 * np.exp(-gap / (2 * 0.05)) + 1e-13
    assert -3.0 < res.mu < 3.0


def test_full_response_equals_canonical_finite_difference():
    rng = np.random.default_rng(12)
    H = _random_sym(rng, 24, 1.5)
    h1 = _random_sym(rng, 24, 0.5)
    kT, nocc, e = 0.3, 9.0, 1e-5
    res = oracle_full(H, [h1], kT, nocc)
    plus = oracle_full(H + e * h1, [], kT, nocc)
    minus = oracle_full(H - e * h1, [], kT, nocc)
    fd = (plus.D - minus.D) / (2 * e)
    np.testing.assert_allclose(res.D1[0], fd, atol=5e-8)
    assert abs(res.mu1[0] - (plus.mu - minus.mu) / (2 * e)) < 5e-8


def test_full_matches_expm_route():
    rng = np.random.default_rng(13)
    H = _random_sym(rng, 12, 1.0)
    res = oracle_full(H, [], 0.5, 5.0)
    ref = np.linalg.inv(sla.expm((H - res.mu * np.eye(12)) / 0.5) + np.eye(12))
    np.testing.assert_allclose(res.D, ref, atol=1e-12)


def _one_subgraph(n):
    idx = np.arange(n, dtype=np.int32)
    return Partition(n, np.array([0, n]), idx, np.array([0, n]), idx, idx)


def test_graph_with_one_subgraph_is_full(water64):
    wl, system, h1 = water64
    H = system.H
    full = oracle_full(H.to_dense(), [h.to_dense() for h in h1], wl.kT, system.n_occ)
    g = oracle_graph(H, h1, wl.kT, system.n_occ, _one_subgraph(H.n), mu0=full.mu)
    np.testing.assert_allclose(csc_to_dense(H.n, *g.D), full.D, atol=1e-12)
    np.testing.assert_allclose(csc_to_dense(H.n, *g.D1[0]), full.D1[0], atol=1e-11)
    assert abs(g.mu1[0] - full.mu1[0]) < 1e-8


def test_graph_exact_on_disconnected_blocks():
    # block-diagonal H with each block a core: the graph method is exact
    rng = np.random.default_rng(14)
    sizes = [5, 7, 4, 6]
    n = sum(sizes)
    H = np.zeros((n, n))
    H1 = np.zeros((n, n))
    groups = np.zeros(n, dtype=np.int32)
    o = 0
    for g, s in enumerate(sizes):
        H[o:o + s, o:o + s] = _random_sym(rng, s, 1.0) + rng.normal() * np.eye(s)
        H1[o:o + s, o:o + s] = _random_sym(rng, s, 0.2)
        groups[o:o + s] = g
        o += s
    Hc, H1c = CSR.from_dense(H), CSR.from_dense(H1)
    adj = graph_build(n, Hc.indptr, Hc.indices, Hc.data, 1e-12)
    part = partition(adj, groups)
    assert part.n_sub == 4 and np.all(part.sizes() == sizes)
    full = oracle_full(H, [H1], 0.2, 10.0)
    g = oracle_graph(Hc, [H1c], 0.2, 10.0, part)
    np.testing.assert_allclose(csc_to_dense(n, *g.D), full.D, atol=1e-12)
    np.testing.assert_allclose(csc_to_dense(n, *g.D1[0]), full.D1[0], atol=1e-10)
    assert abs(g.mu - full.mu) < 1e-10
    assert abs(g.mu1[0] - full.mu1[0]) < 1e-9 * max(1.0, abs(full.mu1[0]))   # Eq. dmu_1 from core traces


def test_graph_invariants_and_canonical_finite_difference(water64):
    wl, system, h1 = water64
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, wl.tau)
    part = partition(adj, system.orb_group)
    g = oracle_graph(H, h1, wl.kT, system.n_occ, part)
    D = csc_to_dense(H.n, *g.D)
    D1 = csc_to_dense(H.n, *g.D1[0])
    # Tr D_G = N_occ and Tr D1_G = 0 (Eq. dmu_1 keeps the electron count)
    assert abs(np.trace(D) - system.n_occ) < 1e-9
    assert abs(np.trace(D1)) < 1e-12
    assert abs(g.trace_core - system.n_occ) < 1e-9
    # dN/dmu two ways: beta sum_k f(1 - f) w_k from the spectra, and the core
    # traces of the d1_mu = beta d (I - d) matrices (Eq. dddmu)
    assert abs(g.trace_d1mu - g.trace_core_dd / wl.kT) < 1e-10 * g.trace_d1mu
    # canonical finite difference on the same graph, mu re-solved each side
    e = 1e-4
    Hp = CSR(H.n, H.indptr, H.indices, H.data.copy())
    Hm = CSR(H.n, H.indptr, H.indices, H.data.copy())
    dense_h1 = h1[0].to_dense()
    # H1 is diagonal; add it on the diagonal entries of H's CSR
    rows = np.repeat(np.arange(H.n), np.diff(H.indptr))
    diag = rows == H.indices
    Hp.data[diag] += e * np.diag(dense_h1)[rows[diag]]
    Hm.data[diag] -= e * np.diag(dense_h1)[rows[diag]]
    gp = oracle_graph(Hp, [], wl.kT, system.n_occ, part)
    gm = oracle_graph(Hm, [], wl.kT, system.n_occ, part)
    fd = (csc_to_dense(H.n, *gp.D) - csc_to_dense(H.n, *gm.D)) / (2 * e)
    np.testing.assert_allclose(D1, fd, atol=1e-7)
    # neutral system: Mulliken charges sum to zero
    q = mulliken_charges(np.diag(D), system.orb_atom, system.z_valence)
    assert abs(q.sum()) < 1e-8


def test_mulliken_two_atom_closed_form():
    # two atoms with one orbital each and two electrons (one occupied
    # orbital): at low temperature the bonding orbital (cos t, sin t) is
    # filled, D_11 = cos^2 t, and q_1 = 1 - 2 D_11 = -(e2 - e1) / sqrt((e2 -
    # e1)^2 + 4 h^2): the atom with the lower on-site energy is negative.  A
    # sign error (population minus Z) or a dropped spin factor of 2 fails.
    from oracle.solve import mulliken_charges
    e1, e2, h = -2.0, 1.0, -0.8
    H = np.array([[e1, h], [h, e2]])
    full = oracle_full(H, [], 0.001, 1.0)
    q = mulliken_charges(np.diag(full.D), np.array([0, 1]), np.array([1.0, 1.0]))
    expect = -(e2 - e1) / np.sqrt((e2 - e1) ** 2 + 4 * h * h)
    assert abs(q[0] - expect) < 1e-12 and abs(q[1] + expect) < 1e-12
    assert q[0] < 0


def test_mulliken_response_is_the_charge_derivative():
    # q1 = -2 sum_o D1_oo is dq/dlambda of H + lambda H1 at fixed electron
    # count: central difference of the charges themselves
    from oracle.solve import mulliken_charges
    rng = np.random.default_rng(5)
    n = 12
    A = rng.normal(size=(n, n))
    H = 0.5 * (A + A.T) + np.diag(rng.normal(0, 2, n))
    H1 = np.diag(rng.normal(0, 0.3, n))
    atom = np.repeat(np.arange(4), 3)
    z = np.array([2.0, 1.0, 2.0, 1.0])
    kT, nocc = 0.3, 3.0
    full = oracle_full(H, [H1], kT, nocc)
    q1 = mulliken_charges(np.diag(full.D1[0]), atom, np.zeros(4))
    eps = 1e-4
    qp = mulliken_charges(np.diag(oracle_full(H + eps * H1, [], kT, nocc).D), atom, z)
    qm = mulliken_charges(np.diag(oracle_full(H - eps * H1, [], kT, nocc).D), atom, z)
    assert np.abs((qp - qm) / (2 * eps) - q1).max() < 1e-7


def test_graph_oracle_is_the_same_serial_and_in_a_process_pool(water64):
    # the tests and the CPU baseline run the oracle over a process pool: every
    # subgraph's block lands in its own place and the sums keep their order.
    # The pool's workers run single-threaded BLAS, so a product may round
    # differently in its last bit; nothing more may change.
    wl, system, h1 = water64
    H = system.H
    part = partition(graph_build(H.n, H.indptr, H.indices, H.data, wl.tau), system.orb_group)
    a = oracle_graph(H, h1, wl.kT, system.n_occ, part, workers=0)
    b = oracle_graph(H, h1, wl.kT, system.n_occ, part, workers=2)
    assert abs(a.mu - b.mu) < 1e-13 and np.abs(a.mu1 - b.mu1).max() < 1e-13
    for x, y in zip([a.D] + a.D1, [b.D] + b.D1):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert np.abs(x[2] - y[2]).max() < 1e-15
