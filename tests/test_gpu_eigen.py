"""The eigenbasis path (GB_PREC_EIGEN) against the oracle: each subgraph's
principal submatrix diagonalised in FP64 on the GPU (Eq. SmallKS), mu from the
eigenvalue sums, d, d1 in the eigenbasis (Eqs. DD, ddlambda, dddmu).  Same
1e-9 bound as the FP64 recursion."""

import numpy as np
import pytest
import torch

from oracle import graph_build as o_graph, oracle_full, oracle_graph, partition as o_part
from synth import make_workload
from tests.helpers import dense_result, max_abs_block_error, to_device
from tests.test_gpu_density import _random_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2212_01997_gb300 as gb
    from paper_2212_01997_gb300 import build
    build.build()
    return gb


@pytest.mark.parametrize("name,kT,paths2", [("water64", 0.1, False), ("water64", 0.1, True),
                                            ("water1k", 0.05, False), ("chains_small", 0.1, False)])
def test_eigen_parity(gb, name, kT, paths2):
    wl, system, h1 = make_workload(name, n_rhs=2)
    H = system.H
    adj = o_graph(H.n, H.indptr, H.indices, H.data, wl.tau, paths2=paths2)
    part = o_part(adj, system.orb_group)
    ref = oracle_graph(H, h1, kT, system.n_occ, part, workers=4)
    Hd = to_device(H)
    P = gb.partition(gb.graph_build(Hd, wl.tau, paths2=paths2), torch.as_tensor(system.orb_group))
    # cold start: mu from the spectral bracket, every iteration an eigenvalue sum
    R = gb.density_and_response(Hd, [to_device(h) for h in h1], kT, system.n_electrons, P, precision="eigen")
    eD, eD1 = max_abs_block_error(R, ref, part)
    print(f"eigen {name}{' paths2' if paths2 else ''} kT={kT}: sizes {part.sizes().min()}..{part.sizes().max()} "
          f"max|dD|={eD:.2e} max|dD1|={eD1:.2e} dmu={R.mu - ref.mu:.2e} passes={R.report['passes']} "
          f"ms={R.report['pass_kernel_ms']:.1f}")
    assert eD <= 1e-9 and eD1 <= 1e-9
    assert abs(R.report["occ_residual"]) <= 1e-10 * system.n_occ
    for r in range(2):
        assert abs(R.mu1[r] - ref.mu1[r]) <= 1e-8 * max(1.0, abs(ref.mu1[r]))


def test_eigen_single_subgraph_equals_full(gb):
    Hc, H1c = _random_system(300, 12, density=0.05)
    n = Hc.n
    Hd = to_device(Hc)
    P = gb.partition(gb.graph_build(Hd, 0.0), torch.zeros(n, dtype=torch.int32))
    full = oracle_full(Hc.to_dense(), [H1c.to_dense()], 0.25, 120.0)
    R = gb.density_and_response(Hd, [to_device(H1c)], 0.25, 240.0, P, precision="eigen")
    eD = np.abs(dense_result(R.D) - full.D).max()
    eD1 = np.abs(dense_result(R.D, R.D1[0].val) - full.D1[0]).max()
    print(f"eigen single 300: max|dD|={eD:.2e} max|dD1|={eD1:.2e} dmu={R.mu - full.mu:.2e}")
    assert eD <= 1e-9 and eD1 <= 1e-9 and abs(R.mu - full.mu) < 1e-9


def test_eigen_degenerate_and_tiny(gb):
    # exact degeneracies (a block-diagonal H with repeated blocks) and 1-, 2-,
    # 3-orbital subgraphs: the bisection, the twists and the divided differences
    blocks = [np.array([[-1.0]]), np.array([[-2.0, 0.5], [0.5, -2.0]]),
              np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 0.0]])]
    A = np.zeros((18, 18))
    groups = []
    o = 0
    for rep in range(3):
        for g, b in enumerate(blocks):
            k = b.shape[0]
            A[o:o + k, o:o + k] = b
            groups += [3 * rep + g] * k
            o += k
    from synth import CSR
    Hc = CSR.from_dense(A)
    H1c = CSR.from_dense(np.diag(np.linspace(-0.2, 0.3, 18)))
    groups = np.array(groups, dtype=np.int32)
    adj = o_graph(18, Hc.indptr, Hc.indices, Hc.data, 0.0)
    part = o_part(adj, groups)
    ref = oracle_graph(Hc, [H1c], 0.2, 7.0, part)
    Hd = to_device(Hc)
    P = gb.partition(gb.graph_build(Hd, 0.0), torch.as_tensor(groups))
    R = gb.density_and_response(Hd, [to_device(H1c)], 0.2, 14.0, P, precision="eigen")
    eD, eD1 = max_abs_block_error(R, ref, part)
    assert eD <= 1e-9 and eD1 <= 1e-9


def test_eigen_degenerate_inside_one_subgraph(gb):
    # one subgraph holding repeated blocks and isolated orbitals of equal
    # energy, coupled at rounding level (as decoupled p orbitals appear in a
    # water subgraph): runs of equal eigenvalues inside one tridiagonal matrix,
    # split where the coupling is negligible, each member on its own twist
    rng = np.random.default_rng(7)
    chain = np.array([[-3.0, 1.0, 0.0], [1.0, -2.5, 0.7], [0.0, 0.7, -1.0]])
    pair = np.array([[-9.0, 0.4], [0.4, -8.5]])
    blocks = [chain, pair, chain, np.array([[-9.3]]), pair, np.array([[-9.3]]), chain,
              np.array([[-9.3]]), np.array([[-9.3]])]
    n = sum(b.shape[0] for b in blocks)
    A = np.zeros((n, n))
    o = 0
    for b in blocks:
        k = b.shape[0]
        A[o:o + k, o:o + k] = b
        o += k
    # rounding-level couplings between the blocks
    for _ in range(12):
        i, j = rng.integers(0, n, 2)
        if i != j:
            A[i, j] = A[j, i] = 1e-16 * rng.normal()
    from synth import CSR
    Hc = CSR.from_dense(A)
    H1c = CSR.from_dense(np.diag(np.linspace(-0.3, 0.2, n)))
    # 4 occupied: mu at the four-fold -9.3 level, which is half filled
    full = oracle_full(A, [np.diag(np.linspace(-0.3, 0.2, n))], 0.2, 4.0)
    Hd = to_device(Hc)
    P = gb.partition(gb.graph_build(Hd, 0.0), torch.zeros(n, dtype=torch.int32))
    R = gb.density_and_response(Hd, [to_device(H1c)], 0.2, 8.0, P, precision="eigen")
    eD = np.abs(dense_result(R.D) - full.D).max()
    eD1 = np.abs(dense_result(R.D, R.D1[0].val) - full.D1[0]).max()
    print(f"eigen degenerate runs in one subgraph (n={n}): max|dD|={eD:.2e} max|dD1|={eD1:.2e}")
    assert eD <= 1e-9 and eD1 <= 1e-9


def test_eigen_size_limit(gb):
    Hc, _ = _random_system(1100, 3, density=0.003)
    Hd = to_device(Hc)
    P = gb.partition(gb.graph_build(Hd, 0.0), torch.zeros(1100, dtype=torch.int32))
    R = gb.density_and_response(Hd, [], 0.2, 1000.0, P, precision="eigen", raise_on_error=False)
    assert R.status == 8  # GB_ERR_UNSUPPORTED
