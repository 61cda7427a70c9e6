"""Graph truncation of the method itself: the graph-based D and D1 against the
full diagonalisation of H (FP64), on the small water boxes.

TEST INFRASTRUCTURE ONLY (see the package docstring).  This measures a
property of the graph method (Sec. "Estimating the connectivity graph"; Eq.
sub_f), not of any implementation: how far the collected core columns of the
subgraph solutions lie from the exact D = f(H) and its response at the
thresholds the workloads use.  Every collected entry (j, k) is compared with
the exact (j, k); entries the graph drops are not counted.

    python -m oracle.truncation            # prints one line per case
"""

from __future__ import annotations

import numpy as np

from .graph import graph_build, partition
from .solve import oracle_full, oracle_graph


def collected_error(ref_csc, full: np.ndarray) -> float:
    """max |collected - exact| over the collected entries of a CSC result."""
    ptr, idx, val = ref_csc
    col = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    return float(np.abs(val - full[idx, col]).max())


def truncation(H, h1, kT: float, n_occ: float, groups, tau: float, *, paths2: bool = False, d_prev=None,
               workers: int = 0):
    """(max|dD|, max|dD1|, mu_graph - mu_full) for one graph."""
    adj = graph_build(H.n, H.indptr, H.indices, H.data, tau, paths2=paths2, d_prev=d_prev)
    part = partition(adj, groups)
    g = oracle_graph(H, h1, kT, n_occ, part, workers=workers)
    f = oracle_full(H.to_dense(), [x.to_dense() for x in h1], kT, n_occ)
    return (collected_error(g.D, f.D), max(collected_error(a, b) for a, b in zip(g.D1, f.D1)), g.mu - f.mu,
            part.sizes().min(), part.sizes().max(), g)


def main():  # pragma: no cover - a measurement script
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from synth import make_workload
    workers = os.cpu_count() or 1
    for name, kT in (("water64", 0.1), ("water1k", 0.1)):
        wl, system, h1 = make_workload(name, n_rhs=1)
        H = system.H
        eD, eD1, dmu, lo, hi, g = truncation(H, h1, kT, system.n_occ, system.orb_group, wl.tau, workers=workers)
        print(f"{name} kT {kT} H graph tau {wl.tau:g} ({lo}-{hi} orbitals): max|dD| {eD:.2e} max|dD1| {eD1:.2e} "
              f"dmu {dmu:.2e}", flush=True)
        eD, eD1, dmu, lo, hi, _ = truncation(H, h1, kT, system.n_occ, system.orb_group, wl.tau, d_prev=g.D,
                                             workers=workers)
        print(f"{name} kT {kT} two-pass graph tau {wl.tau:g} ({lo}-{hi} orbitals): max|dD| {eD:.2e} "
              f"max|dD1| {eD1:.2e} dmu {dmu:.2e}", flush=True)
        eD, eD1, dmu, lo, hi, _ = truncation(H, h1, kT, system.n_occ, system.orb_group, wl.tau, paths2=True,
                                             workers=workers)
        print(f"{name} kT {kT} paths-of-two graph tau {wl.tau:g} ({lo}-{hi} orbitals): max|dD| {eD:.2e} "
              f"max|dD1| {eD1:.2e} dmu {dmu:.2e}", flush=True)


if __name__ == "__main__":  # pragma: no cover
    main()
