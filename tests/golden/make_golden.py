"""Write the oracle's regression fixtures (tests/golden/*.json).

The paper prints no worked values for this path: its results are plots of
molecular-dynamics observables of SCC-DFTB systems.  These fixtures are the
oracle's own results on seeded synthetic inputs, written by this script, which
calls only ``oracle/`` and the input generators (``synth/``).  They are not
pins -- the pins are the closed forms, brute force and finite differences in
tests/test_oracle_*.py -- but a record of what the pinned oracle returns, so
that any later change to its arithmetic shows up as a failing comparison.

    python tests/golden/make_golden.py
"""

from __future__ import annotations

import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import graph_build, oracle_full, oracle_graph, partition  # noqa: E402
from oracle.graph import csc_to_dense  # noqa: E402
from oracle.solve import mulliken_charges  # noqa: E402
from synth import make_workload  # noqa: E402

FIXTURE = os.path.join(HERE, "water64_oracle.json")
N_SAMPLES = 64


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def compute() -> dict:
    """The water64 box (384 orbitals, kT 0.1 eV, tau 1e-5, one molecule per
    core, one H1): graph, partition, graph-method and full results."""
    wl, system, h1 = make_workload("water64", n_rhs=1)
    H = system.H
    adj = graph_build(H.n, H.indptr, H.indices, H.data, wl.tau)
    part = partition(adj, system.orb_group)
    g = oracle_graph(H, h1, wl.kT, system.n_occ, part)
    full = oracle_full(H.to_dense(), [h.to_dense() for h in h1], wl.kT, system.n_occ)
    ptr, idx, val = g.D
    val1 = g.D1[0][2]
    # a fixed spread of collected entries (every (nnz / N_SAMPLES)-th one)
    col = np.repeat(np.arange(H.n), np.diff(ptr))
    pick = np.linspace(0, len(val) - 1, N_SAMPLES).round().astype(np.int64)
    dg = csc_to_dense(H.n, *g.D).diagonal()
    q = mulliken_charges(dg, system.orb_atom, system.z_valence)
    return {
        "workload": "water64: 64 waters, 384 orbitals, kT 0.1 eV, tau 1e-5, H graph, one molecule per core, one H1",
        "graph": {"nnz": int(len(adj.indices)), "indptr_sha256": digest(adj.indptr.astype(np.int64)),
                  "indices_sha256": digest(adj.indices.astype(np.int32))},
        "partition": {"n_sub": int(part.n_sub), "sub_nnz": int(part.sub_ptr[-1]),
                      "sub_idx_sha256": digest(part.sub_idx.astype(np.int32)),
                      "core_pos_sha256": digest(part.core_pos.astype(np.int32))},
        "graph_method": {"mu": g.mu, "mu1": float(g.mu1[0]), "trace_core": g.trace_core,
                         "trace_core_dd": g.trace_core_dd, "trace_d1mu": g.trace_d1mu,
                         "samples": [[int(col[k]), int(idx[k]), float(val[k]), float(val1[k])] for k in pick],
                         "charges_first_8": [float(x) for x in q[:8]]},
        "full": {"mu": full.mu, "mu1": float(full.mu1[0]),
                 "samples": [[int(col[k]), int(idx[k]), float(full.D[idx[k], col[k]]),
                              float(full.D1[0][idx[k], col[k]])] for k in pick]},
    }


if __name__ == "__main__":
    with open(FIXTURE, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print("wrote", FIXTURE)
