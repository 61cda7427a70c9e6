"""CPU FP64 oracle for the graph-based density-matrix and response path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or calls it,
and this package imports nothing from the product.  The two share only the
seeded input generators in ``synth``.

What it computes, plainly and slowly, in float64 (numpy / LAPACK):

* ``graph``     -- the thresholded data-dependency graph (Sec. "Estimating the
                   connectivity graph": |H| and |D_prev| above tau, optional
                   paths of length two), the core/halo partition (Fig. 1 and
                   Sec. "Choosing the graph partitioning"), principal-submatrix
                   gather and column collect (Eq. sub_f / Eq. dCollect), and the
                   matrix polynomial on a graph masked after every product
                   (Fig. 0, Eq. f_tau).
* ``fermi``     -- Fermi occupations, the Newton-Raphson chemical potential
                   (Eq. NewtonRaphson) with a bisection bracket, and the
                   divided-difference form of the canonical first-order
                   response (Eqs. D1_a, D1_b, ddlambda, dddmu, dmu_1).
* ``solve``     -- ``oracle_full`` (one diagonalisation of the whole H) and
                   ``oracle_graph`` (Eqs. DD0-SmallKS: per-subgraph
                   diagonalisation, one shared mu, core-column collect, graph
                   response with the global mu_1 of Eq. dmu_1).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants the paper states, brute force on tiny inputs and finite differences.
"""

from .fermi import (fermi, fermi_weight, fermi_divided_difference, solve_mu,
                    dense_density, dense_response)
from .graph import (graph_build, partition, gather, collect_columns,
                    polynomial_on_graph, column_mask)
from .solve import oracle_full, oracle_graph, GraphResult, FullResult

__all__ = [
    "fermi", "fermi_weight", "fermi_divided_difference", "solve_mu", "dense_density",
    "dense_response", "graph_build", "partition", "gather", "collect_columns",
    "polynomial_on_graph", "column_mask", "oracle_full", "oracle_graph", "GraphResult",
    "FullResult",
]
