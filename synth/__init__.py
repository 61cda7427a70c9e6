"""Seeded synthetic inputs for the graph-based density / response path.

This package only *produces inputs*: atom positions, an orthogonal
tight-binding Hamiltonian H and perturbations H1 in CSR form, the
orbital -> molecule map that places the cores, and the electron count.
It holds none of the method's arithmetic (no Fermi function, no graph,
no partition, no response) and is the one module that both the CUDA path's
tests and the CPU oracle import.
"""

from .system import CSR, System
from .water import water_box, water_perturbation, thermal_trajectory, softened_coulomb_matrix
from .workloads import WORKLOADS, make_workload

__all__ = ["CSR", "System", "water_box", "water_perturbation", "thermal_trajectory",
           "WORKLOADS", "make_workload", "softened_coulomb_matrix"]
