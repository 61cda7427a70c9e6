"""Named synthetic workloads: sizes, temperatures and thresholds.

Each workload is a seeded water box, or a seeded solvated chain system
(seed 20221204 + index), with a set of perturbations H1 (seed
20221204 + index + 100 * (r + 1) for right-hand side r).
"""

from __future__ import annotations

from dataclasses import dataclass

from .chains import chain_system
from .system import CSR, System
from .water import water_box, water_perturbation

BASE_SEED = 20221204


@dataclass(frozen=True)
class Workload:
    name: str
    index: int
    n_waters: int
    kT: float
    tau: float
    m: int = 1
    precision: str = "fp64"
    paths2: bool = False
    # heterogeneous systems (kind "chains"): n_waters sizes the box; chains of
    # chain_len heavy atoms, at most max_atoms atoms, cores of core_atoms atoms
    kind: str = "water"
    n_chains: int = 0
    chain_len: int = 0
    max_atoms: int = 0
    core_atoms: int = 30


WORKLOADS = {
    # 64 waters, 384 orbitals, one molecule per core, FP64
    "water64": Workload("water64", 0, 64, 0.1, 1e-5),
    # 1,000 waters, 6,000 orbitals, FP64
    "water1k": Workload("water1k", 1, 1000, 0.1, 1e-5),
    # 10,000 waters, 60,000 orbitals, mixed vs FP64, kT 0.05 / 0.2, tau 1e-4 / 1e-6
    "water10k": Workload("water10k", 2, 10000, 0.2, 1e-4, precision="mixed"),
    "water10k_kT0.05": Workload("water10k_kT0.05", 2, 10000, 0.05, 1e-6, precision="mixed"),
    "water10k_kT0.05_tau1e-4": Workload("water10k_kT0.05_tau1e-4", 2, 10000, 0.05, 1e-4, precision="mixed"),
    "water10k_tau1e-6": Workload("water10k_tau1e-6", 2, 10000, 0.2, 1e-6, precision="mixed"),
    # 20,000 waters, 120,000 orbitals, m = 6 right-hand sides
    "water20k_m6": Workload("water20k_m6", 4, 20000, 0.1, 1e-5, m=6, precision="mixed"),
    # 30,000 atoms: 8 chains of 500 C/N/O heavy atoms with H caps, solvated
    # (61,773 orbitals); cores of ~30 atoms by coordinate bisection
    "chains30k": Workload("chains30k", 3, 12000, 0.1, 1e-5, precision="mixed", kind="chains", n_chains=8,
                          chain_len=500, max_atoms=30000),
    # one 60-atom chain in a small water box (3,401 orbitals), for the tests
    "chains_small": Workload("chains_small", 5, 600, 0.1, 1e-5, kind="chains", n_chains=1, chain_len=60,
                             max_atoms=1800),
}


def make_workload(name_or_wl, n_rhs: int | None = None) -> tuple[Workload, System, list[CSR]]:
    wl = WORKLOADS[name_or_wl] if isinstance(name_or_wl, str) else name_or_wl
    seed = BASE_SEED + wl.index
    if wl.kind == "chains":
        system = chain_system(wl.n_waters, wl.n_chains, wl.chain_len, wl.max_atoms, wl.core_atoms, seed)
    else:
        system = water_box(wl.n_waters, seed)
    m = wl.m if n_rhs is None else n_rhs
    h1 = [water_perturbation(system, seed + 100 * (r + 1)) for r in range(m)]
    return wl, system, h1
