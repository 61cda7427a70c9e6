"""Named synthetic workloads: sizes, temperatures and thresholds.

Each workload is a seeded water box (seed 20221204 + index) with a set of
perturbations H1 (seed 20221204 + index + 100 * (r + 1) for right-hand side r).
"""

from __future__ import annotations

from dataclasses import dataclass

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


WORKLOADS = {
    # 64 waters, 384 orbitals, one molecule per core, FP64
    "water64": Workload("water64", 0, 64, 0.1, 1e-5),
    # 1,000 waters, 6,000 orbitals, FP64
    "water1k": Workload("water1k", 1, 1000, 0.1, 1e-5),
    # 10,000 waters, 60,000 orbitals, mixed vs FP64, kT 0.05 / 0.2, tau 1e-4 / 1e-6
    "water10k": Workload("water10k", 2, 10000, 0.2, 1e-4, precision="mixed"),
    "water10k_kT0.05": Workload("water10k_kT0.05", 2, 10000, 0.05, 1e-6, precision="mixed"),
    # 20,000 waters, 120,000 orbitals, m = 6 right-hand sides
    "water20k_m6": Workload("water20k_m6", 4, 20000, 0.1, 1e-5, m=6, precision="mixed"),
}


def make_workload(name_or_wl, n_rhs: int | None = None) -> tuple[Workload, System, list[CSR]]:
    wl = WORKLOADS[name_or_wl] if isinstance(name_or_wl, str) else name_or_wl
    seed = BASE_SEED + wl.index
    system = water_box(wl.n_waters, seed)
    m = wl.m if n_rhs is None else n_rhs
    h1 = [water_perturbation(system, seed + 100 * (r + 1)) for r in range(m)]
    return wl, system, h1
