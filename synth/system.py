"""Plain containers for synthetic systems (no method arithmetic)."""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """Square sparse matrix in compressed-sparse-row form.

    ``indptr`` is int64 (n+1), ``indices`` int32 (nnz, ascending inside each
    row), ``data`` float64 (nnz).
    """

    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        out[rows, self.indices] = self.data
        return out

    @staticmethod
    def from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> "CSR":
        """Build a CSR matrix from triplets (duplicates are summed)."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        vals = np.asarray(vals, dtype=np.float64)
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        key, vals = key[order], vals[order]
        uniq, start = np.unique(key, return_index=True)
        summed = np.add.reduceat(vals, start) if len(vals) else vals
        r = uniq // n
        c = uniq % n
        indptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(indptr, r + 1, 1)
        indptr = np.cumsum(indptr)
        return CSR(n, indptr, c.astype(np.int32), summed.astype(np.float64))

    @staticmethod
    def from_dense(a: np.ndarray) -> "CSR":
        r, c = np.nonzero(a)
        return CSR.from_coo(a.shape[0], r, c, a[r, c])


# species codes
SPECIES = {"H": 0, "C": 1, "N": 2, "O": 3}
SPECIES_NAME = {v: k for k, v in SPECIES.items()}
# orbitals per species (s only for H; s, px, py, pz otherwise)
N_ORB = {0: 1, 1: 4, 2: 4, 3: 4}
# neutral valence electron counts
VALENCE = {0: 1, 1: 4, 2: 5, 3: 6}


@dataclass
class System:
    """A periodic molecular system and its tight-binding Hamiltonian."""

    box: float                      # cubic box edge, Angstrom
    positions: np.ndarray           # (n_atoms, 3), Angstrom, wrapped into [0, box)
    species: np.ndarray             # (n_atoms,) int8 species codes (SPECIES)
    molecule: np.ndarray            # (n_atoms,) int32 molecule id
    orb_atom: np.ndarray            # (n_orb,) int32 atom of each orbital
    H: CSR                          # orthogonal TB Hamiltonian, eV
    n_electrons: int                # neutral valence electron count
    atom_core: np.ndarray | None = None  # (n_atoms,) core id of each atom, when not one per molecule
    meta: dict = field(default_factory=dict)

    @property
    def n_orb(self) -> int:
        return self.H.n

    @property
    def n_atoms(self) -> int:
        return len(self.species)

    @property
    def n_occ(self) -> float:
        """Spin-restricted occupied-state count, Ne / 2."""
        return self.n_electrons / 2.0

    @property
    def orb_group(self) -> np.ndarray:
        """Core id of every orbital: its atom's core when set, else its molecule."""
        owner = self.atom_core if self.atom_core is not None else self.molecule
        return owner[self.orb_atom].astype(np.int32)

    @property
    def z_valence(self) -> np.ndarray:
        return np.array([VALENCE[int(s)] for s in self.species], dtype=np.float64)
