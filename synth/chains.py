"""Seeded heterogeneous system: self-avoiding C/N/O chains with hydrogen caps,
solvated in water, with the water boxes' tight-binding model.

Recipe (inputs only, stated so a reader can rebuild them):

* Box: the cubic box of ``n_box_waters`` waters at 1.0 g/cm^3 (edge
  (n * 29.915 A^3)^(1/3)), periodic.
* Chains: ``n_chains`` self-avoiding walks of ``chain_len`` heavy atoms, species
  C, N, O drawn with probabilities 0.7, 0.15, 0.15.  Bonds 1.5 A.  Each new bond
  makes a bond angle of 109.5 +- 10 degrees (uniform) with the previous one,
  with a uniform random dihedral.  A position closer than 2.5 A (minimum image)
  to any placed heavy atom other than its two predecessors is rejected; after
  50 rejections in a row the walk backs up 3 atoms.  Start points are uniform
  in the box, at least 2.5 A from every placed heavy atom.
* Hydrogens fill each heavy atom's valence (C 4, N 3, O 2) minus its chain
  bonds, at 1.09 / 1.01 / 0.96 A, along the remaining directions of a
  tetrahedron around the chain bonds (random twist for chain ends).
* Water: the water box generator's lattice waters for the same box; every
  water with an atom closer than 2.5 A to a solute atom is dropped, then waters
  are kept in a seeded order until the system holds at most ``max_atoms``.
* Molecules: each chain with its hydrogens is one molecule, each water one.
* Cores (``atom_core``): recursive coordinate bisection of the atoms -- split
  the longest axis of the cell's bounding box at the median (ties by atom
  index) until a cell holds at most ``core_atoms`` atoms; cores are numbered in
  depth-first order (lower half first).
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .system import SPECIES, VALENCE, System
from .water import VOLUME_PER_WATER, tb_hamiltonian, water_positions

BOND = 1.5
MIN_DIST = 2.5
ANGLE = np.deg2rad(109.5)
ANGLE_SPREAD = np.deg2rad(10.0)
MAX_REJECT = 50
BACKUP = 3
H_BOND = {SPECIES["C"]: 1.09, SPECIES["N"]: 1.01, SPECIES["O"]: 0.96}
HEAVY = (SPECIES["C"], SPECIES["N"], SPECIES["O"])
HEAVY_P = (0.7, 0.15, 0.15)
BONDS = {SPECIES["C"]: 4, SPECIES["N"]: 3, SPECIES["O"]: 2}  # covalent valence


def _wrap(d, box):
    return d - box * np.round(d / box)


def _perp_basis(u):
    a = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(u, e1)


class _Cells:
    """Periodic cell list of heavy atoms (cell edge >= MIN_DIST)."""

    def __init__(self, box):
        self.box = box
        self.nc = max(1, int(box // MIN_DIST))
        self.edge = box / self.nc
        self.cells: dict = {}
        self.pos: list = []

    def _key(self, p):
        return tuple((np.floor(np.mod(p, self.box) / self.edge).astype(int)) % self.nc)

    def add(self, p):
        self.pos.append(p)
        self.cells.setdefault(self._key(p), []).append(len(self.pos) - 1)

    def remove_last(self):
        p = self.pos.pop()
        self.cells[self._key(p)].remove(len(self.pos))

    def clear(self, p, skip=()):
        k = self._key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in self.cells.get(((k[0] + dx) % self.nc, (k[1] + dy) % self.nc, (k[2] + dz) % self.nc), ()):
                        if j in skip:
                            continue
                        if np.linalg.norm(_wrap(self.pos[j] - p, self.box)) < MIN_DIST:
                            return False
        return True


def _walk(rng, cells, box, length):
    """One self-avoiding chain; returns heavy-atom positions (unwrapped) and cell ids."""
    while True:
        p0 = rng.random(3) * box
        if cells.clear(p0):
            break
    chain = [p0]
    ids = [len(cells.pos)]
    cells.add(p0)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    dirs = [u]
    rejects = 0
    while len(chain) < length:
        prev = dirs[-1]
        theta = np.pi - (ANGLE + rng.uniform(-ANGLE_SPREAD, ANGLE_SPREAD))  # turn from the previous bond
        phi = rng.uniform(0.0, 2.0 * np.pi)
        e1, e2 = _perp_basis(prev)
        d = np.cos(theta) * prev + np.sin(theta) * (np.cos(phi) * e1 + np.sin(phi) * e2)
        p = chain[-1] + BOND * d
        skip = set(ids[-2:])
        if cells.clear(p, skip):
            chain.append(p)
            ids.append(len(cells.pos))
            cells.add(p)
            dirs.append(d)
            rejects = 0
            continue
        rejects += 1
        if rejects >= MAX_REJECT and len(chain) > BACKUP:
            for _ in range(BACKUP):
                chain.pop()
                ids.pop()
                dirs.pop()
                cells.remove_last()
            rejects = 0
    return np.array(chain)


def _hydrogen_dirs(rng, bonds):
    """Unit vectors completing a tetrahedron around the given bond directions."""
    if len(bonds) == 2:
        b1, b2 = bonds
        bis = -(b1 + b2)
        bis /= np.linalg.norm(bis)
        nrm = np.cross(b1, b2)
        nrm /= np.linalg.norm(nrm)
        half = 0.5 * ANGLE
        return [np.cos(half) * bis + np.sin(half) * nrm, np.cos(half) * bis - np.sin(half) * nrm]
    b1 = bonds[0]
    e1, e2 = _perp_basis(b1)
    tw = rng.uniform(0.0, 2.0 * np.pi)
    out = []
    for k in range(3):
        a = tw + 2.0 * np.pi * k / 3.0
        out.append(-np.cos(np.pi - ANGLE) * b1 + np.sin(np.pi - ANGLE) * (np.cos(a) * e1 + np.sin(a) * e2))
    return out


def rcb_cores(pos: np.ndarray, core_atoms: int) -> np.ndarray:
    """Recursive coordinate bisection: core id of every atom (depth-first order)."""
    core = np.empty(len(pos), dtype=np.int32)
    stack = [np.arange(len(pos))]
    nxt = 0
    while stack:
        idx = stack.pop()
        if len(idx) <= core_atoms:
            core[idx] = nxt
            nxt += 1
            continue
        ext = pos[idx].max(axis=0) - pos[idx].min(axis=0)
        ax = int(np.argmax(ext))
        order = idx[np.lexsort((idx, pos[idx, ax]))]
        h = len(order) // 2
        stack.append(order[h:])   # popped second
        stack.append(order[:h])   # lower half first
    return core


def chain_system(n_box_waters: int, n_chains: int, chain_len: int, max_atoms: int, core_atoms: int,
                 seed: int) -> System:
    rng = np.random.default_rng(seed)
    box = float((n_box_waters * VOLUME_PER_WATER) ** (1.0 / 3.0))
    cells = _Cells(box)
    heavy_pos, heavy_sp, heavy_mol, bonds_of = [], [], [], []
    for c in range(n_chains):
        chain = _walk(rng, cells, box, chain_len)
        sp = rng.choice(HEAVY, size=chain_len, p=HEAVY_P)
        for k in range(chain_len):
            b = []
            if k > 0:
                d = chain[k - 1] - chain[k]
                b.append(d / np.linalg.norm(d))
            if k + 1 < chain_len:
                d = chain[k + 1] - chain[k]
                b.append(d / np.linalg.norm(d))
            bonds_of.append(b)
        heavy_pos.append(chain)
        heavy_sp.append(sp)
        heavy_mol.append(np.full(chain_len, c, dtype=np.int32))
    heavy_pos = np.concatenate(heavy_pos)
    heavy_sp = np.concatenate(heavy_sp)
    heavy_mol = np.concatenate(heavy_mol)
    # hydrogen caps
    h_pos, h_mol = [], []
    for a in range(len(heavy_pos)):
        s = int(heavy_sp[a])
        n_h = BONDS[s] - len(bonds_of[a])
        if n_h <= 0 or not bonds_of[a]:
            continue
        dirs = _hydrogen_dirs(rng, bonds_of[a])
        for d in dirs[:n_h]:
            h_pos.append(heavy_pos[a] + H_BOND[s] * d)
            h_mol.append(heavy_mol[a])
    sol_pos = np.mod(np.concatenate([heavy_pos, np.array(h_pos).reshape(-1, 3)]), box)
    sol_sp = np.concatenate([heavy_sp, np.full(len(h_pos), SPECIES["H"], dtype=heavy_sp.dtype)]).astype(np.int8)
    sol_mol = np.concatenate([heavy_mol, np.array(h_mol, dtype=np.int32)])
    # solvent: lattice waters of the same box, minus overlaps, up to max_atoms
    wpos, wsp, wmol, wbox = water_positions(n_box_waters, seed + 1)
    wpos = np.mod(wpos * (box / wbox), box)
    tree = cKDTree(sol_pos, boxsize=box)
    near = tree.query_ball_point(wpos, MIN_DIST, return_length=True) > 0
    n_w = int(wmol.max()) + 1
    bad = np.zeros(n_w, dtype=bool)
    np.logical_or.at(bad, wmol, near)
    keep_mols = np.nonzero(~bad)[0]
    keep_mols = keep_mols[rng.permutation(len(keep_mols))]
    room = max(0, (max_atoms - len(sol_pos)) // 3)
    keep_mols = np.sort(keep_mols[:room])
    keep = np.isin(wmol, keep_mols)
    remap = np.full(n_w, -1, dtype=np.int32)
    remap[keep_mols] = np.arange(len(keep_mols), dtype=np.int32) + n_chains
    pos = np.concatenate([sol_pos, wpos[keep]])
    species = np.concatenate([sol_sp, wsp[keep].astype(np.int8)])
    molecule = np.concatenate([sol_mol, remap[wmol[keep]]])
    H, orb_atom = tb_hamiltonian(pos, species, box)
    ne = int(sum(VALENCE[int(s)] for s in species))
    atom_core = rcb_cores(pos, core_atoms)
    return System(box=box, positions=pos, species=species, molecule=molecule, orb_atom=orb_atom, H=H,
                  n_electrons=ne, atom_core=atom_core,
                  meta={"kind": "chains", "n_chains": n_chains, "chain_len": chain_len,
                        "n_solute_atoms": len(sol_pos), "n_waters": len(keep_mols), "seed": seed,
                        "core_atoms": core_atoms})
