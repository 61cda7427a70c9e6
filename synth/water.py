"""Seeded water boxes with an orthogonal sp tight-binding Hamiltonian.

Recipe (inputs only, stated so a reader can rebuild them):

* Density 1.0 g/cm^3: 29.915 A^3 per molecule, cubic box L = (N_w * 29.915)^(1/3).
* Molecules sit on the smallest cubic lattice with n^3 >= N_w; sites are filled
  in a seeded random order; the oxygen of each molecule is the site centre plus
  a Gaussian jitter of 0.3 A per axis; each molecule gets a uniform random
  rotation (random unit quaternion).  O-H 0.9572 A, H-O-H 104.52 degrees.
* Basis: O has s, px, py, pz; H has s.  Onsites O_s -23.9, O_p -9.3, H_s -6.5 eV
  (C_s -13.6, C_p -5.4, N_s -18.5, N_p -7.2 eV for other species).
* Two-centre Slater-Koster hoppings V(r) = t0 exp(-(r - 1.0 A) / 0.5 A) with
  t0 = ss -3.5, sp 3.0, pp_sigma 4.0, pp_pi -1.2 eV, hard cutoff 4 A, minimum
  image, no intra-atomic hoppings.  For orbitals on atoms I, J and direction
  cosines l of R_J - R_I:  E_ss = V_ss;  E_(s on I, p_b on J) = l_b V_sp;
  E_(p_a on I, s on J) = -l_a V_sp;  E_(p_a, p_b) = l_a l_b (V_pps - V_ppp)
  + delta_ab V_ppp.
* Perturbation H1 = diag(v): per atom v_i = sum_j dq_j / sqrt(r_ij^2 + 1 A^2)
  over all atoms j and periodic images with r_ij < 10 A (j = i included),
  dq ~ N(0, variance 0.01) shifted to zero sum; every orbital of atom i gets v_i.
* Electron count: neutral valence (O 6, H 1, C 4, N 5).
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .system import CSR, N_ORB, SPECIES, VALENCE, System

VOLUME_PER_WATER = 29.915  # A^3 at 1.0 g/cm^3 (18.015 g/mol)
R_OH = 0.9572
ANGLE_HOH = np.deg2rad(104.52)
JITTER = 0.3

ONSITE = {
    SPECIES["H"]: (-6.5,),
    SPECIES["C"]: (-13.6, -5.4),
    SPECIES["N"]: (-18.5, -7.2),
    SPECIES["O"]: (-23.9, -9.3),
}
T0 = {"ss": -3.5, "sp": 3.0, "pps": 4.0, "ppp": -1.2}
R0 = 1.0
DECAY = 0.5
CUTOFF = 4.0
H1_CUTOFF = 10.0


def water_box_edge(n_waters: int) -> float:
    return float((n_waters * VOLUME_PER_WATER) ** (1.0 / 3.0))


def _lattice_side(n: int) -> int:
    k = 1
    while k ** 3 < n:
        k += 1
    return k


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    x, y = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    z, w = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    rot = np.empty((n, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return rot


def water_positions(n_waters: int, seed: int):
    """Positions (n_atoms, 3), species, molecule ids and the box edge."""
    rng = np.random.default_rng(seed)
    box = water_box_edge(n_waters)
    side = _lattice_side(n_waters)
    spacing = box / side
    sites = rng.permutation(side ** 3)[:n_waters]
    ijk = np.stack([sites // (side * side), (sites // side) % side, sites % side], axis=1)
    centre = (ijk + 0.5) * spacing + rng.normal(0.0, JITTER, size=(n_waters, 3))
    rot = _random_rotations(rng, n_waters)
    half = ANGLE_HOH / 2.0
    frame = np.array([[0.0, 0.0, 0.0],
                      [R_OH * np.sin(half), R_OH * np.cos(half), 0.0],
                      [-R_OH * np.sin(half), R_OH * np.cos(half), 0.0]])
    pos = centre[:, None, :] + np.einsum("mij,aj->mai", rot, frame)
    pos = np.mod(pos.reshape(-1, 3), box)
    species = np.tile(np.array([SPECIES["O"], SPECIES["H"], SPECIES["H"]], dtype=np.int8), n_waters)
    molecule = np.repeat(np.arange(n_waters, dtype=np.int32), 3)
    return pos, species, molecule, box


def _orbital_layout(species: np.ndarray):
    norb = np.array([N_ORB[int(s)] for s in species], dtype=np.int64)
    first = np.zeros(len(species) + 1, dtype=np.int64)
    first[1:] = np.cumsum(norb)
    orb_atom = np.repeat(np.arange(len(species), dtype=np.int32), norb)
    return norb, first, orb_atom


def tb_hamiltonian(pos: np.ndarray, species: np.ndarray, box: float) -> tuple[CSR, np.ndarray]:
    """Orthogonal sp Slater-Koster Hamiltonian (CSR, eV) and orbital->atom map."""
    norb, first, orb_atom = _orbital_layout(species)
    n = int(first[-1])
    rows, cols, vals = [], [], []
    # onsite terms
    for a in range(len(species)):
        eps = ONSITE[int(species[a])]
        for k in range(norb[a]):
            o = first[a] + k
            rows.append(np.array([o]))
            cols.append(np.array([o]))
            vals.append(np.array([eps[0] if k == 0 else eps[1]]))
    tree = cKDTree(pos, boxsize=box)
    pairs = tree.query_pairs(CUTOFF, output_type="ndarray")
    if len(pairs):
        i, j = pairs[:, 0], pairs[:, 1]
        d = pos[j] - pos[i]
        d -= box * np.round(d / box)
        r = np.linalg.norm(d, axis=1)
        keep = r < CUTOFF
        i, j, d, r = i[keep], j[keep], d[keep], r[keep]
        l = d / r[:, None]
        radial = np.exp(-(r - R0) / DECAY)
        vss, vsp = T0["ss"] * radial, T0["sp"] * radial
        vpps, vppp = T0["pps"] * radial, T0["ppp"] * radial
        # full 4x4 block (s, px, py, pz) x (s, px, py, pz) for orbital a on I, b on J
        blk = np.zeros((len(i), 4, 4))
        blk[:, 0, 0] = vss
        blk[:, 0, 1:] = l * vsp[:, None]
        blk[:, 1:, 0] = -l * vsp[:, None]
        blk[:, 1:, 1:] = (l[:, :, None] * l[:, None, :]) * (vpps - vppp)[:, None, None]
        blk[:, 1:, 1:] += np.eye(3)[None] * vppp[:, None, None]
        ni, nj = norb[i], norb[j]
        for a in range(4):
            for b in range(4):
                m = (a < ni) & (b < nj)
                if not np.any(m):
                    continue
                oi = first[i[m]] + a
                oj = first[j[m]] + b
                v = blk[m, a, b]
                rows += [oi, oj]
                cols += [oj, oi]
                vals += [v, v]
    H = CSR.from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return H, orb_atom


def water_box(n_waters: int, seed: int) -> System:
    """A seeded periodic water box with its tight-binding Hamiltonian."""
    pos, species, molecule, box = water_positions(n_waters, seed)
    H, orb_atom = tb_hamiltonian(pos, species, box)
    ne = int(sum(VALENCE[int(s)] for s in species))
    return System(box=box, positions=pos, species=species, molecule=molecule,
                  orb_atom=orb_atom, H=H, n_electrons=ne,
                  meta={"kind": "water", "n_waters": n_waters, "seed": seed})


def softened_coulomb_potential(pos: np.ndarray, box: float, dq: np.ndarray,
                               cutoff: float = H1_CUTOFF) -> np.ndarray:
    """v_i = sum_j dq_j / sqrt(r_ij^2 + 1) over all periodic images with r_ij < cutoff."""
    n = len(pos)
    v = np.zeros(n)
    nimg = int(np.ceil(cutoff / box))
    shifts = np.array([(a, b, c) for a in range(-nimg, nimg + 1)
                       for b in range(-nimg, nimg + 1)
                       for c in range(-nimg, nimg + 1)], dtype=np.float64) * box
    if box >= 2.0 * cutoff:
        tree = cKDTree(pos, boxsize=box)
        sdm = tree.sparse_distance_matrix(tree, cutoff, output_type="coo_matrix")
        r = sdm.data
        np.add.at(v, sdm.row, dq[sdm.col] / np.sqrt(r * r + 1.0))
        # the self term (j = i, r = 0) is part of the distance matrix
        if not np.any(sdm.row == sdm.col):
            v += dq
        return v
    tree = cKDTree(pos)
    for s in shifts:
        img = pos + s
        lists = tree.query_ball_point(img, cutoff)
        for j, nb in enumerate(lists):
            if not nb:
                continue
            nb = np.asarray(nb)
            r = np.linalg.norm(pos[nb] - img[j], axis=1)
            v[nb] += dq[j] / np.sqrt(r * r + 1.0)
    return v


def softened_coulomb_matrix(pos: np.ndarray, box: float, cutoff: float = H1_CUTOFF) -> CSR:
    """C_IJ = sum over periodic images of J within the cutoff of 1 / sqrt(r_IJ^2 + 1)
    (atoms x atoms, J = I included): the charge -> on-site potential map of the
    perturbation model, v = C dq (softened_coulomb_potential applies the same sum)."""
    import scipy.sparse as sp
    n = len(pos)
    if box >= 2.0 * cutoff:
        tree = cKDTree(pos, boxsize=box)
        sdm = tree.sparse_distance_matrix(tree, cutoff, output_type="coo_matrix")
        off = sdm.row != sdm.col
        rows = np.concatenate([sdm.row[off], np.arange(n)])
        cols = np.concatenate([sdm.col[off], np.arange(n)])
        vals = np.concatenate([1.0 / np.sqrt(sdm.data[off] ** 2 + 1.0), np.ones(n)])
    else:
        nimg = int(np.ceil(cutoff / box))
        tree = cKDTree(pos)
        rows, cols, vals = [], [], []
        for a in range(-nimg, nimg + 1):
            for b in range(-nimg, nimg + 1):
                for c in range(-nimg, nimg + 1):
                    img = pos + np.array([a, b, c], dtype=np.float64) * box
                    for j, nb in enumerate(tree.query_ball_point(img, cutoff)):
                        if not nb:
                            continue
                        nb = np.asarray(nb)
                        r = np.linalg.norm(pos[nb] - img[j], axis=1)
                        rows.append(nb)
                        cols.append(np.full(len(nb), j))
                        vals.append(1.0 / np.sqrt(r * r + 1.0))
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    m = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64))


def water_perturbation(system: System, seed: int) -> CSR:
    """H1 = diag(v) from seeded charge fluctuations (variance 0.01, zero sum)."""
    rng = np.random.default_rng(seed)
    dq = rng.normal(0.0, 0.1, size=system.n_atoms)
    dq -= dq.mean()
    v_atom = softened_coulomb_potential(system.positions, system.box, dq)
    v = v_atom[system.orb_atom]
    n = system.n_orb
    idx = np.arange(n)
    return CSR(n, np.arange(n + 1, dtype=np.int64), idx.astype(np.int32), v.astype(np.float64))


AMU_EV_TO_A_PER_FS = 0.0982269  # sqrt(1 eV / 1 amu) in A/fs
KB_EV = 8.617333262e-5
MASS = {SPECIES["H"]: 1.008, SPECIES["C"]: 12.011, SPECIES["N"]: 14.007, SPECIES["O"]: 15.999}


def thermal_trajectory(system: System, n_steps: int, seed: int, temperature: float = 300.0,
                       dt_fs: float = 0.25):
    """Positions along a force-free trajectory with Maxwell velocities (x += v dt, wrapped)."""
    rng = np.random.default_rng(seed)
    mass = np.array([MASS[int(s)] for s in system.species])
    sigma = np.sqrt(KB_EV * temperature / mass) * AMU_EV_TO_A_PER_FS
    vel = rng.normal(size=(system.n_atoms, 3)) * sigma[:, None]
    pos = system.positions.copy()
    for _ in range(n_steps):
        pos = np.mod(pos + vel * dt_fs, system.box)
        yield pos.copy()
