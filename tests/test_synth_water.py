"""The water generator follows its stated recipe (CPU only).

Inputs are synthetic: the seeded water boxes stand in for the paper's water
workloads.  These checks tie the generator to the recipe by invariants that
do not restate its code: molecular geometry, density, electron count, the
rotation invariants of the Slater-Koster blocks, the parity of the s-p
hopping, the hopping cutoff, and two routes to the perturbation potential.
"""

import numpy as np
import pytest

from synth import make_workload, softened_coulomb_matrix, water_box
from synth.water import softened_coulomb_potential, water_perturbation

T0 = {"ss": -3.5, "sp": 3.0, "pps": 4.0, "ppp": -1.2}
ONSITE = {"O": (-23.9, -9.3), "H": (-6.5,)}


def _radial(r):
    return np.exp(-(r - 1.0) / 0.5)


def _min_image(d, box):
    return d - box * np.round(d / box)


@pytest.fixture(scope="module")
def water64():
    return make_workload("water64")[1]


def test_box_density_counts_and_molecules(water64):
    s = water64
    assert abs(s.box - (64 * 29.915) ** (1 / 3)) < 1e-12 and abs(s.box - 12.42) < 0.01
    assert s.n_atoms == 192 and s.n_orb == 384 and s.n_electrons == 512 and s.n_occ == 256
    pos = s.positions.reshape(64, 3, 3)
    assert np.all((s.positions >= 0) & (s.positions < s.box))
    oh1 = _min_image(pos[:, 1] - pos[:, 0], s.box)
    oh2 = _min_image(pos[:, 2] - pos[:, 0], s.box)
    r1, r2 = np.linalg.norm(oh1, axis=1), np.linalg.norm(oh2, axis=1)
    np.testing.assert_allclose(r1, 0.9572, atol=1e-12)
    np.testing.assert_allclose(r2, 0.9572, atol=1e-12)
    ang = np.degrees(np.arccos(np.sum(oh1 * oh2, axis=1) / (r1 * r2)))
    np.testing.assert_allclose(ang, 104.52, atol=1e-9)
    # every orbital of a molecule shares its core id
    assert np.array_equal(s.orb_group, s.molecule[s.orb_atom])


def test_tight_binding_blocks(water64):
    s = water64
    H = s.H.to_dense()
    assert np.array_equal(H, H.T)
    first = np.concatenate([[0], np.cumsum(np.bincount(s.orb_atom))])
    name = {0: "H", 3: "O"}
    for a in range(s.n_atoms):
        sp = name[int(s.species[a])]
        o = slice(first[a], first[a + 1])
        block = H[o, o]
        assert np.array_equal(np.diag(block), [ONSITE[sp][0]] + [ONSITE[sp][-1]] * (len(np.diag(block)) - 1))
        assert not np.any(block - np.diag(np.diag(block)))          # no intra-atomic hoppings
    checked = 0
    for a in range(s.n_atoms):
        for b in range(a + 1, s.n_atoms):
            d = _min_image(s.positions[b] - s.positions[a], s.box)
            r = np.linalg.norm(d)
            blk = H[first[a]:first[a + 1], first[b]:first[b + 1]]
            if r >= 4.0:
                assert not np.any(blk)                                 # hard 4 A cutoff
                continue
            v = {k: t * _radial(r) for k, t in T0.items()}
            kinds = (name[int(s.species[a])], name[int(s.species[b])])
            # rotation invariants: the squared norm of the block depends on r only
            norm2 = {("O", "O"): v["ss"] ** 2 + 2 * v["sp"] ** 2 + v["pps"] ** 2 + 2 * v["ppp"] ** 2,
                     ("O", "H"): v["ss"] ** 2 + v["sp"] ** 2, ("H", "O"): v["ss"] ** 2 + v["sp"] ** 2,
                     ("H", "H"): v["ss"] ** 2}[kinds]
            assert abs(np.sum(blk ** 2) - norm2) < 1e-12 * max(1.0, norm2)
            if kinds == ("O", "O"):
                # the p-p block has eigenvalues pp_sigma (along d) and pp_pi (twice)
                w = np.sort(np.linalg.eigvalsh(0.5 * (blk[1:, 1:] + blk[1:, 1:].T)))
                np.testing.assert_allclose(w, np.sort([v["pps"], v["ppp"], v["ppp"]]), atol=1e-12)
            if kinds == ("O", "H"):
                # s-p parity: <p_a on O | H | s on H> = -l_a V_sp, l from O to H
                np.testing.assert_allclose(blk[1:, 0], -d / r * v["sp"], atol=1e-12)
            if kinds == ("H", "O"):
                np.testing.assert_allclose(blk[0, 1:], d / r * v["sp"], atol=1e-12)
            checked += 1
    assert checked > 1000


@pytest.mark.parametrize("n_waters", [64, 400])
def test_perturbation_is_the_softened_coulomb_sum(n_waters):
    # two codings of v_i = sum_j dq_j / sqrt(r_ij^2 + 1) over periodic images
    # within 10 A: the potential routine (image loop below a 20 A box, a
    # periodic tree above) and the matrix C applied to dq
    s = water_box(n_waters, 1234 + n_waters)
    dq = np.random.default_rng(5).normal(0.0, 0.1, s.n_atoms)
    C = softened_coulomb_matrix(s.positions, s.box)
    Cd = np.zeros((s.n_atoms, s.n_atoms))
    Cd[np.repeat(np.arange(s.n_atoms), np.diff(C.indptr)), C.indices] = C.data
    np.testing.assert_allclose(np.diag(Cd), 1.0, atol=1e-15)                # r = 0: no image within 10 A
    assert np.allclose(Cd, Cd.T, atol=1e-13)
    np.testing.assert_allclose(softened_coulomb_potential(s.positions, s.box, dq), Cd @ dq, atol=1e-11)


def test_perturbation_recipe(water64):
    # H1 = diag(v[atom(o)]) with v = C dq, dq of variance 0.01 and zero sum:
    # recover dq from v through C and check its moments
    s = water64
    h1 = water_perturbation(s, 20221204 + 100)
    assert np.array_equal(h1.indices, np.arange(s.n_orb)) and np.array_equal(h1.indptr, np.arange(s.n_orb + 1))
    first = np.concatenate([[0], np.cumsum(np.bincount(s.orb_atom))])
    v = h1.data[first[:-1]]
    assert np.array_equal(h1.data, v[s.orb_atom])                      # one value per atom
    C = softened_coulomb_matrix(s.positions, s.box)
    Cd = np.zeros((s.n_atoms, s.n_atoms))
    Cd[np.repeat(np.arange(s.n_atoms), np.diff(C.indptr)), C.indices] = C.data
    dq = np.linalg.solve(Cd, v)
    assert abs(dq.sum()) < 1e-8
    assert 0.07 < dq.std() < 0.13


def test_thermal_trajectory_recipe(water64):
    # force-free steps x += v dt (dt 0.25 fs, wrapped) with Maxwell velocities
    # at 300 K: constant displacement per step, per-axis velocity spread
    # sqrt(kB T / m) for each species
    from synth.water import thermal_trajectory
    s = water64
    steps = list(thermal_trajectory(s, 3, seed=20221204 + 1000))
    d1 = _min_image(steps[0] - s.positions, s.box)
    d2 = _min_image(steps[1] - steps[0], s.box)
    np.testing.assert_allclose(d2, d1, atol=1e-12)
    assert np.all((steps[2] >= 0) & (steps[2] < s.box))
    v = d1 / 0.25                                              # A/fs
    kB, conv = 8.617333262e-5, 0.0982269                       # eV/K; sqrt(eV/amu) in A/fs
    for code, mass in ((0, 1.008), (3, 15.999)):
        sigma = np.sqrt(kB * 300.0 / mass) * conv
        got = v[s.species == code].std()
        assert abs(got / sigma - 1.0) < 0.15, (code, got, sigma)
