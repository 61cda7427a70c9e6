"""The heterogeneous chain generator: its recipe's invariants (CPU)."""

import numpy as np

from synth import make_workload
from synth.chains import BONDS, H_BOND, MIN_DIST, chain_system, rcb_cores
from synth.system import SPECIES


def _min_image(d, box):
    return d - box * np.round(d / box)


def test_chain_recipe_invariants():
    s = chain_system(600, 2, 40, 2000, 30, 11)
    box = s.box
    heavy = np.nonzero(s.species != SPECIES["H"])[0]
    solute = np.nonzero(s.molecule < 2)[0]
    assert s.n_atoms <= 2000 and len(heavy) >= 80
    # chain atoms: consecutive heavy atoms of a chain are 1.5 A apart, the
    # others (beyond the two predecessors) at least 2.5 A apart
    for c in range(2):
        ch = heavy[s.molecule[heavy] == c]  # stored in chain order
        p = s.positions[ch]
        step = np.linalg.norm(_min_image(np.diff(p, axis=0), box), axis=1)
        assert np.allclose(step, 1.5, atol=1e-6)
        for i in range(len(ch)):
            for j in range(i + 3, len(ch)):
                assert np.linalg.norm(_min_image(p[j] - p[i], box)) >= MIN_DIST - 1e-9
    # valence: chain bonds plus hydrogens fill C 4, N 3, O 2; H at the stated lengths
    hyd = [a for a in solute if s.species[a] == SPECIES["H"]]
    nh = np.zeros(s.n_atoms, dtype=int)
    for h in hyd:
        d = np.linalg.norm(_min_image(s.positions[heavy] - s.positions[h], box), axis=1)
        a = heavy[np.argmin(d)]
        assert abs(d.min() - H_BOND[int(s.species[a])]) < 1e-6
        nh[a] += 1
    for c in range(2):
        ch = np.sort([a for a in heavy if s.molecule[a] == c])
        for k, a in enumerate(ch):
            nb = (k > 0) + (k + 1 < len(ch))
            assert nh[a] + nb == BONDS[int(s.species[a])]
    # waters keep 2.5 A from the solute; molecules are chains then waters
    wat = np.nonzero(s.molecule >= 2)[0]
    d = np.linalg.norm(_min_image(s.positions[wat][:, None, :] - s.positions[solute][None], box), axis=2)
    assert d.min() >= MIN_DIST - 1e-9
    assert np.all(np.bincount(s.molecule[wat] - 2) == 3)
    # neutral valence electrons
    assert s.n_electrons == int(sum({0: 1, 1: 4, 2: 5, 3: 6}[int(x)] for x in s.species))


def test_rcb_cores_cover_and_bound():
    rng = np.random.default_rng(3)
    pos = rng.random((1000, 3)) * 50.0
    core = rcb_cores(pos, 30)
    sizes = np.bincount(core)
    assert sizes.sum() == 1000 and sizes.max() <= 30 and sizes.min() >= 15
    assert np.array_equal(core, rcb_cores(pos, 30))  # deterministic


def test_chain_workload_is_deterministic_and_grouped_by_cores():
    wl, a, h1 = make_workload("chains_small")
    _, b, _ = make_workload("chains_small")
    assert np.array_equal(a.positions, b.positions) and np.array_equal(a.H.data, b.H.data)
    assert np.array_equal(a.orb_group, a.atom_core[a.orb_atom])
    assert a.atom_core.max() + 1 >= a.n_atoms // 30
    assert len(h1) == 1 and h1[0].n == a.n_orb
