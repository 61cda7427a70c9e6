"""The graph truncation table of the result notes, water64 rows (CPU only).

oracle/truncation.py compares the graph method's collected D and D1 with the
full diagonalisation.  On water64 (kT 0.1 eV, tau 1e-5) the recorded values
are re-derived here to two significant digits, and the error must shrink as
the graph grows from the H graph to the two-pass estimate and to paths of two.
"""

import pytest

from oracle.truncation import truncation
from synth import make_workload

# graph -> (max|dD|, max|dD1|, mu_graph - mu_full in eV), as recorded
RECORDED = {"H": (1.3e-2, 2.3e-3, 0.20), "two-pass": (4.8e-4, 8.1e-5, 0.70), "paths2": (4.0e-4, 1.5e-4, -0.26)}


def test_water64_truncation_rows():
    wl, system, h1 = make_workload("water64", n_rhs=1)
    H = system.H
    rows = {}
    eD, eD1, dmu, _, _, g = truncation(H, h1, 0.1, system.n_occ, system.orb_group, wl.tau)
    rows["H"] = (eD, eD1, dmu)
    rows["two-pass"] = truncation(H, h1, 0.1, system.n_occ, system.orb_group, wl.tau, d_prev=g.D)[:3]
    rows["paths2"] = truncation(H, h1, 0.1, system.n_occ, system.orb_group, wl.tau, paths2=True)[:3]
    for key, (rD, rD1, rmu) in RECORDED.items():
        eD, eD1, dmu = rows[key]
        assert eD == pytest.approx(rD, rel=0.05) and eD1 == pytest.approx(rD1, rel=0.05), key
        assert dmu == pytest.approx(rmu, abs=0.006), key
    assert rows["paths2"][0] < rows["two-pass"][0] < rows["H"][0]
