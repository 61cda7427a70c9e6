"""The oracle reproduces its recorded results (tests/golden/, CPU only).

The fixture was written by tests/golden/make_golden.py, which calls only the
oracle and the input generators.  Integer structure (graph, partition) must
match bit for bit.  Floating-point values get a margin for the BLAS/LAPACK of
another machine: water64's mu sits in a gap where dN/dmu is ~0.02 per eV, so
the 1e-12 N_occ stopping rule of the mu solve leaves mu ~1e-8 eV of freedom,
and D moves by at most ~d1_mu times that.  A change of the oracle's
arithmetic moves these values by far more.
"""

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_recorded_results():
    from tests.golden.make_golden import FIXTURE, compute
    rec = json.load(open(FIXTURE))
    now = compute()
    assert now["workload"] == rec["workload"]
    assert now["graph"] == rec["graph"]
    assert now["partition"] == rec["partition"]
    for key in ("graph_method", "full"):
        a, b = now[key], rec[key]
        assert abs(a["mu"] - b["mu"]) < 1e-7
        assert abs(a["mu1"] - b["mu1"]) < 1e-6 * abs(b["mu1"]) + 1e-12
        sa, sb = np.array(a["samples"]), np.array(b["samples"])
        assert np.array_equal(sa[:, :2], sb[:, :2])
        assert np.abs(sa[:, 2:] - sb[:, 2:]).max() < 1e-7
    g, r = now["graph_method"], rec["graph_method"]
    assert abs(g["trace_core"] - r["trace_core"]) < 1e-9
    assert abs(g["trace_d1mu"] - r["trace_d1mu"]) < 1e-6 * r["trace_d1mu"]
    assert np.abs(np.array(g["charges_first_8"]) - np.array(r["charges_first_8"])).max() < 1e-6
