"""Planted mistakes in the oracle fail its pins (CPU only).

The oracle is trusted because the pins tie it to facts other than itself:
closed forms, brute force, finite differences and identities the paper
states.  This file checks that those pins are sharp.  Each case takes the
source of one oracle function, plants one plausible mistake in it (a flipped
sign, a dropped term or factor, a wrong index, a transposed operand, a
threshold that is not strict), binds the altered function wherever the
original is bound, and runs the pins named for the case: at least one of
them must fail.  The unaltered oracle passes every pin used here (first
test), so a failure is the planted mistake's doing.

Not planted: a sign error in the Newton polish of ``solve_mu``.  The
bisection before it already narrows the bracket to ~1e-13 relative, so a
wrong Newton step leaves the bracket, is rejected, and mu stays exact; that
mistake changes no result.
"""

import __future__
import importlib
import importlib.util
import inspect
import os

import pytest

import oracle
from synth import make_workload

HERE = os.path.dirname(os.path.abspath(__file__))


def _load_pins(name):
    """The pin file as a private module, so it can be rebound freely."""
    spec = importlib.util.spec_from_file_location(f"_pins_{name}", os.path.join(HERE, f"test_oracle_{name}.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# the submodules by name: the package re-exports functions that shadow some of them
F, S, G, K = (importlib.import_module(f"oracle.{m}") for m in ("fermi", "solve", "graph", "krylov"))
PINS = {name: _load_pins(name) for name in ("fermi", "solve", "graph", "krylov")}
MODULES = (oracle, F, S, G, K, *PINS.values())

# (id, module, function, [(text, replacement), ...], pins that must catch it)
MUTANTS = [
    # Fermi function, its weight and divided difference (Eqs. Fermi, ddlambda, dddmu)
    ("fermi-sign", F, "fermi",
     [("expit(-(np.asarray(eps, dtype=np.float64) - mu) / kT)", "expit((np.asarray(eps, dtype=np.float64) - mu) / kT)")],
     ["fermi:test_fermi_limits_and_symmetry", "fermi:test_one_state_chemical_potential_closed_form"]),
    ("fermi-weight-square-dropped", F, "fermi_weight",
     [("return e / (1.0 + e) ** 2", "return e / (1.0 + e)")],
     ["fermi:test_fermi_weight_is_f_one_minus_f", "fermi:test_grand_canonical_response_is_derivative"]),
    ("divided-difference-factor", F, "fermi_divided_difference",
     [("-(beta / 4.0) * ratio * core", "-(beta / 2.0) * ratio * core")],
     ["fermi:test_divided_difference_off_diagonal_and_diagonal"]),
    ("divided-difference-exponent-sign", F, "fermi_divided_difference",
     [("np.exp(y - aa - bb)", "np.exp(y - aa + bb)")],
     ["fermi:test_divided_difference_off_diagonal_and_diagonal"]),
    ("divided-difference-sinhc-sign", F, "fermi_divided_difference",
     [("-np.expm1(-2.0 * y) / (2.0 * y)", "np.expm1(-2.0 * y) / (2.0 * y)")],
     ["fermi:test_divided_difference_off_diagonal_and_diagonal"]),
    ("occupation-derivative-kT-for-beta", F, "occupation",
     [("return n, dn / kT", "return n, dn * kT")],
     ["fermi:test_newton_converges_quadratically"]),
    ("bisection-direction", F, "solve_mu",
     [("if n_mid < n_occ:", "if n_mid > n_occ:")],
     ["fermi:test_one_state_chemical_potential_closed_form", "solve:test_full_trace_symmetry_and_occupation"]),
    ("density-transposed", F, "dense_density",
     [("(V * fermi(eps, mu, kT)) @ V.T", "(V.T * fermi(eps, mu, kT)) @ V")],
     ["fermi:test_two_by_two_density_closed_form", "fermi:test_density_against_matrix_exponential"]),
    ("response-back-transform-transposed", F, "dense_response",
     [("d1lam = V @ (F * h1p) @ V.T", "d1lam = V.T @ (F * h1p) @ V")],
     ["fermi:test_grand_canonical_response_is_derivative",
      "solve:test_full_response_equals_canonical_finite_difference"]),
    ("response-projection-transposed", F, "dense_response",
     [("h1p = V.T @ h1 @ V", "h1p = V @ h1 @ V.T")],
     ["fermi:test_grand_canonical_response_is_derivative",
      "solve:test_full_response_equals_canonical_finite_difference"]),
    ("d1mu-kT-for-beta", F, "dense_response",
     [("(fermi_weight(eps, mu, kT) / kT)", "(fermi_weight(eps, mu, kT) * kT)")],
     ["fermi:test_grand_canonical_response_is_derivative"]),
    # full and graph solutions (Eqs. D1, dmu_1, NewtonRaphson, DD)
    ("full-mu1-sign", S, "oracle_full",
     [("m1 = -np.trace(d1lam) / np.trace(d1mu)", "m1 = np.trace(d1lam) / np.trace(d1mu)")],
     ["solve:test_full_trace_symmetry_and_occupation", "solve:test_full_response_equals_canonical_finite_difference"]),
    ("full-D1-drops-mu1-term", S, "oracle_full",
     [("D1.append(d1lam + m1 * d1mu)", "D1.append(d1lam)")],
     ["solve:test_full_trace_symmetry_and_occupation", "solve:test_full_response_equals_canonical_finite_difference"]),
    ("core-weights-over-all-rows", S, "_spectrum_task",
     [("np.sum(V[core_local, :] ** 2, axis=0)", "np.sum(V ** 2, axis=0)")],
     ["solve:test_graph_invariants_and_canonical_finite_difference"]),
    ("core-weights-transposed", S, "_spectrum_task",
     [("np.sum(V[core_local, :] ** 2, axis=0)", "np.sum(V[:, core_local] ** 2, axis=1)")],
     ["solve:test_graph_invariants_and_canonical_finite_difference"]),
    ("d1lam-trace-over-subgraph", S, "_response_task",
     [("np.trace(d1lam[np.ix_(core_local, core_local)])", "np.trace(d1lam)")],
     ["solve:test_graph_invariants_and_canonical_finite_difference"]),
    ("d1mu-trace-wrong-rows", S, "_response_task",
     [("tr_mu = float(np.trace(d1mu_c[core_local, :]))", "tr_mu = float(np.trace(d1mu_c))")],
     ["solve:test_graph_invariants_and_canonical_finite_difference"]),
    ("graph-occupation-derivative-uses-f", S, "oracle_graph",
     [("tr_dd = sum(float(np.dot(fermi_weight(e, mu, kT), w))", "tr_dd = sum(float(np.dot(fermi(e, mu, kT), w))")],
     ["solve:test_graph_invariants_and_canonical_finite_difference"]),
    ("graph-mu1-term-sign", S, "oracle_graph",
     [("d1_c[r] + mu1[r] * d1mu_c", "d1_c[r] - mu1[r] * d1mu_c")],
     ["solve:test_graph_invariants_and_canonical_finite_difference", "solve:test_graph_exact_on_disconnected_blocks"]),
    ("graph-mu1-sign", S, "oracle_graph",
     [("mu1 = -tr1 / tr_mu if m else np.zeros(0)", "mu1 = tr1 / tr_mu if m else np.zeros(0)")],
     ["solve:test_graph_exact_on_disconnected_blocks"]),
    ("mulliken-sign", S, "mulliken_charges",
     [("return z_val - pop", "return pop - z_val")],
     ["solve:test_mulliken_two_atom_closed_form"]),
    ("mulliken-spin-factor", S, "mulliken_charges",
     [("np.add.at(pop, orb_atom, 2.0 * diag)", "np.add.at(pop, orb_atom, diag)")],
     ["solve:test_mulliken_two_atom_closed_form", "solve:test_mulliken_response_is_the_charge_derivative"]),
    # graph estimate, partition and collect (Sec. "Estimating the connectivity graph", Eq. sub_f)
    ("threshold-not-strict", G, "_pattern",
     [("np.abs(np.asarray(data)) > tau", "np.abs(np.asarray(data)) >= tau")],
     ["graph:test_graph_threshold_is_strict"]),
    ("H-edges-not-symmetrised", G, "graph_build",
     [("rs, cs = [r, c], [c, r]", "rs, cs = [r], [c]")],
     ["graph:test_graph_symmetrises_one_sided_entries"]),
    ("D_prev-edges-not-symmetrised", G, "graph_build",
     [("rs += [dr, dc]", "rs += [dr]"), ("cs += [dc, dr]", "cs += [dc]")],
     ["graph:test_graph_symmetrises_one_sided_entries"]),
    ("paths2-self-loops-kept", G, "graph_build",
     [("        a.setdiag(0)\n", "")],
     ["graph:test_graph_build_matches_pair_enumeration:paths2=True"]),
    ("halo-of-one-core-vertex", G, "partition",
     [("for v in core:", "for v in core[:1]:")],
     ["graph:test_partition_matches_brute_force"]),
    ("core-positions-not-looked-up", G, "partition",
     [("core_pos.append(np.searchsorted(s, core))", "core_pos.append(np.arange(len(core)))")],
     ["graph:test_partition_matches_brute_force", "graph:test_sub_f_multi_vertex_cores_column_collect"]),
    ("collect-core-slots-reversed", G, "collect_columns",
     [("slot[c] = np.arange(len(c))", "slot[c] = np.arange(len(c))[::-1]")],
     ["graph:test_sub_f_multi_vertex_cores_column_collect"]),
    ("gather-columns-reversed", G, "gather",
     [("return X[s][:, s].toarray()", "return X[s][:, s[::-1]].toarray()"),
      ("np.asarray(X)[np.ix_(s, s)]", "np.asarray(X)[np.ix_(s, s[::-1])]")],
     ["graph:test_sub_f_single_vertex_cores", "solve:test_graph_with_one_subgraph_is_full"]),
    ("cap-not-strict", G, "partition_capped",
     [("np.nonzero(sizes > max_sub)", "np.nonzero(sizes >= max_sub)")],
     ["graph:test_partition_capped_rule_by_brute_force"]),
    # charge model, preconditioner and Krylov kernel (Eqs. PreCond, LowRankEEOM)
    ("charge-potential-sign", K, "charge_hamiltonian",
     [("np.asarray(n) - np.asarray(z)", "np.asarray(z) - np.asarray(n)")],
     ["krylov:test_single_core_jacobian_is_the_full_jacobian"]),
    ("populations-spin-factor", K, "atom_populations",
     [("return 2.0 * np.bincount", "return np.bincount")],
     ["krylov:test_single_core_jacobian_is_the_full_jacobian", "krylov:test_krylov_directional_derivatives"]),
    ("jacobian-neutrality-term-dropped", K, "core_jacobians",
     [("jc = chi + np.outer(rho_mu, mu1) - np.eye(na)", "jc = chi - np.eye(na)")],
     ["krylov:test_single_core_jacobian_is_the_full_jacobian",
      "krylov:test_subgraph_blocks_are_charge_neutral_and_inverted"]),
    ("jacobian-neutrality-term-transposed", K, "core_jacobians",
     [("np.outer(rho_mu, mu1)", "np.outer(mu1, rho_mu)")],
     ["krylov:test_single_core_jacobian_is_the_full_jacobian",
      "krylov:test_subgraph_blocks_are_charge_neutral_and_inverted"]),
    ("k0-alpha-sign", K, "core_jacobians",
     [("np.linalg.inv(jc - alpha * np.eye(na))", "np.linalg.inv(jc + alpha * np.eye(na))")],
     ["krylov:test_subgraph_blocks_are_charge_neutral_and_inverted"]),
    ("preconditioner-block-transposed", K, "apply_preconditioner",
     [("y[atoms] = k0 @ np.asarray(x)[atoms]", "y[atoms] = k0.T @ np.asarray(x)[atoms]")],
     ["krylov:test_subgraph_blocks_are_charge_neutral_and_inverted"]),
    ("krylov-drops-minus-v", K, "krylov_update",
     [("apply_preconditioner(blocks, drho - v)", "apply_preconditioner(blocks, drho)")],
     ["krylov:test_krylov_directional_derivatives", "krylov:test_full_rank_krylov_is_the_newton_step"]),
    ("krylov-overlap-not-inverted", K, "krylov_update",
     [("M = np.linalg.inv(O)", "M = O")],
     ["krylov:test_full_rank_krylov_is_the_newton_step"]),
    ("krylov-no-orthogonalisation", K, "krylov_update",
     [("w = fv - sum(float(fv @ vj) * vj for vj in vs)", "w = fv"),
      ("w = w - sum(float(w @ vj) * vj for vj in vs)", "w = w")],
     ["krylov:test_krylov_directional_derivatives"]),
]


@pytest.fixture(scope="module")
def fixtures():
    return {"water64": make_workload("water64"), "model": PINS["krylov"].krylov_model()}


def _run_pin(spec, fixtures):
    """Run one pin, "file:test[:name=value]", with its fixtures supplied."""
    parts = spec.split(":")
    fn = getattr(PINS[parts[0]], parts[1])
    given = {}
    for kv in parts[2:]:
        k, v = kv.split("=")
        given[k] = {"True": True, "False": False}.get(v, v)
    args = {p: given[p] if p in given else fixtures[p] for p in inspect.signature(fn).parameters}
    fn(**args)


def _mutant(module, name, edits):
    original = getattr(module, name)
    src = inspect.getsource(original)
    for text, replacement in edits:
        assert src.count(text) == 1, f"{name}: the planted text no longer occurs once in the oracle's source"
        src = src.replace(text, replacement)
    ns = dict(vars(module))
    exec(compile(src, inspect.getsourcefile(original), "exec",
                 flags=__future__.annotations.compiler_flag, dont_inherit=True), ns)
    return original, ns[name]


def test_pins_pass_on_the_unaltered_oracle(fixtures):
    for spec in sorted({p for case in MUTANTS for p in case[4]}):
        _run_pin(spec, fixtures)


@pytest.mark.parametrize("case", MUTANTS, ids=[case[0] for case in MUTANTS])
def test_planted_mistake_fails_a_pin(case, fixtures, monkeypatch):
    _, module, name, edits, pins = case
    original, mutant = _mutant(module, name, edits)
    for mod in MODULES:
        if getattr(mod, name, None) is original:
            monkeypatch.setattr(mod, name, mutant)
    caught = []
    for spec in pins:
        try:
            _run_pin(spec, fixtures)
        except Exception:  # noqa: BLE001 - an assertion, or numerics the mistake broke
            caught.append(spec)
    assert caught, f"no pin caught the planted mistake {case[0]!r}"
