"""The oracle's pins catch plausible mistakes (no GPU).

Each case below plants one mistake in a copy of the C oracle, compiles the
copy with the oracle's own flags, loads it through a fresh instance of the
oracle's marshalling module and runs every pin of test_oracle.py and
test_oracle_force.py named for it against it: that pin must fail.  The unmodified
source, built and loaded the same way, must pass every pin, so a failure can
only come from the planted mistake.  The mistakes are the ones a from-scratch
implementation of the staggered operator, its CG and its force is likely to
make: a transposed instead of adjoint link, the wrong eta ordering, a boundary
sign on one hop direction or on the wrong three-hop links, the backward link
read at the wrong site, the sign of the normal operator, a rescaled Naik term,
the CG coefficients, and the force's parity sign, field roles, trace term,
conjugation and Naik coefficient.  Two more are planted in the marshalling
module's pseudofermion phi = (M^+ chi)_e: the hopping term with the wrong sign
and m^2 in place of m.
"""

import importlib.util
import os

import pytest

import test_oracle as T
import test_oracle_force as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qex_oracle.c")
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")

# name -> (text in qex_oracle.c, replacement, occurrences, pin that must fail)
MUTANTS = {
    "transpose_not_adjoint": ("t += conj(M[3 * b + a]) * v[b];", "t += M[3 * b + a] * v[b];", 1, "antihermitian"),
    "conjugate_not_transposed": ("t += conj(M[3 * b + a]) * v[b];", "t += conj(M[3 * a + b]) * v[b];", 1,
                                 "antihermitian"),
    "eta_from_later_coordinates": ("for (int nu = 0; nu < mu; ++nu) s += x[nu];",
                                   "for (int nu = mu + 1; nu < 4; ++nu) s += x[nu];", 1, "point_source"),
    "no_antiperiodic_sign": ("if (!antiperiodic || mu != 3) return 1;", "return 1;", 1, "free_spectrum"),
    "sign_on_forward_hop_only": ("add_mdagv(acc, -oracle_eta(mu, y) * oracle_link_bc(L, antiperiodic, mu, y, 1),",
                                 "add_mdagv(acc, -oracle_eta(mu, y),", 1, "antihermitian"),
    "three_hop_sign_as_one_hop": ("oracle_link_bc(L, antiperiodic, mu, x, 3)", "oracle_link_bc(L, antiperiodic, mu, x, 1)",
                                  1, "point_source"),
    "backward_link_at_x": ("                  link_at(U, ly, mu), in + 3 * ly);",
                           "                  link_at(U, s, mu), in + 3 * ly);", 1, "gauge_covariance"),
    "normal_op_sign": ("out[i] = mass * mass * in_e[i] - even[i];", "out[i] = mass * mass * in_e[i] + even[i];", 1,
                       "free_spectrum"),
    "naik_rescaled": ("add_mv(acc, c3 * oracle_eta(mu, x)", "add_mv(acc, 1.125 * c3 * oracle_eta(mu, x)", 1,
                      "free_spectrum"),
    "cg_beta_inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;", 1, "dense_cg"),
    "cg_step_sign": ("x[i] += alpha * p[i];", "x[i] -= alpha * p[i];", 1, "dense_cg"),
    "force_no_parity_sign": ("if (!even) sgn = -sgn;", "", 1, "force_fd"),
    "force_fields_swapped": ("const cplx *a = even ? Y + 3 * ly : X + 3 * ly;",
                             "const cplx *a = even ? X + 3 * ly : Y + 3 * ly;", 1, "force_fd"),
    "force_trace_term": ("if (i == j) ta -= tr / 6.0;", "if (i == j) ta -= tr / 3.0;", 1, "force_traceless"),
    "force_no_conjugate": ("G[3 * i + j] = sgn * a[i] * conj(b[j]);", "G[3 * i + j] = sgn * a[i] * b[j];", 1,
                           "force_fd"),
    "force_long_links_without_c3": ("force_links(L, antiperiodic, W, c3, 3, X, Y, kind, out_long);",
                                    "force_links(L, antiperiodic, W, 1.0, 3, X, Y, kind, out_long);", 1, "force_fd"),
}

# the same, planted in the marshalling module (the C source is left intact)
PY_MUTANTS = {
    "pseudofermion_hop_sign": ("phi = mass * chi - dch", "phi = mass * chi + dch", 1, "pseudofermion"),
    "pseudofermion_mass_squared": ("phi = mass * chi - dch", "phi = mass * mass * chi - dch", 1, "pseudofermion"),
}


def _runs(*calls):
    def run(m):
        for c in calls:
            c(m)
    return run


# every pin of the two pin modules, with their own parameters
PINS = {
    "eo_table": _runs(*[lambda m, d=d: T.test_eo_table_is_parity_ordered_bijection(m, d)
                        for d in T.SHAPES + [(2, 2, 2, 2), (8, 4, 6, 2)]]),
    "neighbor_tables": _runs(*[lambda m, d=d: T.test_neighbor_tables_invariants(m, d) for d in T.SHAPES],
                             T.test_neighbor_table_hand_example),
    "antihermitian": _runs(*[lambda m, d=d, n=n, a=a: T.test_antihermitian(m, d, n, a)
                             for d in T.SHAPES for n in (False, True) for a in (False, True)]),
    "sampled_sites": _runs(T.test_dslash_at_sampled_sites_equals_full_lattice),
    "gauge_covariance": _runs(*[lambda m, n=n: T.test_gauge_covariance(m, n) for n in (False, True)]),
    "point_source": _runs(*[lambda m, n=n: T.test_point_source_hand_values(m, n) for n in (False, True)]),
    "free_spectrum": _runs(*[lambda m, d=d, k=k, c=c, a=a: T.test_free_field_spectrum(m, d, k, c, a)
                             for d, k in T.FREE_CASES for c in (0.0, T.C3) for a in (False, True)],
                           T.test_free_field_full_spectrum_dense),
    "dense_cg": _runs(*[lambda m, n=n: T.test_dense_normal_operator_and_cg(m, n) for n in (False, True)],
                      T.test_cg_plane_wave_exact, T.test_cg_true_residual_and_workload_cfg4,
                      T.test_cg_zero_source_and_maxiter),
    "force_fd": _runs(*[lambda m, n=n: F.test_force_matches_finite_differences_su3(m, n) for n in (False, True)],
                      F.test_gradient_form_matches_finite_differences),
    "force_traceless": _runs(F.test_force_is_traceless_antihermitian_and_relates_to_gradient),
    "force_gauge": _runs(F.test_force_gauge_covariance),
    "pseudofermion": _runs(*[lambda m, d=d, n=n: F.test_pseudofermion_is_mdagger_chi_on_even_sites(m, d, n)
                             for d, n in (((2, 2, 2, 2), False), ((4, 2, 2, 4), True))]),
}


def _failing_pins(module):
    failed = []
    for name, run in PINS.items():
        try:
            run(module)
        except Exception:  # an assertion, or an error the broken copy raises
            failed.append(name)
    return failed


def _load_copy(tmp_path, name, text, py_text=None):
    """Build the C text with the oracle's flags and load it through a fresh
    instance of the marshalling module (``py_text``: a modified copy of it)."""
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    import oracle

    so = oracle.build(force=True, src=str(src), out=str(tmp_path / f"lib{name}.so"))
    py = PY_SRC
    if py_text is not None:
        py = str(tmp_path / f"oracle_{name}.py")
        with open(py, "w") as f:
            f.write(py_text)
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{name}", py)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build = lambda force=False, src=None, out=None: so  # load this copy, never rebuild it
    mod._SO = so
    return mod


def test_unmodified_copy_passes_every_pin(tmp_path):
    with open(SRC) as f:
        text = f.read()
    assert _failing_pins(_load_copy(tmp_path, "control", text)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    """Runs only the named pin (a broken operator sends every solve of the
    other pins to its iteration cap)."""
    old, new, count, pin = MUTANTS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == count, f"mutation site of {name} not found in the oracle source"
    mod = _load_copy(tmp_path, name, text.replace(old, new))
    with pytest.raises(Exception):
        PINS[pin](mod)


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_mistake_in_marshalling_fails_a_pin(tmp_path, name):
    old, new, count, pin = PY_MUTANTS[name]
    with open(SRC) as f:
        text = f.read()
    with open(PY_SRC) as f:
        py_text = f.read()
    assert py_text.count(old) == count, f"mutation site of {name} not found in the marshalling module"
    mod = _load_copy(tmp_path, name, text, py_text.replace(old, new))
    with pytest.raises(Exception):
        PINS[pin](mod)
