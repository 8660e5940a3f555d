"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake (a flipped sign, a wrong index, a dropped term, a non-strict
comparison, ...) in a temporary copy of the oracle's C source, builds it, and
requires at least one pin of tests/test_oracle_pins.py to fail against it.
CPU only; the committed oracle is never modified."""
import os
import subprocess

import pytest

import oracle
from oracle.build import SRC

from . import test_oracle_pins as P

ALL_K = range(7)

PIN_GROUPS = {
    "residual": [(P.test_residual_matches_dense, {"k": k}) for k in ALL_K] + [(P.test_example1_residual_exact_rational, {})],
    "sumsq": [(P.test_sumsq_tree_order_pinned, {}), (P.test_sumsq_error_bound, {"n": 4096 + 7}),
              (P.test_tau_formula_and_infinity_norm_criterion, {}), (P.test_example1_golden_trace, {})],
    "dilate": [(P.test_dilation_is_graph_ball, {"k": k, "layers": 2}) for k in ALL_K] +
              [(P.test_stored_zero_is_no_coupling, {})],
    "expand": [(P.test_example1_golden_trace, {}), (P.test_paper_expansion_brute_force_random, {}),
               (P.test_strict_thresholds_at_equality, {}), (P.test_stored_zero_is_no_coupling, {}),
               (P.test_mark_residual_alg3_brute_force, {})],
    "gradient": [(P.test_gradient_definition, {"k": k}) for k in ALL_K] + [(P.test_gradient_five_point_formula, {}),
                                                                          (P.test_mark_gradient_edges_and_monotone, {}),
                                                                          (P.test_strict_thresholds_at_equality, {}),
                                                                          (P.test_stored_zero_is_no_coupling, {}),
                                                                          (P.test_mark_gradient_layers_brute_force,
                                                                           {"layers": 2})],
    "extract": [(P.test_extract_matches_dense_blocks, {"k": k}) for k in ALL_K] + [(P.test_extract_empty_and_full, {})],
    "pcg": [(P.test_pcg_matches_dense_lu, {"k": k}) for k in ALL_K] + [(P.test_pcg_manufactured_and_warm_start, {}),
                                                                       (P.test_pcg_status_codes, {}),
                                                                       (P.test_pcg_finite_termination, {}),
                                                                       (P.test_pcg_ok_only_when_the_true_residual_meets_the_tolerance, {})],
    "alg1": [(P.test_local_then_global_agrees_with_global, {}), (P.test_local_then_global_edge_cases, {}),
             (P.test_rtilde_identity_and_bound, {}), (P.test_example1_local_solve_converges_without_global, {}),
             (P.test_local_tolerance_is_the_local_solves, {})],
    "adjoint": [(P.test_adjoint_gradient_matches_finite_differences, {})],
    "mark": [(P.test_mark_residual_rel_max_brute_force, {"k": k}) for k in ALL_K] + [
        (P.test_strict_thresholds_at_equality, {}), (P.test_rtilde_identity_and_bound, {})],
    "relres": [(P.test_relres_matches_dense_norm, {"k": k}) for k in ALL_K] + [(P.test_relres_exact_values_and_zero_rhs, {})],
    "gs": [(P.test_gs_sweep_is_lexicographic_gs_on_colour_ordered_system, {"seed": sd, "shape": sh})
           for sd, sh in P.GS_CASES] + [(P.test_gs_sweep_diagonal_and_fixed_point, {}),
                                        (P.test_gs_sweep_reduces_energy_error, {}),
                                        (P.test_local_then_global_applies_gs_to_x_tilde, {})],
    "heat": [(P.test_heat_system_symmetric_and_conservative, {}), (P.test_heat_system_exact_on_linear_steady_profile, {}),
             (P.test_heat_system_exact_across_a_material_interface, {}),
             (P.test_heat_step_steady_nonlinear_profile, {}), (P.test_heat_step_methods_agree_and_picard_fixed_point, {}),
             (P.test_picard_stops_at_the_first_update_below_the_tolerance, {}),
             (P.test_picard_iteration_is_the_papers_algorithm, {})],
}

# (name, pin group, original text, mutated text)
MUTANTS = [
    ("residual_sign", "residual", "s = fma(-av[e], x[ci[e]], s);", "s = fma(av[e], x[ci[e]], s);"),
    ("residual_drop_b", "residual", "double s = b[i];\n        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)\n            s = fma(-av[e], x[ci[e]], s);",
     "double s = 0.0;\n        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)\n            s = fma(-av[e], x[ci[e]], s);"),
    ("residual_wrong_index", "residual", "s = fma(-av[e], x[ci[e]], s);", "s = fma(-av[e], x[i], s);"),
    ("tree_drop_level", "sumsq", "for (int s = 512; s >= 1; s >>= 1)", "for (int s = 512; s > 1; s >>= 1)"),
    ("tree_sequential", "sumsq", "for (int s = 512; s >= 1; s >>= 1)\n            for (int i = 0; i < s; ++i) v[i] = v[i] + v[i + s];",
     "for (int i = 1; i < 1024; ++i) v[0] = v[0] + v[i];"),
    ("tau_no_sqrt", "sumsq", "return (eps * sqrt(S)) / sqrt((double)n);", "return (eps * S) / sqrt((double)n);"),
    ("dilate_self", "dilate", "if (ci[e] != i && av[e] != 0.0 && in[ci[e]]) m = 1;", "if (ci[e] != i && av[e] != 0.0 && in[i]) m = 1;"),
    ("dilate_one_sided", "dilate", "if (ci[e] != i && av[e] != 0.0 && in[ci[e]]) m = 1;", "if (ci[e] > i && av[e] != 0.0 && in[ci[e]]) m = 1;"),
    ("expand_wrong_x", "expand", "t = t + fabs(av[e] * x0[i]);", "t = t + fabs(av[e] * x0[j]);"),
    ("expand_drop_r", "expand", "double c = fabs(r0[j]) + t;", "double c = t;"),
    ("expand_async", "expand", "if (c > tau) { add[j] = 1; ++k0; }", "if (c > tau) { add[j] = 1; mask[j] = 1; ++k0; }"),
    ("expand_nonstrict", "expand", "if (c > tau) { add[j] = 1; ++k0; }", "if (c >= tau) { add[j] = 1; ++k0; }"),
    ("residual_nonstrict", "expand", "mask[i] = fabs(r[i]) > tau ? 1 : 0;", "mask[i] = fabs(r[i]) >= tau ? 1 : 0;"),
    ("gradient_no_abs", "gradient", "s = s + fabs(x[i] - x[j]);", "s = s + (x[i] - x[j]);"),
    ("gradient_wrong_index", "gradient", "s = s + fabs(x[i] - x[j]);", "s = s + fabs(x[i] - x[e]);"),
    ("mark_gradient_nonstrict", "gradient", "mask[i] = g[i] > thr ? 1 : 0;", "mask[i] = g[i] >= thr ? 1 : 0;"),
    ("extract_rhs_index", "extract", "else s = fma(-av[e], x0[j], s);", "else s = fma(-av[e], x0[i], s);"),
    ("extract_global_col", "extract", "bci[nz] = g2l[j];", "bci[nz] = j < K ? j : 0;"),
    ("extract_rhs_sign", "extract", "else s = fma(-av[e], x0[j], s);", "else s = fma(av[e], x0[j], s);"),
    ("relres_no_sqrt", "relres", "return sqrt(rr) / sqrt(bb);", "return rr / bb;"),
    ("relres_norm_of_x", "relres", "double rr = dot(n, r, r), bb = dot(n, b, b);", "double rr = dot(n, r, r), bb = dot(n, x, x);"),
    ("relres_drop_b", "relres", "orc_residual(n, rp, ci, av, b, x, r);\n    double rr", "orc_residual(n, rp, ci, av, b, x, r);\n    for (int32_t i = 0; i < n; ++i) r[i] -= b[i];\n    double rr"),
    ("relres_zero_rhs", "relres", "return rr == 0.0 ? 0.0 : INFINITY;", "return 0.0;"),
    ("pcg_beta_inverted", "pcg", "double beta = rz_new / rz;", "double beta = rz / rz_new;"),
    ("pcg_r_sign", "pcg", "r[i] -= alpha * q[i]; }", "r[i] += alpha * q[i]; }"),
    ("pcg_no_precond", "pcg", "dinv[i] = 1.0 / d;", "dinv[i] = 1.0 / (d * d);"),
    ("assemble_index", "alg1", "for (int32_t l = 0; l < K; ++l) xt[l2g[l]] = xbar[l];", "for (int32_t l = 0; l < K; ++l) xt[l] = xbar[l];"),
    ("alg1_skip_local", "alg1", "if (K > 0) {\n        status = orc_pcg(K,", "if (K < 0) {\n        status = orc_pcg(K,"),
    ("adjoint_wrong_k", "adjoint", "double dT = 2.0 * k[m] * k[m] / (den * den);", "double dT = 2.0 * k[c] * k[c] / (den * den);"),
    ("adjoint_drop_boundary", "adjoint", "s += 2.0 * lam[c] * x[c];", "s += 0.0 * lam[c] * x[c];"),
    ("gs_sign", "gs", "else s = fma(-av[e], x[ci[e]], s);", "else s = fma(av[e], x[ci[e]], s);"),
    ("gs_wrong_diagonal", "gs", "x[i] = s / d;", "x[i] = s / av[rp[i]];"),
    ("gs_colours_reversed", "gs", "for (int32_t c = 0; c < ncol; ++c)", "for (int32_t c = ncol - 1; c >= 0; --c)"),
    ("alg1_gs_one_sweep_short", "gs", "for (int32_t sw = 0; sw < prm->gs_sweeps; ++sw)",
     "for (int32_t sw = 1; sw < prm->gs_sweeps; ++sw)"),
    ("heat_ghost_half", "heat", "const double g = (2.0 * kp) * c;", "const double g = kp * c;"),
    ("heat_arithmetic_mean", "heat", "tf[f] = ((2.0 * kp) * kn / (kp + kn)) * c;", "tf[f] = (0.5 * (kp + kn)) * c;"),
    ("heat_drop_bc_value", "heat", "bi = bi + g * bc_val[f];", "bi = bi + 0.0 * bc_val[f];"),
    ("heat_kappa_from_Tn", "heat", "for (int32_t i = 0; i < n; ++i) kappa[i] = pow(T[i], p);",
     "for (int32_t i = 0; i < n; ++i) kappa[i] = pow(Tn[i], p);"),
    ("heat_wrong_neighbour", "heat", "const double kn = kappa[nb[f]];", "const double kn = kappa[i];"),
    ("heat_rhs_without_dt", "heat", "double d = inv_dt, bi = Tn[i] * inv_dt;", "double d = inv_dt, bi = Tn[i];"),
    ("heat_one_picard_iteration", "heat", "if (status != ORC_OK || hs->last_update < picard_tol) break;", "break;"),
    ("dilate_extra_layer", "dilate", "for (int32_t l = 0; l < layers; ++l)", "for (int32_t l = 0; l <= layers; ++l)"),
    ("expand_signed_coupling", "expand", "t = t + fabs(av[e] * x0[i]);", "t = t + av[e] * x0[i];"),
    ("rel_max_signed", "mark", "if (fabs(r[i]) > mx) mx = fabs(r[i]);", "if (r[i] > mx) mx = r[i];"),
    ("mark_gradient_absolute_threshold", "gradient", "double thr = alpha * gmax;", "double thr = alpha;"),
    ("extract_xl0_zero", "extract", "xL0[l] = x0[i];", "xL0[l] = 0.0;"),
    ("pcg_x_sign", "pcg", "x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }", "x[i] -= alpha * p[i]; r[i] -= alpha * q[i]; }"),
    ("pcg_direction_unpreconditioned", "pcg", "p[i] = z[i] + beta * p[i];", "p[i] = r[i] + beta * p[i];"),
    ("pcg_tolerance_not_squared", "pcg", "double stop = (tol * tol) * bb;", "double stop = tol * bb;"),
    ("alg1_never_early_exit", "alg1", "if (st->relres_tilde <= prm->tol) {", "if (st->relres_tilde < 0.0) {"),
    ("pcg_no_restart", "pcg", "for (int restart = 0; restart <= 3; ++restart) {",
     "for (int restart = 0; restart < 1; ++restart) {"),
    ("pcg_no_true_residual_check", "pcg", "if (dot(n, r, r) <= stop) { status = ORC_OK; break; }",
     "{ status = ORC_OK; break; }"),
    ("gradient_keeps_zero_couplings", "gradient", "if (j == i || av[e] == 0.0) continue;", "if (j == i) continue;"),
    ("dilate_keeps_zero_couplings", "dilate", "if (ci[e] != i && av[e] != 0.0 && in[ci[e]]) m = 1;",
     "if (ci[e] != i && in[ci[e]]) m = 1;"),
    ("expand_zero_coupling_neighbour", "expand", "if (av[e] != 0.0) is_nbr = 1;", "is_nbr = 1;"),
    ("alg1_local_tol_global", "alg1", "status = orc_pcg(K, brp, bci, bav, rhs, xl, prm->tol_local,",
     "status = orc_pcg(K, brp, bci, bav, rhs, xl, prm->tol,"),
    ("heat_picard_update_misreported", "heat", "hs->last_update = sqrt(d2);", "hs->last_update = sqrt(d2) / 1e3;"),
    ("expand_count_empty_rounds", "expand", "if (k0 == 0) break;", "if (k0 == 0) { }"),
    ("heat_columns_unsorted", "heat",
     "if (nb[2] >= 0) { ci[nz] = nb[2]; av[nz++] = -tf[2]; }\n            if (nb[0] >= 0) { ci[nz] = nb[0]; av[nz++] = -tf[0]; }",
     "if (nb[0] >= 0) { ci[nz] = nb[0]; av[nz++] = -tf[0]; }\n            if (nb[2] >= 0) { ci[nz] = nb[2]; av[nz++] = -tf[2]; }"),
    ("mark_gradient_one_layer_short", "gradient", "if (layers > 0) orc_dilate(n, rp, ci, av, mask, layers);",
     "if (layers > 1) orc_dilate(n, rp, ci, av, mask, layers - 1);"),
    ("alg3_tests_b_not_r0", "expand", "done = orc_expand_paper(n, rp, ci, av, r, x0, tau, mask, rounds, NULL);",
     "done = orc_expand_paper(n, rp, ci, av, b, x0, tau, mask, rounds, NULL);"),
    ("picard_solve_from_old_level", "heat", "memcpy(x, T, sizeof(double) * (size_t)n);",
     "memcpy(x, Tn, sizeof(double) * (size_t)n);"),
    ("gmax_skips_last_point", "gradient", "for (int32_t i = 0; i < n; ++i) if (g[i] > gmax) gmax = g[i];",
     "for (int32_t i = 0; i + 1 < n; ++i) if (g[i] > gmax) gmax = g[i];"),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = src.replace(old, new, 1)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(mut)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(cpath), "-lm"],
                   check=True, capture_output=True)
    return str(so)


@pytest.mark.parametrize("name,group,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, group, old, new):
    so = _build_mutant(tmp_path, name, old, new)
    saved = oracle._lib
    oracle._lib = oracle.load(so)
    caught = []
    try:
        for fn, kw in PIN_GROUPS[group]:
            try:
                fn(**kw)
            except (AssertionError, ValueError, FloatingPointError, IndexError, ZeroDivisionError, np_linalg_error()):
                caught.append(fn.__name__)
                break
    finally:
        oracle._lib = saved
    assert caught, f"no pin in group {group!r} caught mutant {name!r}"


def np_linalg_error():
    import numpy as np
    return np.linalg.LinAlgError
