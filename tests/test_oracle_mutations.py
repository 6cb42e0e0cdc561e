"""Do the oracle's pins catch plausible mistakes?

Each case below plants ONE mistake in a copy of an oracle function (a
dropped term, a flipped sign, a transposed operand, an off-by-one index, a
wrong constant), swaps the copy in with monkeypatch for the duration of the
case, and runs the pin tests named beside it (cheapest first).  At least one
of them must fail; a mistake that every named pin lets through is a gap in
the pins.  Mistakes are planted on the CPU, in the oracle only; nothing here
touches the CUDA path.

A mutant is written as (module, function, original text, mutated text); the
original text must occur exactly once in the function's source, so a later
edit of the oracle that removes it fails the case loudly instead of silently
testing nothing.
"""

import __future__
import importlib
import inspect
import textwrap

import numpy as np
import pytest

from oracle import correction, ipm, mlp, pcg, phase1, sketch, vertex

MODULES = {"sketch": sketch, "pcg": pcg, "correction": correction, "ipm": ipm,
           "phase1": phase1, "mlp": mlp, "vertex": vertex}


def _pin(test_module, name, **kwargs):
    mod = importlib.import_module("tests." + test_module)
    fn = getattr(mod, name)
    label = name + ("[" + ",".join(f"{k}={v}" for k, v in kwargs.items()) + "]" if kwargs else "")
    return label, (lambda: fn(**kwargs))


# pins by short name (test module, test function, parameters)
PINS = {
    # oracle.sketch
    "splitmix_golden": ("test_oracle_sketch", "test_splitmix64_reference_outputs", {}),
    "counter_draw": ("test_oracle_sketch", "test_counter_draw_equals_stream_position", {}),
    "cs_redraw": ("test_oracle_sketch", "test_countsketch_redraw_changes_hash", {}),
    "cs_blocks": ("test_oracle_sketch", "test_countsketch_blocks_hash_independently", {}),
    "cs_structure": ("test_oracle_sketch", "test_countsketch_structure", {"w": 128, "s": 4}),
    "cs_gram": ("test_oracle_sketch", "test_sparse_embedding_approximates_gram", {}),
    "gauss_moments": ("test_oracle_sketch", "test_gaussian_sketch_moments", {}),
    "gauss_uniforms": ("test_oracle_sketch", "test_gaussian_uniforms_are_exact_fp32_and_in_range", {}),
    "gauss_grid_ends": ("test_oracle_sketch", "test_gaussian_uniforms_reach_both_ends_of_their_grids", {}),
    "gauss_embedding": ("test_oracle_sketch", "test_gaussian_sketch_subspace_embedding", {}),
    "gauss_pairs": ("test_oracle_sketch", "test_gaussian_sketch_uses_both_box_muller_outputs", {}),
    # oracle.pcg
    "cg_krylov": ("test_oracle_pcg", "test_cg_iterates_minimise_energy_error_over_krylov_space", {}),
    "cg_exact": ("test_oracle_pcg", "test_cg_reaches_exact_solution", {}),
    "cheb_poly": ("test_oracle_pcg", "test_chebyshev_residual_is_scaled_chebyshev_polynomial", {}),
    "cheb_bound_values": ("test_oracle_pcg", "test_chebyshev_bound_closed_form_values", {}),
    "cheb_bound_cs": ("test_oracle_pcg", "test_chebyshev_bound_eq_cs", {"kappa": 10.0}),
    "whiten": ("test_oracle_pcg", "test_preconditioner_whitens_q", {}),
    "identity_sketch": ("test_oracle_pcg", "test_identity_sketch_makes_cg_one_step", {}),
    "contraction": ("test_oracle_pcg", "test_cg_residual_monotone_with_contraction_eq_rec", {}),
    "contraction_band": ("test_oracle_pcg", "test_contraction_is_lemma_3_2_rate_at_the_lemma_3_1_band_edges",
                         {"zeta": 0.5}),
    "theory_tol": ("test_oracle_pcg", "test_theory_tolerance_and_iteration_count", {}),
    "lanczos": ("test_oracle_pcg", "test_lanczos_interval_recovers_the_spectrum", {}),
    # oracle.ipm / oracle.correction
    "planted_exact": ("test_oracle_ipm", "test_planted_optimum_reached", {"solver": "exact", "seed": 0}),
    "planted_sketch": ("test_oracle_ipm", "test_planted_optimum_reached", {"solver": "sketch", "seed": 0}),
    "feasible_planted": ("test_oracle_ipm", "test_feasible_mode_planted", {}),
    "vertices": ("test_oracle_ipm", "test_vertex_enumeration_and_highs_agree_with_oracle", {"seed": 0}),
    "planted_tiny_vertices": ("test_oracle_ipm", "test_planted_tiny_matches_vertex_enumeration", {}),
    "planted_sparse": ("test_oracle_ipm", "test_sparse_input_reaches_the_planted_optimum", {"seed": 0}),
    "vertices_sparse": ("test_oracle_ipm", "test_sparse_input_matches_vertex_enumeration", {"seed": 0}),
    "lemma45_feas": ("test_oracle_ipm", "test_lemma_4_5_identities", {"mode": "feasible"}),
    "lemma45_infeas": ("test_oracle_ipm", "test_lemma_4_5_identities", {"mode": "infeasible"}),
    "feasible_stays": ("test_oracle_ipm", "test_feasible_iterates_stay_feasible_and_in_neighbourhood", {}),
    "residual_linear": ("test_oracle_ipm", "test_infeasible_residual_shrinks_linearly", {}),
    "v_invariant": ("test_oracle_ipm", "test_correction_invariant_and_norm_bound", {}),
    "v_identity": ("test_oracle_ipm", "test_correction_with_identity_sketch_and_minnorm_alternative", {}),
    "first_exit": ("test_oracle_ipm", "test_first_exit_hand_built_quadratics", {}),
    "grid_feas": ("test_oracle_ipm", "test_step_length_against_grid", {"mode": "feasible", "sigma": 0.5}),
    "grid_infeas": ("test_oracle_ipm", "test_step_length_against_grid", {"mode": "infeasible", "sigma": 0.5}),
    "grid_infeas_binding": ("test_oracle_ipm", "test_step_length_against_grid",
                            {"mode": "infeasible", "sigma": 0.3}),
    "steps_feas": ("test_oracle_ipm", "test_step_lengths_on_random_states_against_grid", {"feasible": True}),
    "steps_infeas": ("test_oracle_ipm", "test_step_lengths_on_random_states_against_grid", {"feasible": False}),
    "start_central": ("test_oracle_ipm", "test_feasible_start_is_strictly_feasible_and_central_enough", {}),
    "ns_cholesky": ("test_oracle_ipm", "test_normal_solve_matches_cholesky_at_tight_tolerance", {}),
    "ns_plain": ("test_oracle_ipm", "test_unpreconditioned_normal_solve_is_cg_on_eq_normal", {}),
    "two_rhs": ("test_oracle_ipm", "test_two_rhs_combination_is_the_solve_with_p_sigma", {}),
    "two_rhs_fewer_outer": ("test_oracle_ipm", "test_two_rhs_adaptive_sigma_needs_fewer_outer_iterations",
                            {"col_scale": None}),
    "inner_theory_bound": ("test_oracle_ipm", "test_inner_solves_stop_at_the_theory_bound", {}),
    "orthonormal_rows": ("test_oracle_ipm",
                         "test_orthonormal_rows_and_unit_scaling_give_the_identity_normal_matrix", {}),
    "v_identity_lstsq": ("test_oracle_ipm", "test_identity_sketch_correction_is_the_min_norm_solution_of_ad", {}),
    # oracle.phase1
    "p1_planted": ("test_oracle_phase1", "test_planted_lp_gets_a_strictly_feasible_start", {}),
    "p1_negative_b": ("test_oracle_phase1", "test_negative_right_hand_sides_are_handled", {}),
    "p1_highs": ("test_oracle_phase1", "test_random_lp_family_matches_highs_phase1_optimum", {}),
    "p1_infeasible": ("test_oracle_phase1", "test_constructed_infeasible_lp_is_detected", {}),
    "p1_projection": ("test_oracle_phase1", "test_start_is_projected_onto_a_x_equals_b", {}),
    # oracle.mlp
    "mlp_fd": ("test_oracle_mlp", "test_gradients_match_finite_differences", {}),
    "mlp_layout": ("test_oracle_mlp", "test_flatten_is_the_inverse_of_unflatten_and_column_major", {}),
    "mlp_gelu": ("test_oracle_mlp", "test_gelu_special_values", {}),
    "mlp_adam": ("test_oracle_mlp", "test_adam_first_step_moves_each_weight_by_lr_against_the_gradient_sign", {}),
}

# (id, module, function, original text, mutated text, pins to run, cheapest first)
MUTANTS = [
    # --- the generator and the sketches (Section 2, Section 6) ---
    ("mix64_shift", "sketch", "mix64", "(z >> _U64(30))", "(z >> _U64(29))", ["splitmix_golden"]),
    ("mix64_multiplier", "sketch", "mix64", "0x94D049BB133111EB", "0x94D049BB133111EF", ["splitmix_golden"]),
    ("draw_off_by_one", "sketch", "draw", "(ctr + _U64(1))", "ctr", ["counter_draw"]),
    ("stream_off_by_one", "sketch", "splitmix64_stream", "np.arange(1, count + 1", "np.arange(0, count",
     ["splitmix_golden"]),
    ("counter_block_dropped", "sketch", "countsketch_counter", "* MAX_BLOCKS + block)", "* MAX_BLOCKS)",
     ["cs_blocks"]),
    ("counter_retry_dropped", "sketch", "countsketch_counter", "(k * MAX_RETRY + retry)", "(k * MAX_RETRY)",
     ["cs_redraw"]),
    ("counter_outer_dropped", "sketch", "countsketch_counter", "(k * MAX_RETRY + retry)", "(retry)",
     ["cs_redraw"]),
    ("cg_coeffs_beta_inverted", "ipm", "_cg_coeffs", "beta = rr_new / rr", "beta = rr / rr_new", ["lanczos"]),
    ("flatten_row_major", "mlp", "flatten", "p.T.reshape(-1)", "p.reshape(-1)", ["mlp_layout"]),
    ("vertex_feasibility_sign", "vertex", "enumerate_vertices", "(xB < -feas_tol).any()",
     "(xB > feas_tol).any()", ["planted_tiny_vertices", "vertices"]),
    ("cs_block_offset_dropped", "sketch", "countsketch_hash",
     "cols[b] = b * wb + h.astype(np.int64)", "cols[b] = h.astype(np.int64)", ["cs_structure"]),
    ("cs_scale_dropped", "sketch", "countsketch_matrix", "(signs / np.sqrt(s))", "signs",
     ["cs_structure", "cs_gram"]),
    ("gauss_scale_dropped", "sketch", "gaussian_matrix", "(z / np.sqrt(w))", "z",
     ["gauss_moments", "gauss_embedding"]),
    ("box_muller_factor", "sketch", "gaussian_matrix", "np.sqrt(-2.0 * np.log(u1))",
     "np.sqrt(-np.log(u1))", ["gauss_moments", "gauss_embedding"]),
    ("uniform_u1_open_at_zero", "sketch", "gaussian_uniforms", "+ 1.0) / 8388608.0", ") / 8388608.0",
     ["gauss_uniforms", "gauss_grid_ends"]),
    ("box_muller_one_output", "sketch", "gaussian_matrix", "r * np.sin(ang)", "r * np.cos(ang)",
     ["gauss_pairs"]),
    ("box_muller_pair_index", "sketch", "gaussian_matrix", "[f // 2]\n    ang", "[f % ((n * w + 1) // 2)]\n    ang",
     ["gauss_pairs"]),
    # --- Algorithm 1 (Section 3) ---
    ("precond_q_plus_half", "pcg", "preconditioner", "(U / sv) @ U.T", "(U * sv) @ U.T", ["whiten"]),
    ("precond_transpose_dropped", "pcg", "preconditioner", "(U / sv) @ U.T", "(U / sv) @ U", ["whiten"]),
    ("precond_sv_squared", "pcg", "preconditioner", "(U / sv) @ U.T", "(U / sv ** 2) @ U.T", ["whiten"]),
    ("cg_beta_inverted", "pcg", "cg", "(rr_new / rr)", "(rr / rr_new)", ["cg_krylov", "cg_exact"]),
    ("cg_alpha_denominator", "pcg", "cg", "rr / (d @ Bd)", "rr / (d @ d)", ["cg_krylov", "cg_exact"]),
    ("cg_residual_sign", "pcg", "cg", "r = r - a * Bd", "r = r + a * Bd", ["cg_krylov", "cg_exact"]),
    ("cheb_rho_sign", "pcg", "chebyshev", "1.0 / (2.0 * s1 - rho)", "1.0 / (2.0 * s1 + rho)", ["cheb_poly"]),
    ("cheb_first_step", "pcg", "chebyshev", "d = r / theta", "d = r / delta", ["cheb_poly"]),
    ("cheb_direction_factor", "pcg", "chebyshev", "(2.0 * rho_new / delta)", "(rho_new / delta)",
     ["cheb_poly"]),
    ("cheb_bound_sign", "pcg", "chebyshev_bound", "q ** t + q ** (-t)", "q ** t - q ** (-t)",
     ["cheb_bound_values", "cheb_bound_cs"]),
    ("cheb_bound_sqrt_dropped", "pcg", "chebyshev_bound", "(np.sqrt(U) + 1.0) / (np.sqrt(U) - 1.0)",
     "(U + 1.0) / (U - 1.0)", ["cheb_bound_values", "cheb_bound_cs"]),
    ("contraction_sign", "pcg", "cg_contraction", "(2.0 - zeta)", "(2.0 + zeta)",
     ["contraction", "contraction_band"]),
    ("theory_tol_factor_3", "pcg", "theory_inner_tol", "np.sqrt(3.0 * n)", "np.sqrt(n)", ["theory_tol"]),
    ("iteration_count_floor", "pcg", "inner_iteration_count", "np.ceil(", "np.floor(", ["theory_tol"]),
    ("lanczos_diag_index", "ipm", "lanczos_interval", "betas[j - 1] / alphas[j - 1]",
     "betas[j - 1] / alphas[j]", ["lanczos", "ns_cholesky"]),
    ("lanczos_offdiag_sqrt", "ipm", "lanczos_interval", "np.sqrt(betas[j]) / alphas[j]",
     "betas[j] / alphas[j]", ["lanczos", "ns_cholesky"]),
    # --- the correction vector (Section 4, eq. compv) ---
    ("v_scale_inverted", "correction", "correction_v", "np.sqrt(x * s)", "np.sqrt(x / s)",
     ["v_identity", "v_invariant"]),
    ("v_sign", "correction", "correction_v", "np.linalg.pinv(ADW) @ r_v", "np.linalg.pinv(ADW) @ (-r_v)",
     ["v_identity", "v_invariant"]),
    ("v_q_inverse_dropped", "correction", "correction_v", "np.linalg.pinv(ADW) @ r_v",
     "ADW.T @ r_v", ["v_identity_lstsq", "v_invariant"]),
    ("v_minnorm_scale", "correction", "correction_v_minnorm", "(A / s)", "(A * s)", ["v_identity"]),
    # --- residuals, right-hand side, directions (Sections 4-5) ---
    ("dual_residual_sign", "ipm", "residuals", "A.T @ y + s - c", "A.T @ y - s - c",
     ["planted_exact", "vertices"]),
    ("rhs_infeasible_term_dropped", "ipm", "rhs", "p = p - r_p - A @ (d2 * r_d)", "p = p - r_p",
     ["residual_linear", "planted_exact"]),
    ("rhs_primal_residual_dropped", "ipm", "rhs", "p = p - r_p - A @ (d2 * r_d)",
     "p = p - A @ (d2 * r_d)", ["residual_linear", "planted_exact"]),
    ("rhs_centering_sign", "ipm", "rhs", "p = -sigma * mu", "p = sigma * mu",
     ["lemma45_feas", "feasible_planted"]),
    ("normal_matrix_d_not_d2", "ipm", "normal_matrix", "(A * d2) @ A.T", "(A * np.sqrt(d2)) @ A.T",
     ["planted_exact", "vertices"]),
    ("normal_matrix_sparse_d_not_d2", "ipm", "normal_matrix", "A @ sps.diags(d2) @ A.T",
     "A @ sps.diags(np.sqrt(d2)) @ A.T", ["planted_sparse", "vertices_sparse"]),
    ("normal_matrix_sparse_weights_reversed", "ipm", "normal_matrix", "A @ sps.diags(d2) @ A.T",
     "A @ sps.diags(d2[::-1]) @ A.T", ["planted_sparse", "vertices_sparse"]),
    ("direction_v_dropped", "ipm", "directions", " - v / s", "", ["lemma45_feas", "lemma45_infeas"]),
    ("direction_d2_inverted", "ipm", "directions", "(x / s) * ds", "(s / x) * ds",
     ["lemma45_feas", "lemma45_infeas"]),
    ("direction_dual_residual_sign", "ipm", "directions", "ds = ds - r_d", "ds = ds + r_d",
     ["residual_linear", "planted_exact"]),
    # --- step lengths (Alg. 2 steps 5-6, Alg. 3 steps 6-7) ---
    ("first_exit_wrong_root", "ipm", "_first_exit", "out[sel] = hi[sel]", "out[sel] = lo[sel]",
     ["first_exit"]),
    ("first_exit_linear_sign", "ipm", "_first_exit", "np.maximum(-c[lb] / b[lb], 0.0)",
     "np.maximum(c[lb] / b[lb], 0.0)", ["first_exit"]),
    ("neighbourhood_gamma_swapped", "ipm", "step_lengths", "g = 1.0 - gamma", "g = gamma",
     ["steps_feas", "grid_feas"]),
    ("alpha_bar_factor_2", "ipm", "step_lengths", "-c1 / (2.0 * c2)", "-c1 / c2", ["steps_feas"]),
    ("mu_quadratic_term_dropped", "ipm", "step_lengths", "c2 = (dx @ ds) / n", "c2 = 0.0 * n",
     ["steps_feas", "steps_infeas"]),
    ("infeasible_bound_sign", "ipm", "step_lengths", "c1 / mu0 + res_ratio", "c1 / mu0 - res_ratio",
     ["steps_infeas"]),
    ("neighbourhood_test_gamma", "ipm", "in_neighbourhood", "(1.0 - gamma) * mu", "gamma * mu",
     ["start_central"]),
    # --- one normal solve (Algorithm 1 + eq. compv) and the outer loop ---
    ("ns_back_transform_dropped", "ipm", "normal_solve", "dy = Qmh @ z", "dy = z", ["ns_cholesky"]),
    ("ns_rhs_unpreconditioned", "ipm", "normal_solve", "rhs_ = Qmh @ p", "rhs_ = p", ["ns_cholesky"]),
    ("ns_sketch_of_d2", "ipm", "normal_solve", "d = np.sqrt(x / s)", "d = x / s", ["v_invariant"]),
    ("ns_correction_residual_sign", "ipm", "normal_solve", "r_v = A @ (d2 * (A.T @ dy)) - p",
     "r_v = p - A @ (d2 * (A.T @ dy))", ["v_invariant"]),
    ("ns_chebyshev_interval_too_small", "ipm", "normal_solve", "1.05 * tmax", "0.5 * tmax",
     ["ns_cholesky"]),
    ("ns_inner_target_loosened", "ipm", "normal_solve", 'tol = inner_tol if opt.inner_rule == "theory"',
     'tol = 10 * inner_tol if opt.inner_rule == "theory"', ["inner_theory_bound"]),
    ("plain_cg_d2_inverted", "ipm", "normal_solve_unpreconditioned", "d2 = x / s", "d2 = s / x",
     ["ns_plain"]),
    ("adaptive_sigma_ratio_inverted", "ipm", "_adaptive_sigma_solve", "(mu_aff / mu) ** 3",
     "(mu / mu_aff) ** 3", ["two_rhs_fewer_outer"]),
    ("neighbourhood_residual_ratio_inverted", "ipm", "in_neighbourhood", "res_ratio > (mu / mu0)",
     "res_ratio > (mu0 / mu)", ["grid_infeas_binding", "steps_infeas"]),
    ("two_rhs_affine_part_kept", "ipm", "_adaptive_sigma_solve",
     "rhs(A, x, s, r_p, r_d, 1.0, mu, feasible) - p_aff", "rhs(A, x, s, r_p, r_d, 1.0, mu, feasible)",
     ["two_rhs"]),
    ("gap_sign", "ipm", "converged", "abs(cx - b @ y)", "abs(cx + b @ y)", ["planted_exact"]),
    ("dual_step_sign", "ipm", "solve", "y = y + a_bar * dy", "y = y - a_bar * dy", ["planted_exact"]),
    ("residual_ratio_unnormalised", "ipm", "solve", "np.sqrt(r_p @ r_p + r_d @ r_d) / r0_norm",
     "np.sqrt(r_p @ r_p + r_d @ r_d)", ["grid_infeas_binding"]),
    # --- phase 1 (Appendix, feasible starting point) ---
    ("p1_b_not_flipped", "phase1", "phase1_lp", "b1 = b * sign", "b1 = b", ["p1_negative_b"]),
    ("p1_costs_swapped", "phase1", "phase1_lp", "[np.zeros(n), np.ones(m)]", "[np.ones(n), np.zeros(m)]",
     ["p1_highs", "p1_infeasible"]),
    ("p1_feasibility_test_inverted", "phase1", "phase1_start", "feasible = z_sum <=", "feasible = z_sum >=",
     ["p1_planted"]),
    ("p1_projection_sign", "phase1", "phase1_start", "x0 = x + A.T", "x0 = x - A.T",
     ["p1_planted", "p1_projection"]),
    # --- the warm-start model ---
    ("gelu_scale", "mlp", "gelu", "z / math.sqrt(2.0)", "z / 2.0", ["mlp_gelu", "mlp_fd"]),
    ("gelu_grad_term_dropped", "mlp", "gelu_grad",
     " + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)", "", ["mlp_fd"]),
    ("loss_batch_mean_dropped", "mlp", "loss_and_grads", "d3 = R / B", "d3 = R", ["mlp_fd"]),
    ("backprop_transpose_dropped", "mlp", "loss_and_grads", "(W2.T @ d2)", "(W2 @ d2)", ["mlp_fd"]),
    ("forward_activation_dropped", "mlp", "forward", "A2 = gelu(Z2)", "A2 = Z2", ["mlp_fd"]),
    ("adam_second_moment_unsquared", "mlp", "adam_step", "(1 - b2) * grad * grad", "(1 - b2) * grad",
     ["mlp_adam"]),
    ("adam_bias_correction_dropped", "mlp", "adam_step", "mh = m / (1 - b1 ** step)", "mh = m",
     ["mlp_adam"]),
    ("unflatten_row_major", "mlp", "unflatten", ".reshape(cols, rows).T", ".reshape(rows, cols)",
     ["mlp_layout"]),
]

# pin failures that count as catching a mistake; anything else (a TypeError,
# a NameError) is an error of this harness and propagates
CAUGHT = (AssertionError, np.linalg.LinAlgError)


def _mutant(module, func_name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(module, func_name)))
    assert src.count(old) == 1, f"{module.__name__}.{func_name}: {old!r} occurs {src.count(old)} times"
    code = compile(src.replace(old, new), f"<mutant of {module.__name__}.{func_name}>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    scope = {}
    exec(code, module.__dict__, scope)
    return scope[func_name]


def test_every_mutated_function_exists_and_every_pin_is_known():
    for mid, mod, fn, old, new, pins in MUTANTS:
        assert hasattr(MODULES[mod], fn), mid
        assert old != new, mid
        for p in pins:
            assert p in PINS, (mid, p)
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


@pytest.mark.parametrize("mid,mod,fn,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, mid, mod, fn, old, new, pins):
    module = MODULES[mod]
    monkeypatch.setattr(module, fn, _mutant(module, fn, old, new))
    ran = []
    for p in pins:
        label, run = _pin(PINS[p][0], PINS[p][1], **PINS[p][2])
        with np.errstate(all="ignore"):
            try:
                run()
            except CAUGHT:
                return
        ran.append(label)
    pytest.fail(f"mistake {mid!r} in {mod}.{fn} passed every pin: {ran}")


# Control: rewrites that change nothing (operands of a dot product swapped,
# the terms of a sum reordered) must pass every pin they are run against, so
# a caught mistake is the mistake and not the act of recompiling the function.
EQUIVALENT = [
    ("cg_dot_swapped", "pcg", "cg", "rr / (d @ Bd)", "rr / (Bd @ d)", ["cg_krylov", "cg_exact"]),
    ("rhs_terms_reordered", "ipm", "rhs", "p = -sigma * mu * (A @ (1.0 / s)) + A @ x",
     "p = A @ x - sigma * mu * (A @ (1.0 / s))", ["residual_linear", "lemma45_feas", "planted_exact"]),
    ("mu_dot_swapped", "ipm", "step_lengths", "c2 = (dx @ ds) / n", "c2 = (ds @ dx) / n",
     ["steps_feas", "steps_infeas"]),
    # the pseudo-inverse as the CUDA path forms it, (ADW)^+ = (ADW)^T Q^{-1}
    ("pinv_as_adw_t_q_inverse", "correction", "correction_v", "np.linalg.pinv(ADW) @ r_v",
     "ADW.T @ np.linalg.solve(ADW @ ADW.T, r_v)", ["v_identity", "v_identity_lstsq", "v_invariant"]),
]


@pytest.mark.parametrize("mid,mod,fn,old,new,pins", EQUIVALENT, ids=[m[0] for m in EQUIVALENT])
def test_equivalent_rewrite_passes_every_pin(monkeypatch, mid, mod, fn, old, new, pins):
    module = MODULES[mod]
    monkeypatch.setattr(module, fn, _mutant(module, fn, old, new))
    for p in pins:
        _, run = _pin(PINS[p][0], PINS[p][1], **PINS[p][2])
        run()
