"""Planted mistakes in the oracle are caught by its pins (no GPU).

Each mutant below is one plausible slip in the oracle: a transposed
operand, a wrong index, a dropped term, a flipped sign, swapped scalars, a
wrong rounding rule.  It is made in a copy of the oracle's source, which is
compiled (C) or executed (Python) on the side and put in place of the real
oracle while pins from test_oracle.py run.  At least one pin must reject it.
The oracle's own source is never changed.

Each mutant lists only pins whose inputs keep its reads in bounds: a mutant
that swaps a row index with a column index runs on square matrices only.
"""

import importlib.util
import os
import types

import pytest

import oracle
import oracle.mlp
import oracle.script

HERE = os.path.dirname(os.path.abspath(__file__))


def _load_pins():
    spec = importlib.util.spec_from_file_location("oracle_pins", os.path.join(HERE, "test_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = _load_pins()
BF16, E4M3 = oracle.FMT_BF16, oracle.FMT_E4M3


def P(name, *args):
    return (name, args)


# (id, scope, old, new, pins).  The edit replaces ``old`` by ``new`` inside the
# function whose definition starts with ``scope``; ``old`` must occur there once.
C_MUTANTS = [
    ("gemv_reads_A_transposed", "void kfo_gemv(",
     "acc += A[i * lda + j] * x[j];", "acc += A[j * lda + i] * x[j];",
     [P("test_bicgk_one_hot_pins_index_mapping", 4, 4), P("test_atax_permutation_and_hadamard")]),
    ("gemvt_takes_y_at_the_column_index", "void kfo_gemvt(",
     "acc += A[i * lda + j] * y[i];", "acc += A[i * lda + j] * y[j];",
     [P("test_bicgk_one_hot_pins_index_mapping", 4, 4), P("test_gemver_rank_one_closed_form")]),
    ("gemvt_drops_the_accumulator", "void kfo_gemvt(",
     "x[j] = alpha * acc + (beta != 0.0 ? beta * x0[j] : 0.0);", "x[j] = alpha * acc;",
     [P("test_gemver_rank_one_closed_form"), P("test_gemver_invariant"), P("test_hand_worked_examples")]),
    ("gemvt_alpha_and_beta_swapped", "void kfo_gemvt(",
     "x[j] = alpha * acc + (beta != 0.0 ? beta * x0[j] : 0.0);",
     "x[j] = beta * acc + (alpha != 0.0 ? alpha * x0[j] : 0.0);",
     [P("test_gemv_gemvt_scalars_and_accumulators")]),
    ("gemv_drops_the_accumulator", "void kfo_gemv(",
     "y[i] = alpha * acc + (beta != 0.0 ? beta * y0[i] : 0.0);", "y[i] = alpha * acc;",
     [P("test_gemv_gemvt_scalars_and_accumulators"), P("test_script_elementary_ops")]),
    ("ger_ignores_alpha", "void kfo_ger(",
     "A[i * lda + j] + alpha * u[i] * v[j]", "A[i * lda + j] + u[i] * v[j]",
     [P("test_ger_one_hot_and_alpha"), P("test_script_elementary_ops")]),
    ("ger_outer_product_transposed", "void kfo_ger(",
     "alpha * u[i] * v[j]", "alpha * u[j] * v[i]",
     [P("test_script_elementary_ops")]),
    ("madd_subtracts", "void kfo_madd(",
     "C[i] = A[i] + B[i];", "C[i] = A[i] - B[i];",
     [P("test_madd_vadd_dot_special_cases")]),
    ("vadd_drops_the_third_vector", "void kfo_vadd3(",
     "out[i] = w[i] + y[i] + z[i];", "out[i] = w[i] + y[i];",
     [P("test_madd_vadd_dot_special_cases"), P("test_script_elementary_ops")]),
    ("axpby_drops_the_y_term", "void kfo_axpby(",
     "(beta != 0.0 ? beta * y[i] : 0.0)", "0.0",
     [P("test_waxpby_cases"), P("test_axpydot_cases")]),
    ("dot_skips_the_first_term", "double kfo_dot(",
     "for (int64_t i = 0; i < n; ++i) acc += x[i] * y[i];",
     "for (int64_t i = 1; i < n; ++i) acc += x[i] * y[i];",
     [P("test_axpydot_cases"), P("test_madd_vadd_dot_special_cases")]),
    ("bicgk_s_from_p", "void kfo_bicgk(",
     "kfo_gemvt(m, n, A, lda, r, 1.0, 0.0, 0, s);", "kfo_gemvt(m, n, A, lda, p, 1.0, 0.0, 0, s);",
     [P("test_bicgk_one_hot_pins_index_mapping", 4, 4), P("test_bicgk_rank_one_closed_form", 64, 64)]),
    ("gemver_drops_the_second_update", "void kfo_gemver(",
     " + u2[i] * v2[j];", ";",
     [P("test_gemver_one_hot_updates_pin_indices"), P("test_hand_worked_examples")]),
    ("gemver_update_indices_swapped", "void kfo_gemver(",
     "u1[i] * v1[j]", "u1[j] * v1[i]",
     [P("test_gemver_one_hot_updates_pin_indices"), P("test_gemver_rank_one_closed_form")]),
    ("gemver_w_from_z", "void kfo_gemver(",
     "kfo_gemv(n, n, B, n, x, alpha, 0.0, 0, w);", "kfo_gemv(n, n, B, n, z, alpha, 0.0, 0, w);",
     [P("test_gemver_rank_one_closed_form"), P("test_gemver_invariant")]),
    ("gemver_x_scaled_by_alpha", "void kfo_gemver(",
     "kfo_gemvt(n, n, B, n, y, beta, 1.0, z, x);", "kfo_gemvt(n, n, B, n, y, alpha, 1.0, z, x);",
     [P("test_gemver_rank_one_closed_form"), P("test_gemver_invariant")]),
    ("gemver_x_from_A_not_B", "void kfo_gemver(",
     "kfo_gemvt(n, n, B, n, y, beta, 1.0, z, x);", "kfo_gemvt(n, n, A, lda, y, beta, 1.0, z, x);",
     [P("test_gemver_rank_one_closed_form"), P("test_gemver_one_hot_updates_pin_indices")]),
    ("gesummv_alpha_and_beta_swapped", "void kfo_gesummv(",
     "y[i] = alpha * a + beta * b;", "y[i] = beta * a + alpha * b;",
     [P("test_gesummv_special_cases")]),
    ("gesummv_reads_A_twice", "void kfo_gesummv(",
     "b += B[i * lda + j] * x[j];", "b += A[i * lda + j] * x[j];",
     [P("test_gesummv_special_cases")]),
    ("atax_second_product_not_transposed", "void kfo_atax(",
     "kfo_gemvt(m, n, A, lda, t, 1.0, 0.0, 0, y);", "kfo_gemv(m, n, A, lda, t, 1.0, 0.0, 0, y);",
     [P("test_atax_permutation_and_hadamard")]),
    ("axpydot_adds_alpha_v", "double kfo_axpydot(",
     "kfo_axpby(n, 1.0, w, -alpha, v, z);", "kfo_axpby(n, 1.0, w, alpha, v, z);",
     [P("test_axpydot_cases")]),
    ("waxpby_alpha_and_beta_swapped", "void kfo_waxpby(",
     "kfo_axpby(n, alpha, x, beta, y, w);", "kfo_axpby(n, beta, x, alpha, y, w);",
     [P("test_waxpby_cases")]),
    ("bf16_truncates", "static uint16_t f32_to_bf16_rne(",
     "u += 0x7FFFu + lsb;", "u += 0u * lsb;",
     [P("test_bf16_codes_match_round_to_nearest_even"), P("test_hand_worked_quantisation")]),
    ("bf16_ties_away_from_zero", "static uint16_t f32_to_bf16_rne(",
     "u += 0x7FFFu + lsb;", "u += 0x8000u + 0u * lsb;",
     [P("test_bf16_codes_match_round_to_nearest_even")]),
    ("e4m3_decodes_with_bias_8", "static double e4m3_to_double(",
     "ebits - 7", "ebits - 8",
     [P("test_e4m3_format_definition"), P("test_quantize_exact_rows_are_lossless", E4M3)]),
    ("e4m3_saturates_to_nan", "static uint8_t f32_to_e4m3_rne_sat(",
     "if (x >= 448.0) return (uint8_t)(sign | 0x7E);", "if (x >= 448.0) return (uint8_t)(sign | 0x7F);",
     [P("test_e4m3_format_definition")]),
    ("e4m3_subnormal_quantum_halved", "static uint8_t f32_to_e4m3_rne_sat(",
     "double k = rint(x / ldexp(1.0, -9));", "double k = rint(x / ldexp(1.0, -10));",
     [P("test_e4m3_format_definition")]),
    ("e4m3_ties_away_from_zero", "static uint8_t f32_to_e4m3_rne_sat(",
     "double q = rint(x / quantum) * quantum;", "double q = round(x / quantum) * quantum;",
     [P("test_e4m3_format_definition"), P("test_e4m3_matches_torch_in_range")]),
    ("row_scale_ignores_qmax", "void kfo_quantize_rows(",
     "const float qmax = (fmt == 2) ? 448.0f : 1.0f;", "const float qmax = 1.0f;",
     [P("test_quantize_error_bound", E4M3, 2 ** -4), P("test_quantize_exact_rows_are_lossless", E4M3),
      P("test_hand_worked_quantisation")]),
    ("row_scale_from_the_first_element", "void kfo_quantize_rows(",
     "if (a > amax) amax = a;", "if (j == 0) amax = a;",
     [P("test_quantize_error_bound", BF16, 2 ** -8), P("test_quantize_error_bound", E4M3, 2 ** -4),
      P("test_hand_worked_quantisation")]),
    ("dequantize_with_row_0_scale", "void kfo_dequantize_rows(",
     "Ahat[i * n + j] = (double)scale[i] * q;", "Ahat[i * n + j] = (double)scale[0] * q;",
     [P("test_quantize_error_bound", BF16, 2 ** -8), P("test_quantize_error_bound", E4M3, 2 ** -4)]),
    ("stored_gemver_bound_drops_u2", "void kfo_gemver_rowscaled_store(",
     "bound = bound + fabsf(u2[i]) * n2;", "bound = bound + 0.0f * n2;",
     [P("test_gemver_rowscaled_storage_bound", BF16, 2.0 ** -8, 2.0 ** -126, 64.0),
      P("test_gemver_rowscaled_storage_bound", E4M3, 2.0 ** -4, 2.0 ** -6, 64.0),
      P("test_hand_worked_rowscaled_gemver_storage"),
      P("test_gemver_rowscaled_cost_against_the_amax_rule", BF16),
      P("test_gemver_rowscaled_cost_against_the_amax_rule", E4M3)]),
    ("stored_gemver_updates_mixed", "void kfo_gemver_rowscaled_store(",
     "fmaf(u2[i], v2[j], fmaf(u1[i], v1[j], a))", "fmaf(u1[i], v2[j], fmaf(u2[i], v1[j], a))",
     [P("test_gemver_rowscaled_storage_bound", BF16, 2.0 ** -8, 2.0 ** -126, 1.0),
      P("test_gemver_rowscaled_storage_bound", E4M3, 2.0 ** -4, 2.0 ** -6, 1.0),
      P("test_hand_worked_rowscaled_gemver_storage"),
      P("test_gemver_rowscaled_cost_against_the_amax_rule", BF16),
      P("test_gemver_rowscaled_cost_against_the_amax_rule", E4M3)]),
]

# Python oracles: (id, module, old, new, pins); ``old`` must occur once in the module.
PY_MUTANTS = [
    ("mlp_relu_mask_of_the_wrong_layer", "mlp", "dz2 = dh2 * (z2 > 0)", "dz2 = dh2 * (z1 > 0)",
     [P("test_mlp_gradient_central_differences")]),
    ("mlp_loss_gradient_without_the_2", "mlp", "df = 2.0 * (f - y) / B", "df = (f - y) / B",
     [P("test_mlp_gradient_central_differences")]),
    ("mlp_output_bias_gradient_averaged", "mlp", 'g["b3"] = np.array([df.sum()])', 'g["b3"] = np.array([df.mean()])',
     [P("test_mlp_gradient_central_differences")]),
    ("mlp_forward_drops_b2", "mlp", 'z2 = h1 @ P["W2"].T + P["b2"]', 'z2 = h1 @ P["W2"].T',
     [P("test_mlp_gradient_central_differences"), P("test_mlp_linear_region_closed_form")]),
    ("mlp_forward_W2_transposed", "mlp", 'z2 = h1 @ P["W2"].T + P["b2"]', 'z2 = h1 @ P["W2"] + P["b2"]',
     [P("test_mlp_gradient_central_differences")]),
    ("adam_without_bias_correction", "mlp", "mh = M[k] / (1 - b1 ** t)", "mh = M[k]",
     [P("test_adam_first_step_closed_form")]),
    ("adam_without_the_square_root", "mlp", "P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)",
     "P[k] = P[k] - lr * mh / (vh + eps)",
     [P("test_adam_first_step_closed_form")]),
    ("script_scal_ignores_its_scalar", "script", "r = axpby(a, X[0], 0.0, X[0])", "r = axpby(1.0, X[0], 0.0, X[0])",
     [P("test_script_elementary_ops")]),
    ("script_gemv_drops_the_accumulator", "script",
     "r = gemv(X[0], X[1], a, b, X[2] if len(X) > 2 else None)", "r = gemv(X[0], X[1], a, b, None)",
     [P("test_script_elementary_ops")]),
    ("script_gemvt_drops_the_accumulator", "script",
     "r = gemvt(X[0], X[1], a, b, X[2] if len(X) > 2 else None)", "r = gemvt(X[0], X[1], a, b, None)",
     [P("test_script_matches_sequences")]),
    ("script_ger_takes_the_second_scalar", "script", "r = ger(X[0], X[1], X[2], a)", "r = ger(X[0], X[1], X[2], b)",
     [P("test_script_elementary_ops"), P("test_script_matches_sequences")]),
    ("script_calls_run_in_reverse_order", "script", "for op, outs, ins, sc in calls:",
     "for op, outs, ins, sc in reversed(calls):",
     [P("test_script_in_place_semantics")]),
]


def _mutate_c(src, scope, old, new):
    start = src.index(scope)
    end = src.index("\n}\n", start)
    body = src[start:end]
    assert body.count(old) == 1, f"{old!r} must occur once in {scope}"
    return src[:start] + body.replace(old, new) + src[end:]


def _run_pins(pins):
    """Names of the pins that reject the oracle now in place.  Only a failed
    check counts; any other error propagates, since it would be a fault of
    the harness rather than a rejection."""
    rejected = []
    for name, args in pins:
        try:
            getattr(PINS, name)(*args)
        except AssertionError:
            rejected.append(name)
    return rejected


def _all_pins():
    seen = []
    for *_, pins in C_MUTANTS + PY_MUTANTS:
        for p in pins:
            if p not in seen:
                seen.append(p)
    return seen


def _python_copy(modname, old=None, new=None, label="copy"):
    """A module executed from the oracle module's source, with one edit."""
    src = open(getattr(oracle, modname).__file__).read()
    if old is not None:
        assert src.count(old) == 1, f"{old!r} must occur once in {modname}"
        src = src.replace(old, new)
    mod = types.ModuleType(f"oracle.{modname}")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src, f"<{label}>", "exec"), mod.__dict__)
    return mod


def _swap_in(monkeypatch, modname, mod):
    monkeypatch.setattr(oracle, modname, mod)
    if modname == "script":
        monkeypatch.setattr(PINS, "oscript", mod)


def test_unmutated_copies_pass_every_pin(tmp_path, monkeypatch):
    """The harness itself: the oracle built from unchanged copies of its
    sources passes every pin the mutants use."""
    path = tmp_path / "copy.c"
    path.write_text(open(oracle.SOURCE).read())
    lib = oracle.load(oracle.compile_source(str(path), str(tmp_path / "copy.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    for modname in ("mlp", "script"):
        _swap_in(monkeypatch, modname, _python_copy(modname))
    assert _run_pins(_all_pins()) == []


@pytest.mark.parametrize("mid,scope,old,new,pins", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_rejected(mid, scope, old, new, pins, tmp_path, monkeypatch):
    src = _mutate_c(open(oracle.SOURCE).read(), scope, old, new)
    path = tmp_path / f"{mid}.c"
    path.write_text(src)
    lib = oracle.load(oracle.compile_source(str(path), str(tmp_path / f"{mid}.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    assert _run_pins(pins), f"no pin rejects the mutant {mid}"


@pytest.mark.parametrize("mid,modname,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_is_rejected(mid, modname, old, new, pins, monkeypatch):
    _swap_in(monkeypatch, modname, _python_copy(modname, old, new, mid))
    assert _run_pins(pins), f"no pin rejects the mutant {mid}"
