"""Mutation tests of the oracle's pins.

The parity of the CUDA path is only as good as the oracle it is compared with,
and the oracle is trusted because its pins (tests/test_oracle_pins.py,
tests/test_mlp_oracle.py) tie it to hand-worked cases, closed forms, library
routines and brute force.  This file checks that those pins would notice the
mistakes one plausibly makes when writing such an oracle: each mutant below
plants one (a dropped term, a wrong sign or index, a transposed operand, a
rounding rule, a validation rule or a checker condition) in a copy of the
oracle, on the CPU, and the pin suites must fail on every copy.

A mutant is a list of exact (old, new) source edits; each `old` must occur
exactly once, so a refactor of the oracle that silently makes a mutant a no-op
fails here instead of passing."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")
ORACLE_MLP = os.path.join(ROOT, "oracle", "mlp.py")
PINS = ["tests/test_oracle_pins.py"]
MLP_PINS = ["tests/test_mlp_oracle.py"]

# ---------------------------------------------------------------------------
# mistakes in the DAG oracle (oracle.c)
C_MUTANTS = {
    # GEMM epilogue and K loop
    "gemm_drops_bias": [("        if (n->bias >= 0) v += get(&bias, 0, c0 + j);\n", "")],
    "gemm_drops_scale": [("double v = n->scale * acc[j];", "double v = acc[j];")],
    "gemm_activation_before_bias": [(
        "        double v = n->scale * acc[j];\n"
        "        if (n->bias >= 0) v += get(&bias, 0, c0 + j);\n"
        "        put(&O, r, c0 + j, activate(n->act, v));",
        "        double v = activate(n->act, n->scale * acc[j]);\n"
        "        if (n->bias >= 0) v += get(&bias, 0, c0 + j);\n"
        "        put(&O, r, c0 + j, v);")],
    "gemm_skips_first_k": [("      for (int64_t k = 0; k < K; ++k) {\n        double a = get(&A, r, k);",
                            "      for (int64_t k = 1; k < K; ++k) {\n        double a = get(&A, r, k);")],
    "gemm_ignores_trans_b": [("bp[k * w + j] = n->trans_b ?", "bp[k * w + j] = !n->trans_b ?")],
    "gemm_transposed_b_index": [("get(&Bm, bt * N + c0 + j, k)", "get(&Bm, bt * N + k, c0 + j)")],
    "gemm_b_ignores_batch": [("get(&Bm, bt * K + k, c0 + j)", "get(&Bm, k, c0 + j)")],
    "gemm_a_reads_row_zero": [("        double a = get(&A, r, k);", "        double a = get(&A, r % M, k);")],
    # activations and elementwise kernels
    "relu_wrong_sign": [("x < 0.0 ? 0.0 : x", "x > 0.0 ? 0.0 : x")],
    "gelu_wrong_scale": [("erf(x / sqrt(2.0))", "erf(x / 2.0)")],
    "gelu_tanh_form": [("0.5 * x * (1.0 + erf(x / sqrt(2.0)))",
                        "0.5 * x * (1.0 + tanh(0.7978845608028654 * (x + 0.044715 * x * x * x)))")],
    "add_subtracts": [("get(&A, r, j) + get(&Bm, r, j)", "get(&A, r, j) - get(&Bm, r, j)")],
    "add_drops_activation": [("activate(n->act, get(&A, r, j) + get(&Bm, r, j))", "get(&A, r, j) + get(&Bm, r, j)")],
    "unary_drops_activation": [("put(&O, r, j, activate(n->act, get(&A, r, j)));", "put(&O, r, j, get(&A, r, j));")],
    # softmax
    "softmax_not_stabilised": [("s += exp(n->scale * get(&A, r, j) - m);", "s += exp(n->scale * get(&A, r, j));"),
                               ("double y = exp(n->scale * get(&A, r, j) - m) / s;",
                                "double y = exp(n->scale * get(&A, r, j)) / s;")],
    "softmax_output_unscaled": [("double y = exp(n->scale * get(&A, r, j) - m) / s;",
                                 "double y = exp(get(&A, r, j) - m) / s;")],
    "softmax_sum_skips_first": [("for (int64_t j = 0; j < N; ++j) s +=", "for (int64_t j = 1; j < N; ++j) s +=")],
    "softmax_not_normalised": [("double y = exp(n->scale * get(&A, r, j) - m) / s;",
                                "double y = exp(n->scale * get(&A, r, j) - m);")],
    "softmax_sum_over_tile_columns": [("for (int64_t j = 0; j < N; ++j) s +=", "for (int64_t j = c0; j < c1; ++j) s +=")],
    # storage
    "bf16_truncates": [("q = rint(q);", "q = trunc(q);")],
    "bf16_ties_away": [("q = rint(q);", "q = round(q);")],
    "bf16_nine_bits": [("double q = ldexp(a, 7 - E);", "double q = ldexp(a, 8 - E);"),
                       ("v = ldexp(q, E - 7);", "v = ldexp(q, E - 8);")],
    "bf16_no_subnormal_floor": [("    if (E < -126) E = -126;   /* subnormal spacing 2^-133 */\n", "")],
    "bf16_load_shift": [("uint32_t u = (uint32_t)h << 16;", "uint32_t u = (uint32_t)h << 15;")],
    "view_offset_ignored": [("  a.coff = coff;", "  a.coff = 0;")],
    # validation and order
    "kahn_largest_id_first": [("    for (int v = 0; v < nn; ++v)\n      if (!done[v] && indeg[v] == 0)",
                               "    for (int v = nn - 1; v >= 0; --v)\n      if (!done[v] && indeg[v] == 0)")],
    "no_multiwriter_check": [("        if (overlap(&wu, &wv)) return OR_EMULTIWRITER;\n", "")],
    "no_in_place_check": [("        if (v == u && overlap(&wu, &r)) return OR_EMULTIWRITER;  /* in-place */\n", "")],
    "no_bias_shape_check": [("        if (B[n->bias].rows != 1 || B[n->bias].cols != N) return OR_ESHAPE;\n", "")],
    "no_inner_dim_check": [("      if (Kb != K || O->rows != A->rows || O->cols != N) return OR_ESHAPE;",
                            "      if (O->rows != A->rows || O->cols != N) return OR_ESHAPE;")],
    "no_add_shape_check": [(
        "      if (B[n->b].rows != O->rows || B[n->b].cols != O->cols || A->rows != O->rows || A->cols != O->cols)",
        "      if (A->rows != O->rows || A->cols != O->cols)")],
    "no_view_dtype_check": [("      if (p->dtype != B[i].dtype) return OR_EDTYPE;\n", "")],
    "edges_ignore_bias": [("  const or_node *n = &nodes[v];\n  int ins[3] = {n->a, n->b, n->bias};\n"
                           "  for (int q = 0; q < 3; ++q) {\n    if (ins[q] < 0) continue;\n"
                           "    or_region r = phys(B, ins[q], 0, B[ins[q]].rows, 0, B[ins[q]].cols);\n"
                           "    if (overlap(&w, &r)) return 1;",
                           "  const or_node *n = &nodes[v];\n  int ins[3] = {n->a, n->b, -1};\n"
                           "  for (int q = 0; q < 3; ++q) {\n    if (ins[q] < 0) continue;\n"
                           "    or_region r = phys(B, ins[q], 0, B[ins[q]].rows, 0, B[ins[q]].cols);\n"
                           "    if (overlap(&w, &r)) return 1;")],
    "topological_check_reversed": [("if (node_edge(B, nodes, u, v) && pos[u] > pos[v]) ok = 0;",
                                    "if (node_edge(B, nodes, u, v) && pos[u] < pos[v]) ok = 0;")],
    # tile regions, tiling and the trace checker
    "gemm_tile_reads_part_of_a": [("out[k++] = phys(B, n->a, t->r0, t->r1, 0, K);",
                                   "out[k++] = phys(B, n->a, t->r0, t->r1, t->c0, t->c1 < K ? t->c1 : K);")],
    "gemm_tile_reads_b_rows": [("else out[k++] = phys(B, n->b, bt * K, bt * K + K, t->c0, t->c1);",
                                "else out[k++] = phys(B, n->b, bt * K, bt * K + 1, t->c0, t->c1);")],
    "gemm_tile_ignores_bias_read": [("    if (n->bias >= 0) out[k++] = phys(B, n->bias, 0, 1, t->c0, t->c1);\n", "")],
    "add_tile_ignores_second_input": [("    if (n->op == OR_ADD) out[k++] = phys(B, n->b, t->r0, t->r1, t->c0, t->c1);\n", "")],
    "softmax_tile_reads_own_columns": [("out[k++] = phys(B, n->a, t->r0, t->r1, 0, B[n->a].cols);",
                                        "out[k++] = phys(B, n->a, t->r0, t->r1, t->c0, t->c1);")],
    "trace_allows_equal_tickets": [("!(end[u] < start[v])", "!(end[u] <= start[v])")],
    "trace_no_start_end_check": [("if (!(start[t] < end[t])) { *bad_u = t; return 2; }",
                                  "if (0) { *bad_u = t; return 2; }")],
    "trace_allows_double_cover": [("if (++cnt[r * C + c] > 1) { bad = 1; *bad_u = t; break; }",
                                   "++cnt[r * C + c];")],
    "trace_allows_gaps": [("      if (cnt[i] != 1) { bad = 1; *bad_v = v; }", "      if (cnt[i] > 1) { bad = 1; *bad_v = v; }")],
}

# mistakes in the cost model's oracle (mlp.py)
MLP_MUTANTS = {
    "loss_grad_drops_factor_two": [("dout = 2.0 * e / n", "dout = e / n")],
    "loss_grad_drops_mean": [("dout = 2.0 * e / n", "dout = 2.0 * e")],
    "second_relu_mask_dropped": [("dz2 = np.outer(dout, W3) * (z2 > 0)", "dz2 = np.outer(dout, W3)")],
    "first_relu_mask_dropped": [("dz1 = (dz2 @ W2.T) * (z1 > 0)", "dz1 = dz2 @ W2.T")],
    "w2_not_transposed": [("dz1 = (dz2 @ W2.T) * (z1 > 0)", "dz1 = (dz2 @ W2) * (z1 > 0)")],
    "grad_w2_transposed": [("gW2 = h1.T @ dz2", "gW2 = (h1.T @ dz2).T")],
    "grad_b1_dropped": [("gb1 = dz1.sum(axis=0)", "gb1 = 0.0 * dz1.sum(axis=0)")],
    "forward_second_relu_dropped": [("h2 = np.maximum(z2, 0.0)", "h2 = z2")],
    "forward_drops_b3": [("out = h2 @ W3 + b3", "out = h2 @ W3")],
    "adam_no_bias_correction": [("p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)",
                                 "p -= lr * m / (np.sqrt(v) + eps)")],
    "adam_eps_inside_sqrt": [("p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)",
                              "p -= lr * (m / (1 - b1 ** t)) / np.sqrt(v / (1 - b2 ** t) + eps)")],
    "adam_first_moment_weights_swapped": [("m = b1 * m + (1 - b1) * g", "m = (1 - b1) * m + b1 * g")],
    "adam_always_first_batch": [("s = ((t - 1) * batch) % n", "s = 0")],
    "adam_step_counter_from_zero": [("(m / (1 - b1 ** t))", "(m / (1 - b1 ** (t + 1)))"),
                                    ("(np.sqrt(v / (1 - b2 ** t))", "(np.sqrt(v / (1 - b2 ** (t + 1)))")],
}


def _mutate(src: str, edits):
    for old, new in edits:
        n = src.count(old)
        assert n == 1, f"edit target occurs {n} times: {old!r}"
        src = src.replace(old, new)
    return src


def _run_pins(env_key, path, pins):
    env = dict(os.environ, **{env_key: path})
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", *pins],
                       cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True,
                       timeout=600)
    return r.returncode, r.stdout


def _survivors(kind, mutants, tmp):
    src = open(ORACLE_C if kind == "c" else ORACLE_MLP).read()

    def one(item):
        name, edits = item
        text = _mutate(src, edits)
        if kind == "c":
            c_path = os.path.join(tmp, f"{name}.c")
            so_path = os.path.join(tmp, f"lib{name}.so")
            with open(c_path, "w") as f:
                f.write(text)
            oracle.compile_source(c_path, so_path)
            rc, out = _run_pins("ORACLE_MUTANT_LIB", so_path, PINS)
        else:
            py_path = os.path.join(tmp, f"mlp_{name}.py")
            with open(py_path, "w") as f:
                f.write(text)
            rc, out = _run_pins("ORACLE_MUTANT_MLP", py_path, MLP_PINS)
        # exit code 1 = some test failed; 0 = every pin passed (the mutant survived);
        # anything else (collection error, crash) is not a pin catching the mistake
        return name, rc, out

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(one, sorted(mutants.items())))
    survived = [n for n, rc, _ in results if rc == 0]
    odd = [(n, rc, out[-600:]) for n, rc, out in results if rc not in (0, 1)]
    return survived, odd


def test_unmutated_oracle_passes_its_pins(tmp_path):
    """The control: an unmodified copy, loaded the same way, passes."""
    so_path = str(tmp_path / "liboracle_copy.so")
    oracle.compile_source(ORACLE_C, so_path)
    rc, out = _run_pins("ORACLE_MUTANT_LIB", so_path, PINS)
    assert rc == 0, out[-2000:]
    rc, out = _run_pins("ORACLE_MUTANT_MLP", ORACLE_MLP, MLP_PINS)
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("kind,mutants", [("c", C_MUTANTS), ("mlp", MLP_MUTANTS)], ids=["dag_oracle", "mlp_oracle"])
def test_every_planted_mistake_fails_a_pin(kind, mutants, tmp_path):
    survived, odd = _survivors(kind, mutants, str(tmp_path))
    assert not odd, odd
    assert not survived, f"mistakes no pin catches: {survived}"
