"""Planted mistakes: every pin of the oracle catches the mistakes it is there for.

Each case copies oracle/cwc_oracle.c, replaces one snippet (it must occur
exactly once) with a plausible mistake, and compiles the copy with the
oracle's own flags into a temporary library. The mistakes are a dropped term,
a wrong coefficient, a swapped operand, a missing guard, or a wrong order.
The named pin tests then run in a child pytest, with CWC_ORACLE_LIBRARY
pointing the oracle module at the copy.

The child must report every named test as failed. It must do so through
pytest's "tests failed" exit status, not a crash. Where a case also names
pins that must still pass, it shows which pin catches which mistake: a
context scan in the wrong order keeps the law, and only the exact-draw pins
see it.

Everything happens on the CPU, in copies: the built oracle is untouched, and
it passes every pin in the main run.
"""
import os
import re
import shutil
import subprocess
import sys

import pytest

from oracle import build as oracle_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CTX = "tests/test_oracle_context.py::"
PRIM = "tests/test_oracle_primitives.py::"
PROP = "tests/test_oracle_propensity.py::"
LAWS = "tests/test_oracle_laws.py::"
GEN = "tests/test_oracle_general_patterns.py::"
SENS = "tests/test_oracle_sensitivity.py::"
RATE = "tests/test_oracle_rate_laws.py::"
HASH = "tests/test_oracle_hash.py::"
CTX_LAWS = [CTX + "test_dissolution_releases_the_content_of_a_child_chosen_with_probability_h",
            CTX + "test_local_rule_context_law_with_binomial_weights",
            CTX + "test_parent_child_context_law_over_children_of_different_parents"]
CTX_DRAWS = [CTX + "test_context_draw_equals_integer_recomputation_large_counts",
             CTX + "test_context_draw_equals_integer_recomputation_dissolve_small_counts"]
LOG_PINS = [PRIM + "test_log_spec_within_0p55_ulp_of_60_digit_logarithms", PRIM + "test_log_spec_accuracy_random"]

# name: (snippet of cwc_oracle.c, planted replacement, pins that must fail, pins that must still pass)
CASES = {
    # Resolve step, the context choice (Sec. 2.2 "in the same context"; the simulator's stochastic_choice)
    "context: first positive slot instead of the drawn one": (
        "        if (xc < cum) { ctx = c; break; }",
        "        if (hc > 0) { ctx = c; break; }",
        CTX_LAWS + CTX_DRAWS, []),
    "context: slots scanned in descending order": (
        "for (int c = 0; c < C && m->kind[j] != K_FUSION && m->kind[j] != K_PAIR; c++) {",
        "for (int c = C - 1; c >= 0 && m->kind[j] != K_FUSION && m->kind[j] != K_PAIR; c--) {",
        CTX_DRAWS, CTX_LAWS),
    "context: the Philox word's halves swapped": (
        "uint64_t W = (uint64_t)wc[0] | ((uint64_t)wc[1] << 32);",
        "uint64_t W = (uint64_t)wc[1] | ((uint64_t)wc[0] << 32);",
        CTX_DRAWS, CTX_LAWS),
    "context: parent's label not checked": (
        "  return t->label[c] == m->child_label[j] && t->label[q] == m->ctx_label[j];",
        "  return t->label[c] == m->child_label[j];",
        [PROP + "test_label_filtering", CTX + "test_parent_child_context_law_over_children_of_different_parents"],
        []),
    # Match step, Match_Populations counts
    "match: C(n, 2) without its 1/2": (
        "*out = n * (n - 1) / 2;",
        "*out = n * (n - 1);",
        [PROP + "test_brute_force_counts", LAWS + "test_dimerisation_cme"], []),
    "match: FUSION / PAIR occurrences never unordered": (
        "      if (rhs[S + x] != rhs[3 * S + x] || rhs[2 * S + x] != rhs[4 * S + x]) return 0;\n  return 1;",
        "      if (rhs[S + x] != rhs[3 * S + x] || rhs[2 * S + x] != rhs[4 * S + x]) return 0;\n  return 0;",
        [GEN + "test_fusion_counts_unordered_pairs_only_for_identical_patterns",
         GEN + "test_pair_counts_unordered_pairs_only_for_fully_symmetric_rules"], []),
    "rate law: Michaelis-Menten denominator without the substrate": (
        "const double den = m->rate_par[j] + (double)x[sub];",
        "const double den = m->rate_par[j];",
        [RATE + "test_michaelis_menten_value_closed_forms"], []),
    # time step: tau = -ln(u) / a0 with the fixed logarithm
    "time step: multiplied by a0 instead of divided": (
        "double tau = (-oracle_log_spec(u_tau)) / a0;",
        "double tau = (-oracle_log_spec(u_tau)) * a0;",
        [LAWS + "test_birth_death_transient_law[25]"], []),
    "logarithm: a wrong coefficient in the ln 2 series": (
        "acc += (((u128)1) << (120 - k)) / (u128)k;",
        "acc += (((u128)1) << (120 - k)) / (u128)(k + 1);",
        LOG_PINS, []),
    "logarithm: ln(1 + y) series without its y^2 / 2 term": (
        "for (int k = 10; k >= 2; k--) p = cq[k] - mulhi64(p, yq);",
        "for (int k = 10; k >= 3; k--) p = cq[k] - mulhi64(p, yq);",
        LOG_PINS, []),
    "logarithm: Mercator series near one without its last step": (
        "for (int n = 8; n >= 1; n--) q = cq[n] + mulhi64(q, dq);",
        "for (int n = 8; n >= 2; n--) q = cq[n] + mulhi64(q, dq);",
        [PRIM + "test_log_spec_within_0p55_ulp_of_60_digit_logarithms", PRIM + "test_log_spec_edges"], []),
    "uniform: (k + 1/2) 2^-52 without the half": (
        "return ((double)k + 0.5) * 0x1p-52;",
        "return ((double)k) * 0x1p-52;",
        [PRIM + "test_u52_boundaries_and_exactness"], []),
    "Philox: a wrong round multiplier": (
        "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
        "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;",
        [PRIM + "test_philox_known_answer_vectors"], []),
    "Philox: the key bumped before the first round": (
        "    if (round > 0) {\n      k0 += 0x9E3779B9u;",
        "    if (round >= 0) {\n      k0 += 0x9E3779B9u;",
        [PRIM + "test_philox_known_answer_vectors"], []),
    # the 32-lane blocked tree and the guarded descent
    "tree: a node keeps only its left child": (
        "nodes[LEVEL_BASE[k] + i] = nodes[LEVEL_BASE[k - 1] + 2 * i] + nodes[LEVEL_BASE[k - 1] + 2 * i + 1];",
        "nodes[LEVEL_BASE[k] + i] = nodes[LEVEL_BASE[k - 1] + 2 * i];",
        [PRIM + "test_tree_sum_exact_cases"], []),
    "descent: the guard against an empty right subtree dropped": (
        "    if (x < SL || SR == 0.0) {",
        "    if (x < SL || SR != SR) {",
        [PRIM + "test_select_never_picks_zero"], []),
    # Update step, the rewrite of the matched multisets (Sec. 2.1)
    "update: a dissolved compartment's children not re-parented": (
        "if (t->alive[d] && d != c && t->parent[d] == c) t->parent[d] = q;",
        "if (t->alive[d] && d != c && t->parent[d] == c) t->parent[d] = t->parent[d];",
        [LAWS + "test_cwc_dissolve_reparents_children"], []),
    "update: a dissolved compartment's wrap lost": (
        "      xp[s] = xp[s] + rhs[s] - lhs[s] + (w[s] - lhs[S + s]) + (xc[s] - lhs[2 * S + s]);",
        "      xp[s] = xp[s] + rhs[s] - lhs[s] + (xc[s] - lhs[2 * S + s]);",
        [LAWS + "test_cwc_create_dissolve_token_law"], []),
    "update: transport applied in the other direction": (
        "      xp[s] = xp[s] + rhs[s] - lhs[s];\n      w[s] = w[s] + rhs[S + s] - lhs[S + s];\n"
        "      xc[s] = xc[s] + rhs[2 * S + s] - lhs[2 * S + s];",
        "      xp[s] = xp[s] + rhs[2 * S + s] - lhs[2 * S + s];\n      w[s] = w[s] + rhs[S + s] - lhs[S + s];\n"
        "      xc[s] = xc[s] + rhs[s] - lhs[s];",
        [LAWS + "test_cwc_transport_two_children_binomial"], []),
    "update: a created compartment takes the context's label": (
        "    t->label[e] = m->child_label[j];",
        "    t->label[e] = m->ctx_label[j];",
        [LAWS + "test_cwc_create_dissolve_token_law"], []),
    "update: FUSION drops the second compartment's content": (
        "      int32_t xm = x1[s] - lhs[2 * S + s] + x2[s] - lhs[4 * S + s] + rhs[2 * S + s];",
        "      int32_t xm = x1[s] - lhs[2 * S + s] + rhs[2 * S + s];",
        [GEN + "test_fusion_merges_wraps_and_contents_and_moves_children"], []),
    "update: PAIR rewrites the first compartment twice": (
        "    int32_t* ms[5] = {t->content + (size_t)q * S, t->wrap + (size_t)d1 * S, t->content + (size_t)d1 * S,\n"
        "                      t->wrap + (size_t)d2 * S, t->content + (size_t)d2 * S};",
        "    int32_t* ms[5] = {t->content + (size_t)q * S, t->wrap + (size_t)d1 * S, t->content + (size_t)d1 * S,\n"
        "                      t->wrap + (size_t)d1 * S, t->content + (size_t)d1 * S};",
        [GEN + "test_pair_rewrites_both_compartments_in_place"], []),
    "update: NESTED rewrites the child's content for the grandparent's": (
        "    int32_t* ms[5] = {t->content + (size_t)a * S, t->wrap + (size_t)q * S, t->content + (size_t)q * S,",
        "    int32_t* ms[5] = {t->content + (size_t)q * S, t->wrap + (size_t)q * S, t->content + (size_t)q * S,",
        [GEN + "test_nested_transport_from_grandchildren_is_binomial"], []),
    "update: no int32 overflow check": (
        "static int fits(int64_t v) { return v >= 0 && v <= 2147483647LL; }",
        "static int fits(int64_t v) { return v >= 0; }",
        [LAWS + "test_bad_input_and_overflow_statuses"], []),
    # the event hash compared by parity
    "hash: the slot's bytes before the rule's": (
        "  for (int i = 0; i < 4; i++) bytes[i] = (uint8_t)(rule >> (8 * i));\n"
        "  for (int i = 0; i < 4; i++) bytes[4 + i] = (uint8_t)(slot >> (8 * i));",
        "  for (int i = 0; i < 4; i++) bytes[4 + i] = (uint8_t)(rule >> (8 * i));\n"
        "  for (int i = 0; i < 4; i++) bytes[i] = (uint8_t)(slot >> (8 * i));",
        [HASH + "test_flat_hash_is_fnv1a_of_the_event_log",
         HASH + "test_compartment_hash_is_fnv1a_of_the_event_log"], [HASH + "test_fnv1a64_published_values"]),
    "hash: a wrong FNV prime": (
        "    h *= 0x100000001b3ull;",
        "    h *= 0x100000001b5ull;",
        [HASH + "test_flat_hash_is_fnv1a_of_the_event_log",
         HASH + "test_compartment_hash_is_fnv1a_of_the_event_log"], []),
    # the likelihood-ratio score
    "score: the integral of h dropped": (
        "for (int i = 0; i < M; i++) x.I[i] = x.I[i] + x.Hs[i] * (tnext - tnow);",
        "for (int i = 0; i < M; i++) x.I[i] = x.I[i];",
        [SENS + "test_birth_death_lr_matches_analytic_gradient"], []),
}


def _child_pytest(lib_path, node_ids):
    env = dict(os.environ)
    env["CWC_ORACLE_LIBRARY"] = lib_path
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-rf", *node_ids],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    failed = set(re.findall(r"^FAILED (\S+?)(?: - .*)?$", r.stdout, re.M))
    return r.returncode, failed, r.stdout[-3000:]


@pytest.mark.parametrize("name", list(CASES))
def test_planted_mistake_fails_its_pins(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new, must_fail, must_pass = CASES[name]
    with open(oracle_build.SRC) as f:
        src = f.read()
    assert src.count(old) == 1, "snippet not found exactly once: %r" % old
    c_path = tmp_path / "mutant.c"
    so_path = tmp_path / "libmutant.so"
    c_path.write_text(src.replace(old, new))
    subprocess.run(["gcc", *oracle_build.FLAGS, "-o", str(so_path), str(c_path), "-lm"], check=True,
                   capture_output=True)
    rc, failed, out = _child_pytest(str(so_path), must_fail)
    assert rc == 1, "expected failing pins, got exit status %d:\n%s" % (rc, out)
    assert set(must_fail) <= failed, "pins that did not catch the mistake: %s\n%s" % (set(must_fail) - failed, out)
    if must_pass:
        rc, failed, out = _child_pytest(str(so_path), must_pass)
        assert rc == 0, "pins expected to keep passing failed:\n%s" % out
