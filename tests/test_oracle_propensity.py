"""Pins of the oracle's combinatorial counts (Match / Match_Populations, Sec. 2.2, 5.1)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1010_2438_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_worked_example():
    """Sec. 2.2: l: a b X -> c X on a a b b has 4 reactant combinations, rate 4k."""
    g = json.load(open(os.path.join(GOLDEN, "paper_example.json")))
    sp = g["species"]
    model = W.flat_model(len(sp), [({sp.index(s): c for s, c in g["rule"]["lhs"].items()},
                                    {sp.index(s): c for s, c in g["rule"]["rhs"].items()})])
    term = np.array([[g["term"][s] for s in sp]], np.int32)
    H = oracle.rule_totals(model, term)
    assert H[0] == g["combinations"] == 4
    # the rate k*4 is what the simulator uses: with k = 0.25 the term a a b b
    # reacts with total propensity 1, and after one event a b c remains
    b = W.Batch(model, np.array([[0.25]]), term, np.array([0.0, 1e9]), 1, 5)
    res = oracle.simulate(b, log_cap=4)
    assert res["events"][0] == 2          # a a b b -> a b c -> c c, then absorbed
    assert res["status"][0] == oracle.ST_ABSORBED
    assert list(res["states"][0, -1]) == [0, 0, 2]


def test_paper_term_example_observables():
    """Sec. 2.1: the term a b (c d | e f)^l, observed by label."""
    g = json.load(open(os.path.join(GOLDEN, "paper_term_example.json")))
    sp = g["species"]
    S = len(sp)
    rule = W.RuleSpec(W.LOCAL, 1, lhs_ctx={sp.index("e"): 1}, rhs_ctx={sp.index("e"): 1})
    model = W.cwc_model(S, 2, 2, [rule])
    img = W.empty_slot_image(model)
    for s, c in g["top_content"].items():
        img[0, 3 + S + sp.index(s)] = c
    img[1, :3] = [1, 1, 0]
    for s, c in g["compartment"]["wrap"].items():
        img[1, 3 + sp.index(s)] = c
    for s, c in g["compartment"]["content"].items():
        img[1, 3 + S + sp.index(s)] = c
    b = W.Batch(model, np.array([[1.0]]), img[None], np.array([0.0]), 1, 1)
    st = oracle.simulate(b)["states"][0, 0]
    O = model.n_observables
    assert O == 2 * S + S + 2
    top = st[:S]
    inner = st[S:2 * S]
    wrap = st[2 * S:3 * S]
    alive = st[3 * S:]
    assert list(top) == [1, 1, 0, 0, 0, 0]
    assert list(inner) == [0, 0, 0, 0, 1, 1]
    assert list(wrap) == [0, 0, 1, 1, 0, 0]
    assert list(alive) == [1, 1]


def _brute_force(term_counts, pattern):
    """Count distinct reactant combinations by enumerating molecule identities."""
    molecules = [(s, i) for s, n in enumerate(term_counts) for i in range(n)]
    need = sum(pattern)
    count = 0
    for combo in itertools.combinations(molecules, need):
        got = [0] * len(term_counts)
        for s, _ in combo:
            got[s] += 1
        if got == list(pattern):
            count += 1
    return count


def test_brute_force_counts():
    rng = np.random.default_rng(31)
    S = 4
    for _ in range(150):
        pattern = [0] * S
        for s in rng.choice(S, size=rng.integers(0, 3), replace=False):
            pattern[s] = int(rng.integers(1, 3))
        term = [int(v) for v in rng.integers(0, 6, S)]
        model = W.flat_model(S, [({s: c for s, c in enumerate(pattern) if c}, {})])
        H = oracle.rule_totals(model, np.array([term], np.int32))
        assert H[0] == _brute_force(term, pattern)


def _transport_model(n_children, k_in=1.0, k_out=1.0):
    rules = [
        W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_ctx={0: 1}, rhs_child={0: 1}),
        W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_child={0: 1}, rhs_ctx={0: 1}),
    ]
    return W.cwc_model(1, 2, 1 + n_children, rules)


def test_parent_child_count_is_population_times_compartments():
    """Fig. simd pseudocode: stoch_rate = count_population * count_compartments * k
    when the child patterns are empty; per-child contexts sum to exactly that."""
    for n_children in (1, 2, 5):
        model = _transport_model(n_children)
        img = W.empty_slot_image(model)
        img[0, 3 + 1] = 7            # 7 A in the root content
        for d in range(1, n_children + 1):
            img[d, :3] = [1, 1, 0]
            img[d, 3 + 1] = d        # d A inside child d
        H = oracle.rule_totals(model, img)
        assert H[0] == 7 * n_children
        assert H[1] == sum(range(1, n_children + 1))


def test_parent_child_wrap_and_child_factors():
    # rule: top: a X (b x | c c Y)^1 -> ... ; h = n_a * w_b * C(n_c, 2) per child
    rule = W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_ctx={0: 1}, lhs_wrap={1: 1}, lhs_child={2: 2})
    model = W.cwc_model(3, 2, 4, [rule])
    img = W.empty_slot_image(model)
    img[0, 3 + 3 + 0] = 5
    vals = [(2, 4), (0, 9), (3, 1)]
    for d, (wb, nc) in enumerate(vals, start=1):
        img[d, :3] = [1, 1, 0]
        img[d, 3 + 1] = wb
        img[d, 3 + 3 + 2] = nc
    H = oracle.rule_totals(model, img)
    assert H[0] == sum(5 * wb * (nc * (nc - 1) // 2) for wb, nc in vals)


def test_label_filtering():
    # LOCAL rule of label 2 only sees label-2 compartments; PARENT_CHILD(1 -> 2)
    # only children of label 2 whose parent has label 1
    rules = [W.RuleSpec(W.LOCAL, 2, lhs_ctx={0: 1}),
             W.RuleSpec(W.PARENT_CHILD, 1, 2, lhs_child={0: 1})]
    model = W.cwc_model(1, 3, 5, rules)
    img = W.empty_slot_image(model)
    # slot 1: label 1 in root; slot 2: label 2 in slot 1; slot 3: label 2 in root
    for d, lab, par, cnt in ((1, 1, 0, 3), (2, 2, 1, 4), (3, 2, 0, 6)):
        img[d, :3] = [1, lab, par]
        img[d, 3 + 1] = cnt
    H = oracle.rule_totals(model, img)
    assert H[0] == 4 + 6
    assert H[1] == 4
