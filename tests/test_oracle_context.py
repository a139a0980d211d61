"""Pins of the oracle's choice of the context (compartment) a rule fires in.

Sec. 2.2 counts the reactant combinations of a rule "in the same context" and
the simulator's Resolve step (Sec. 5.1, Fig. "CWC simulator pseudo-code")
first draws the rule with probability proportional to its total propensity
and then, by a separate stochastic choice, the context: compartment c of rule
j must fire with probability h_c / H_j, h_c the number of reactant
combinations at c and H_j = sum_c h_c.  The written specification makes the
choice an integer one: with W the 64-bit purpose-1 Philox word of the event,
x_c = floor(W H_j / 2^64) and the context is the first slot, in ascending
order, whose running sum of h exceeds x_c.

Two pins, each chosen so that which compartment fires changes what is checked:

* the law: three compartments with different contents; after one event the
  released content (dissolution) or the chosen slot must follow h_c / H_j
  (chi-square at fixed seeds).  A scan biased to the first positive context
  puts every firing in slot 1, and a uniform choice among contexts gives 1/3
  each; both fail with p far below 1e-4 (with n = 1, 3, 8 the expected shares
  are 1/12, 3/12, 8/12).
* the exact draw: on hand-built terms, every replica's chosen slot equals a
  recomputation with Python integers from the Philox word (the oracle's
  Philox is pinned against cuRAND's Philox4_32_10 on the GPU).  Scanning
  the slots in descending order, or taking W's two 32-bit words in the other
  order, keeps the law but fails this pin (each planted in the oracle on the
  CPU: the law tests pass, both exact-draw tests fail; a first-positive scan
  fails all five).
"""
import numpy as np
from scipy import stats

import oracle
from paper_1010_2438_gb300 import workloads as W

P_MIN = 1e-4


def _run(model, img, R, seed, rates=None, max_events=1):
    rates = np.ones((1, model.n_rules)) if rates is None else np.atleast_2d(rates)
    b = W.Batch(model, rates, img[None].astype(np.int32), np.array([0.0, 1e12]), R, seed,
                max_events=max_events)
    return oracle.simulate(b, log_cap=1, threads=8)


def _chi2(counts, probs):
    counts = np.asarray(counts, np.float64)
    exp = np.asarray(probs, np.float64) * counts.sum()
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    return float(stats.chi2.sf(chi2, len(counts) - 1))


def test_dissolution_releases_the_content_of_a_child_chosen_with_probability_h():
    """DISSOLVE top: X (x | a Y)^1 -> a X x Y with a child-content pattern a:
    h_d = n_d (the child's count of a), so after the first event the top
    level holds exactly the content of the dissolved child, n_d, with
    probability n_d / sum n."""
    n = [1, 3, 8]
    rules = [W.RuleSpec(W.DISSOLVE, 0, 1, lhs_child={0: 1}, rhs_ctx={0: 1})]
    model = W.cwc_model(1, 2, 4, rules)
    img = W.empty_slot_image(model)
    for d, nd in enumerate(n, start=1):
        img[d, :3] = [1, 1, 0]
        img[d, 3 + 1 + 0] = nd          # content of species 0 (after 3 header words + 1 wrap word)
    res = _run(model, img, 24000, 77)
    assert np.all(res["events"] == 1)
    top = res["states"][:, -1, 0]        # observable 0: top-level content of species 0
    slot = res["log_slot"][:, 0]
    assert set(np.unique(slot)) <= {1, 2, 3}
    assert np.array_equal(top, np.asarray(n)[slot - 1])
    # alive label-1 compartments after the event: two of three
    assert np.all(res["states"][:, -1, model.n_observables - 1] == 2)
    counts = [(top == nd).sum() for nd in n]
    probs = np.asarray(n, np.float64) / sum(n)
    assert _chi2(counts, probs) > P_MIN, (counts, probs)


def test_local_rule_context_law_with_binomial_weights():
    """LOCAL label-1 rule 2a -> b: h_c = C(n_c, 2); contexts with n = 2, 5, 0,
    9 (the empty one must never fire).  The chosen slot follows h_c / H."""
    n = [2, 5, 0, 9]
    rules = [W.RuleSpec(W.LOCAL, 1, lhs_ctx={0: 2}, rhs_ctx={1: 1})]
    model = W.cwc_model(2, 2, 6, rules)
    img = W.empty_slot_image(model)
    for d, nd in enumerate(n, start=1):
        img[d, :3] = [1, 1, 0]
        img[d, 3 + 2 + 0] = nd
    res = _run(model, img, 30000, 1234)
    slot = res["log_slot"][:, 0]
    h = np.array([v * (v - 1) // 2 for v in n], np.float64)
    counts = [(slot == d).sum() for d in range(1, 5)]
    assert counts[2] == 0
    keep = h > 0
    assert _chi2(np.asarray(counts)[keep], h[keep] / h.sum()) > P_MIN, counts


def test_parent_child_context_law_over_children_of_different_parents():
    """PARENT_CHILD top <- label-1 'out' rule with a child-content pattern,
    whose contexts are the label-1 children of the top only: a label-1
    compartment nested in a label-2 one is not a context.  h_d = n_d."""
    rules = [W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_child={0: 1}, rhs_ctx={0: 1})]
    model = W.cwc_model(1, 3, 6, rules)
    img = W.empty_slot_image(model)
    img[1, :3] = [1, 1, 0]
    img[1, 4] = 4
    img[2, :3] = [1, 2, 0]               # a label-2 compartment of the top
    img[3, :3] = [1, 1, 2]               # label 1 inside label 2: not a context
    img[3, 4] = 50
    img[4, :3] = [1, 1, 0]
    img[4, 4] = 6
    res = _run(model, img, 20000, 5)
    slot = res["log_slot"][:, 0]
    assert set(np.unique(slot)) <= {1, 4}
    counts = [(slot == 1).sum(), (slot == 4).sum()]
    assert _chi2(counts, [0.4, 0.6]) > P_MIN, counts


# ----------------------------------------------------------------------------
# The exact integer draw
# ----------------------------------------------------------------------------

def _expected_slots(model, img, R, seed, h_of_slot):
    """Recompute the chosen context of event 0 of every replica with Python
    integers: W from the purpose-1 Philox word, x = floor(W H / 2^64), first
    ascending slot whose running h exceeds x."""
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    ctr = np.zeros((R, 4), np.uint32)
    ctr[:, 1] = 1                        # purpose 1: the context word
    ctr[:, 2] = np.arange(R, dtype=np.uint32)
    words = oracle.philox(ctr, key)
    slots = sorted(h_of_slot)
    H = sum(h_of_slot.values())
    out = []
    for r in range(R):
        Wd = int(words[r, 0]) | (int(words[r, 1]) << 32)
        x = (Wd * H) >> 64
        cum = 0
        pick = None
        for c in slots:
            cum += h_of_slot[c]
            if x < cum:
                pick = c
                break
        out.append(pick)
    return np.array(out)


def test_context_draw_equals_integer_recomputation_large_counts():
    """h_c up to ~7e9 (so W H needs the full 128-bit product), a zero-h
    context between positive ones and a dead slot."""
    rules = [W.RuleSpec(W.LOCAL, 1, lhs_ctx={0: 1, 1: 1}, rhs_ctx={2: 1})]
    model = W.cwc_model(3, 2, 8, rules)
    img = W.empty_slot_image(model)
    counts = {1: (100000, 70000), 2: (3, 1), 3: (0, 12345), 5: (65536, 65536), 6: (7, 900001)}
    for c, (a, b) in counts.items():
        img[c, :3] = [1, 1, 0]
        img[c, 3 + 3 + 0] = a
        img[c, 3 + 3 + 1] = b
    h = {c: a * b for c, (a, b) in counts.items()}
    R, seed = 4096, 0x0123456789ABCDEF
    res = _run(model, img, R, seed)
    assert np.all(res["events"] == 1)
    want = _expected_slots(model, img, R, seed, h)
    assert np.array_equal(res["log_slot"][:, 0], want)
    # the three large contexts all fire in 4096 draws (slot 2, h = 3 of H ~ 1.1e10,
    # practically never), the empty one never
    assert {1, 5, 6} <= set(np.unique(want).tolist()) and 3 not in set(want.tolist())


def test_context_draw_equals_integer_recomputation_dissolve_small_counts():
    """Small h (1, 2, 1) over children of the top, where floor(W H / 2^64)
    decides between adjacent contexts at every boundary."""
    rules = [W.RuleSpec(W.DISSOLVE, 0, 1, lhs_wrap={0: 1})]
    model = W.cwc_model(1, 2, 5, rules)
    img = W.empty_slot_image(model)
    wraps = {1: 1, 3: 2, 4: 1}
    for c, w in wraps.items():
        img[c, :3] = [1, 1, 0]
        img[c, 3] = w                    # wrap count of species 0
    R, seed = 2048, 99
    res = _run(model, img, R, seed)
    want = _expected_slots(model, img, R, seed, wraps)
    assert np.array_equal(res["log_slot"][:, 0], want)
