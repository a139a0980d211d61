"""Pins of the oracle's general CWC patterns: two compartments in one
left-hand side, merged (FUSION) or both kept (PAIR), and a pattern of depth
two (NESTED).

Sec. 2.1 lets a pattern be any term with variables, so a left-hand side may
hold several compartments, themselves holding compartments; Sec. 2.2 counts
the "distinct occurrences, in the same context, of subterms matching" the
rule.  The pins check the oracle against that definition and against laws:

* brute force: every atom of a small term gets an identity; every way of
  matching the left-hand side (compartment choices and atom choices) yields
  the set of identified items it consumes; the number of distinct sets is the
  rule's combinatorial count.  This fixes, among others, that a FUSION whose
  two compartment patterns are identical counts unordered pairs and one
  whose patterns differ counts ordered pairs (the oracle's rule), and that
  NESTED matches only grandchildren under the right labels.  A PAIR keeps
  both compartments, each with its own right-hand side, so a match and its
  swap are one application only when both the left- and the right-hand
  patterns of the two compartments are identical (same consumed items, same
  resulting term); the brute force then keys an application by its consumed
  items plus, when the right-hand patterns differ, which compartment played
  the first role.
* laws: fusion of m empty compartments at rate k per pair is a pure-death
  chain with rate k C(n, 2) (Kingman's coalescent), checked against the
  chemical master equation; content is conserved by fusion; transport from a
  grandchild to its grandparent at rate k per atom leaves Bin(N, 1 - e^-kt)
  atoms at the top; PAIR transport of one atom at a time between two sibling
  compartments at rate k per atom is the Ehrenfest model: every atom flips
  independently at rate k, so N atoms started in the first compartment leave
  Bin(N, (1 + e^-2kt) / 2) there.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import linalg, stats

import oracle
from paper_1010_2438_gb300 import workloads as W

P_MIN = 1e-4


# ----------------------------------------------------------------------------
# Brute-force count of distinct occurrences
# ----------------------------------------------------------------------------

def _choices(place, counts, pattern):
    """All ways to pick the pattern's atoms from one multiset of identified
    atoms: place = (slot, 'w' or 'c'); counts[s] atoms of species s."""
    per_species = []
    for s, nu in enumerate(pattern):
        if nu == 0:
            continue
        per_species.append([frozenset((place, s, i) for i in comb)
                            for comb in itertools.combinations(range(counts[s]), nu)])
    out = []
    for combo in itertools.product(*per_species):
        items = frozenset()
        for c in combo:
            items |= c
        out.append(items)
    return out


def brute_force_count(model, img, j):
    S = model.n_species
    lhs5, _, grand = model.rows5()
    lhs = lhs5[j]
    alive = [c for c in range(img.shape[0]) if img[c, 0] == 1]
    label = {c: int(img[c, 1]) for c in alive}
    parent = {c: int(img[c, 2]) for c in alive}
    wrap = {c: img[c, 3:3 + S] for c in alive}
    cont = {c: img[c, 3 + S:3 + 2 * S] for c in alive}
    kind, lab, ch = int(model.kind[j]), int(model.ctx_label[j]), int(model.child_label[j])
    occ = set()
    if kind in (W.FUSION, W.PAIR):
        _, rhs5, _ = model.rows5()
        role = kind == W.PAIR and not (np.array_equal(rhs5[j][1], rhs5[j][3]) and
                                       np.array_equal(rhs5[j][2], rhs5[j][4]))
        for d1 in alive:
            for d2 in alive:
                if d1 == d2 or d1 == 0 or d2 == 0 or label[d1] != ch or label[d2] != ch:
                    continue
                if parent[d1] != parent[d2] or label[parent[d1]] != lab:
                    continue
                q = parent[d1]
                for parts in itertools.product(_choices((q, "c"), cont[q], lhs[0]),
                                               _choices((d1, "w"), wrap[d1], lhs[1]),
                                               _choices((d1, "c"), cont[d1], lhs[2]),
                                               _choices((d2, "w"), wrap[d2], lhs[3]),
                                               _choices((d2, "c"), cont[d2], lhs[4])):
                    key = frozenset().union(*parts) | {("comp", d1), ("comp", d2)}
                    occ.add(key | {("first", d1)} if role else key)
    elif kind == W.NESTED:
        for g in alive:
            if g == 0 or label[g] != grand[j]:
                continue
            q = parent[g]
            if q == 0 or label[q] != ch or label[parent[q]] != lab:
                continue
            a = parent[q]
            for parts in itertools.product(_choices((a, "c"), cont[a], lhs[0]),
                                           _choices((q, "w"), wrap[q], lhs[1]),
                                           _choices((q, "c"), cont[q], lhs[2]),
                                           _choices((g, "w"), wrap[g], lhs[3]),
                                           _choices((g, "c"), cont[g], lhs[4])):
                occ.add(frozenset().union(*parts) | {("comp", q), ("comp", g)})
    else:
        raise ValueError("brute force covers FUSION, PAIR and NESTED")
    return len(occ)


def _general_rules():
    F, N, P = W.FUSION, W.NESTED, W.PAIR
    return [
        W.RuleSpec(P, 0, 1, lhs_child={0: 1}, rhs_child2={0: 1}),                # transport d1 -> d2
        W.RuleSpec(P, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1},
                   rhs_wrap={1: 1}, rhs_wrap2={1: 1}),                           # symmetric rewrite
        W.RuleSpec(P, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1},
                   rhs_wrap={1: 1}, rhs_wrap2={0: 1}),                           # same lhs, one-sided rhs
        W.RuleSpec(P, 1, 2, lhs_ctx={1: 1}, lhs_child={0: 1}, lhs_child2={1: 1}, rhs_ctx={0: 1}),
        W.RuleSpec(F, 0, 1),                                                     # empty patterns
        W.RuleSpec(F, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}),                  # identical patterns
        W.RuleSpec(F, 0, 1, lhs_wrap={0: 1}, lhs_child2={1: 1}),                 # different patterns
        W.RuleSpec(F, 0, 1, lhs_ctx={1: 1}, lhs_child={0: 2}, lhs_child2={0: 1}),  # parent pattern too
        W.RuleSpec(F, 1, 2, lhs_wrap={1: 1}, lhs_wrap2={1: 1}),                  # inside label-1 compartments
        W.RuleSpec(N, 0, 1, grand_label=2, lhs_child2={0: 1}),
        W.RuleSpec(N, 0, 1, grand_label=2, lhs_ctx={1: 1}, lhs_wrap={0: 1}, lhs_wrap2={1: 1}, lhs_child2={0: 2}),
        W.RuleSpec(N, 1, 2, grand_label=1, lhs_child={1: 1}, lhs_child2={0: 1}),
    ]


def _random_term(rng, model, n_comp):
    """Slot image: the root plus n_comp compartments with random labels 1..2,
    each placed under the root or an earlier compartment, 0-2 atoms per
    species in every wrap and content."""
    S, C = model.n_species, model.max_compartments
    img = W.empty_slot_image(model)
    for c in range(1, n_comp + 1):
        img[c, 0] = 1
        img[c, 1] = int(rng.integers(1, 3))
        img[c, 2] = int(rng.integers(0, c))
        img[c, 3:3 + S] = rng.integers(0, 3, S)
    img[:n_comp + 1, 3 + S:3 + 2 * S] = rng.integers(0, 3, (n_comp + 1, S))
    img[0, 3:3 + S] = 0
    return img


def test_brute_force_counts_fusion_pair_and_nested():
    model = W.cwc_model(2, 3, 8, _general_rules())
    rng = np.random.default_rng(2024)
    nonzero = np.zeros(model.n_rules, int)
    for trial in range(300):
        img = _random_term(rng, model, int(rng.integers(3, 8)))
        H = oracle.rule_totals(model, img)
        for j in range(model.n_rules):
            want = brute_force_count(model, img, j)
            assert H[j] == want, (trial, j, H[j], want)
            nonzero[j] += want > 0
    print("terms with occurrences, per rule:", nonzero.tolist())
    assert np.all(nonzero >= 8)   # the random terms exercise every rule


def test_fusion_counts_unordered_pairs_only_for_identical_patterns():
    """Three label-1 children of the top with wraps (a, b) = (1,0), (1,1), (2,1)."""
    rules = [W.RuleSpec(W.FUSION, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}),
             W.RuleSpec(W.FUSION, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={1: 1})]
    model = W.cwc_model(2, 2, 4, rules)
    img = W.empty_slot_image(model)
    wraps = {1: (1, 0), 2: (1, 1), 3: (2, 1)}
    for c, (a, b) in wraps.items():
        img[c, :3] = [1, 1, 0]
        img[c, 3:5] = [a, b]
    H = oracle.rule_totals(model, img)
    a = {c: v[0] for c, v in wraps.items()}
    b = {c: v[1] for c, v in wraps.items()}
    pairs = [(x, y) for x in wraps for y in wraps if x != y]
    assert H[0] == sum(a[x] * a[y] for x, y in pairs) // 2       # unordered
    assert H[1] == sum(a[x] * b[y] for x, y in pairs)            # ordered
    assert [H[j] for j in range(2)] == [brute_force_count(model, img, j) for j in range(2)]


# ----------------------------------------------------------------------------
# Laws
# ----------------------------------------------------------------------------

def _run(model, img, rates, grid, R, seed, **kw):
    b = W.Batch(model, np.atleast_2d(np.asarray(rates, np.float64)), img[None].astype(np.int32),
                np.asarray(grid, np.float64), R, seed)
    return oracle.simulate(b, threads=8, **kw)


def _chi2(samples, pmf):
    K = len(pmf)
    obs = np.bincount(samples, minlength=K)[:K].astype(np.float64)
    exp = np.asarray(pmf) * len(samples)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    if len(e) < 2:                 # a point mass: every sample must sit on it
        return 1.0 if obs[~keep].sum() == 0 else 0.0
    e *= o.sum() / e.sum()
    return float(stats.chi2.sf(((o - e) ** 2 / e).sum(), len(e) - 1))


def test_fusion_of_empty_compartments_is_kingmans_coalescent():
    """m label-1 compartments in the top, one FUSION rule with empty patterns
    at rate k: n -> n-1 at rate k n (n-1) / 2.  The CME of this pure-death
    chain on {1..m} gives the law of the number alive at each grid time; the
    atoms inside (one per compartment) are conserved."""
    m, k = 6, 0.7
    model = W.cwc_model(1, 2, m + 1, [W.RuleSpec(W.FUSION, 0, 1)])
    img = W.empty_slot_image(model)
    for c in range(1, m + 1):
        img[c, :3] = [1, 1, 0]
        img[c, 3 + 1] = 1
    grid = np.array([0.0, 0.1, 0.3, 0.8, 2.0])
    res = _run(model, img, [k], grid, 20000, 41)
    st = res["states"]
    # observables: top content, label-1 content, label-1 wrap, alive top, alive label 1
    assert np.all(st[:, :, 1] == m)                  # content conserved
    alive = st[:, :, 4]
    Q = np.zeros((m + 1, m + 1))
    for n in range(2, m + 1):
        Q[n, n - 1] = k * n * (n - 1) / 2
        Q[n, n] = -Q[n, n - 1]
    p0 = np.zeros(m + 1)
    p0[m] = 1.0
    for g, t in enumerate(grid):
        pt = p0 @ linalg.expm(Q * t)
        assert _chi2(alive[:, g], pt) > P_MIN, (t, np.bincount(alive[:, g]), pt)
    # absorbed exactly when one compartment is left (no pair to fuse)
    assert np.array_equal(res["status"] == oracle.ST_ABSORBED, alive[:, -1] == 1)
    assert np.all(np.isin(res["status"], [oracle.ST_OK, oracle.ST_ABSORBED]))


def test_fusion_merges_wraps_and_contents_and_moves_children():
    """Two label-1 compartments with wraps/contents and one label-2 child each
    fuse (rule 0), then a NESTED rule drains the grandchildren's atoms to the
    top: the merged compartment must hold both wraps and contents minus the
    matched atoms plus the rule's own, and both grandchildren under it."""
    rules = [W.RuleSpec(W.FUSION, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_child={1: 3}),
             W.RuleSpec(W.NESTED, 0, 1, grand_label=2, lhs_child2={0: 1}, rhs_ctx={0: 1})]
    model = W.cwc_model(2, 3, 6, rules)
    img = W.empty_slot_image(model)
    img[1, :5] = [1, 1, 0, 2, 0]           # wrap: 2 a
    img[1, 5:7] = [4, 0]                   # content: 4 a
    img[3, :5] = [1, 1, 0, 1, 5]           # wrap: 1 a, 5 b
    img[3, 5:7] = [0, 7]
    img[2, :3] = [1, 2, 1]                 # grandchildren, one under each
    img[2, 5] = 3
    img[4, :3] = [1, 2, 3]
    img[4, 5] = 2
    # fusion first (rate 1e6), then drainage
    res = _run(model, img, [1e6, 1.0], [0.0, 1e-3, 100.0], 64, 3, log_cap=8)
    assert np.all(res["log_rule"][:, 0] == 0)
    assert np.all(res["log_slot"][:, 0] == (1 | (3 << 16)))      # the unordered pair (1, 3)
    st = res["states"]
    S, L = 2, 3
    # after the fusion: one label-1 compartment, wrap a = 2 - 1 + 1 - 1 = 1, b = 5 + 1, content a 4, b 7 + 3
    at = st[:, 1]
    assert np.all(at[:, L * S + (L - 1) * S + 1] == 1)          # alive label 1
    assert np.all(at[:, L * S + 0 * S + 0] == 1) and np.all(at[:, L * S + 0 * S + 1] == 6)   # wrap totals
    assert np.all(at[:, 1 * S + 0] == 4) and np.all(at[:, 1 * S + 1] == 10)                 # content totals
    # in the end the 5 grandchild atoms sit in the top, both grandchildren still alive
    end = st[:, -1]
    assert np.all(end[:, 0] == 5) and np.all(end[:, 2 * S + 0] == 0)
    assert np.all(end[:, L * S + (L - 1) * S + 2] == 2)
    assert np.all(res["status"] == oracle.ST_ABSORBED)


def test_nested_transport_from_grandchildren_is_binomial():
    """Top > label-1 > label-2 (two such grandchildren, 20 atoms each) and a
    decoy label-2 compartment directly in the top: a NESTED rule moves one
    atom from a grandchild's content to the top at rate k per atom, so the top
    holds Bin(40, 1 - e^-kt) atoms and the decoy keeps its own."""
    k = 0.6
    model = W.cwc_model(1, 3, 7, [W.RuleSpec(W.NESTED, 0, 1, grand_label=2, lhs_child2={0: 1}, rhs_ctx={0: 1})])
    img = W.empty_slot_image(model)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 2, 1]
    img[2, 4] = 20
    img[3, :3] = [1, 1, 0]
    img[4, :3] = [1, 2, 3]
    img[4, 4] = 20
    img[5, :3] = [1, 2, 0]                 # decoy: label 2 directly in the top
    img[5, 4] = 9
    grid = np.array([0.0, 0.5, 1.5, 4.0])
    res = _run(model, img, [k], grid, 20000, 12)
    st = res["states"]
    assert np.all(st[:, :, 0] + st[:, :, 2] == 49)              # top + label-2 content
    for g, t in enumerate(grid):
        pmf = stats.binom.pmf(np.arange(41), 40, 1 - math.exp(-k * t))
        assert _chi2(st[:, g, 0], pmf) > P_MIN
    assert np.all(st[:, -1, 2] >= 9)                            # the decoy is never drained


def test_pair_counts_unordered_pairs_only_for_fully_symmetric_rules():
    """Three label-1 children of the top with wraps (a, b) = (1,0), (1,1), (2,1):
    identical left- and right-hand patterns count unordered pairs; identical
    left-hand but different right-hand patterns count ordered pairs (the two
    roles give different terms); different left-hand patterns count ordered
    pairs."""
    rules = [W.RuleSpec(W.PAIR, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_wrap2={1: 1}),
             W.RuleSpec(W.PAIR, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_wrap2={0: 1}),
             W.RuleSpec(W.PAIR, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={1: 1})]
    model = W.cwc_model(2, 2, 4, rules)
    img = W.empty_slot_image(model)
    wraps = {1: (1, 0), 2: (1, 1), 3: (2, 1)}
    for c, (a, b) in wraps.items():
        img[c, :3] = [1, 1, 0]
        img[c, 3:5] = [a, b]
    H = oracle.rule_totals(model, img)
    a = {c: v[0] for c, v in wraps.items()}
    b = {c: v[1] for c, v in wraps.items()}
    pairs = [(x, y) for x in wraps for y in wraps if x != y]
    assert H[0] == sum(a[x] * a[y] for x, y in pairs) // 2       # unordered
    assert H[1] == sum(a[x] * a[y] for x, y in pairs)            # ordered
    assert H[2] == sum(a[x] * b[y] for x, y in pairs)            # ordered
    assert [H[j] for j in range(3)] == [brute_force_count(model, img, j) for j in range(3)]


def test_pair_rewrites_both_compartments_in_place():
    """One event of a PAIR rule: the chosen (d1, d2) loses the matched atoms,
    gains its own right-hand atoms, and both compartments stay alive with
    their labels and parents; the parent content changes by row 0."""
    rules = [W.RuleSpec(W.PAIR, 0, 1, lhs_ctx={2: 1}, lhs_child={0: 1}, lhs_wrap2={1: 1},
                        rhs_child={1: 1}, rhs_wrap2={0: 2}, rhs_child2={2: 1})]
    model = W.cwc_model(3, 2, 4, rules)
    S = 3
    img = W.empty_slot_image(model)
    img[0, 3 + S + 2] = 5
    img[1, :3] = [1, 1, 0]
    img[1, 3 + S + 0] = 1          # content a of slot 1
    img[2, :3] = [1, 1, 0]
    img[2, 3 + 1] = 1              # wrap b of slot 2
    # the only occurrence: first = slot 1 (has a), second = slot 2 (wrap b)
    assert oracle.rule_totals(model, img)[0] == 5
    res = _run(model, img, [1.0], np.array([0.0, 50.0]), 1, 3, log_cap=4)
    assert res["log_rule"][0, 0] == 0 and res["log_slot"][0, 0] == 1 | (2 << 16)
    st = res["states"][0, 1]                      # observables after the only event
    L = 2
    cont = st[:L * S].reshape(L, S)
    wr = st[L * S:L * S + (L - 1) * S].reshape(L - 1, S)
    alive = st[L * S + (L - 1) * S:]
    assert cont[0].tolist() == [0, 0, 4]          # root lost one c
    assert cont[1].tolist() == [0, 1, 1]          # slot 1: a -> b; slot 2 gained c
    assert wr[0].tolist() == [2, 0, 0]            # slot 2's wrap b -> 2 a
    assert alive.tolist() == [1, 2]


def test_pair_transport_between_siblings_is_the_ehrenfest_model():
    """Two label-1 compartments, N atoms a in the first; PAIR (a X)(Y) -> (X)(a Y)
    at rate k per atom, in both directions (ordered pairs): each atom flips
    independently at rate k, so the first compartment holds
    Bin(N, (1 + e^-2kt) / 2)."""
    N, k = 12, 0.7
    model = W.cwc_model(1, 2, 3, [W.RuleSpec(W.PAIR, 0, 1, lhs_child={0: 1}, rhs_child2={0: 1})])
    img = W.empty_slot_image(model)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 1, 0]
    img[1, 3 + 1] = N
    grid = np.array([0.0, 0.2, 0.6, 1.5, 4.0])
    R = 20000
    b = W.Batch(model, np.array([[k]]), img[None].astype(np.int32), grid, R, 41)
    res = oracle.simulate(b, threads=8, log_cap=128)
    ls = res["log_slot"][res["log_rule"] >= 0]
    assert set(np.unique(ls).tolist()) == {1 | (2 << 16), 2 | (1 << 16)}
    # the observables hold label totals only (always N at label 1), so slot
    # 1's count is rebuilt from the event log: each event moves one atom
    lt, ev = res["log_t"], res["events"]
    assert np.all(ev < 128)
    n1 = np.full((R, len(grid)), N)
    for r in range(R):
        cnt = N
        e = 0
        for g, t in enumerate(grid):
            while e < ev[r] and lt[r, e] < t:
                cnt += -1 if res["log_slot"][r, e] == (1 | (2 << 16)) else 1
                e += 1
            n1[r, g] = cnt
    for g, t in enumerate(grid):
        p = (1 + math.exp(-2 * k * t)) / 2
        pmf = stats.binom.pmf(np.arange(N + 1), N, p)
        assert _chi2(n1[:, g], pmf) > P_MIN, (t, n1[:, g].mean(), N * p)
