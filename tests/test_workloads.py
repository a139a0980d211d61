"""The synthetic inputs that stand in for the paper's workloads (its E. coli
and Lotka-Volterra models come without parameters): each generator must build
what the input recipe states, deterministically from its seed.  CPU only; the
generators hold no simulation arithmetic."""
import numpy as np
import pytest

from paper_1010_2438_gb300 import workloads as W

FLAT = [
    # name, builder, S, M, inflow/outflow pairs, conversions, bimolecular, x_lo, x_hi
    ("flat8x12", W.flat8x12, 8, 12, 0, 8, 4, 50, 500),
    ("flat32x64", W.flat32x64, 32, 64, 8, 32, 16, 100, 5000),
    ("flat16x24", W.flat16x24, 16, 24, 2, 16, 4, 50, 500),
]


def _orders(model):
    return model.lhs[:, 0, :].sum(axis=1)


def _strongly_connected(S, edges):
    adj = [set() for _ in range(S)]
    radj = [set() for _ in range(S)]
    for a, b in edges:
        adj[a].add(b)
        radj[b].add(a)

    def reach(g):
        seen, stack = {0}, [0]
        while stack:
            for v in g[stack.pop()]:
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        return len(seen) == S
    return reach(adj) and reach(radj)


@pytest.mark.parametrize("name,build,S,M,pairs,n1,n2,x_lo,x_hi", FLAT)
def test_flat_network_composition(name, build, S, M, pairs, n1, n2, x_lo, x_hi):
    b = build(R=4, G=10)
    m = b.model
    assert (m.n_species, m.n_rules, m.n_labels, m.max_compartments) == (S, M, 1, 1)
    assert np.all(m.kind == W.LOCAL) and np.all(m.ctx_label == 0)
    assert np.all(m.lhs[:, 1:, :] == 0) and np.all(m.rhs[:, 1:, :] == 0)
    order = _orders(m)
    prod = m.rhs[:, 0, :].sum(axis=1)
    inflow = [j for j in range(M) if order[j] == 0]
    outflow = [j for j in range(M) if order[j] == 1 and prod[j] == 0]
    assert len(inflow) == pairs and len(outflow) == pairs
    # each inflow species has its outflow, on distinct species
    in_sp = sorted(int(np.argmax(m.rhs[j, 0])) for j in inflow)
    out_sp = sorted(int(np.argmax(m.lhs[j, 0])) for j in outflow)
    assert in_sp == out_sp and len(set(in_sp)) == pairs
    conv = [j for j in range(M) if order[j] == 1 and prod[j] == 1]
    bi = [j for j in range(M) if order[j] == 2]
    assert len(conv) == n1 and len(bi) == n2
    # every reaction but the pairs conserves the molecule count
    for j in conv + bi:
        assert m.lhs[j, 0].sum() == m.rhs[j, 0].sum()
    # stoichiometry 1-2 per species, both bimolecular forms (A + B and 2A)
    assert m.lhs.max() <= 2 and m.rhs.max() <= 2
    assert any(m.lhs[j, 0].max() == 2 for j in bi) and any(m.lhs[j, 0].max() == 1 for j in bi)
    # the conversions contain a cycle through every species: no sink species
    edges = [(int(np.argmax(m.lhs[j, 0])), int(np.argmax(m.rhs[j, 0]))) for j in conv]
    assert all(a != b for a, b in edges)
    assert _strongly_connected(S, edges)


@pytest.mark.parametrize("name,build,S,M,pairs,n1,n2,x_lo,x_hi", FLAT)
def test_flat_rates_counts_and_grid(name, build, S, M, pairs, n1, n2, x_lo, x_hi):
    b = build(R=4, G=10)
    m = b.model
    omega = 0.5 * (x_lo + x_hi)
    order = _orders(m)
    # log-uniform over [1e-3, 1] in concentration units, volume-scaled by omega^(1 - order)
    k = b.rates[0] / omega ** (1.0 - order)
    assert b.rates.shape == (1, M) and np.all(k >= 1e-3 * (1 - 1e-12)) and np.all(k <= 1.0 * (1 + 1e-12))
    assert np.log10(k).max() - np.log10(k).min() > 1.5          # spread over the decades
    assert b.init.shape == (1, S) and b.init.dtype == np.int32
    assert np.all(b.init >= x_lo) and np.all(b.init <= x_hi)
    T = b.grid[-1]
    assert b.grid[0] == 0.0 and T > 0
    assert np.allclose(b.grid, np.arange(10) * T / 9, rtol=0, atol=1e-15 * T)
    assert np.all(np.diff(b.grid) > 0)


@pytest.mark.parametrize("build", [W.flat8x12, W.flat32x64, W.flat16x24, W.cwc3x24, W.sweep256x256])
def test_generators_are_deterministic(build):
    a, b = build(R=2, G=5), build(R=2, G=5)
    for x, y in ((a.rates, b.rates), (a.init, b.init), (a.grid, b.grid), (a.model.lhs, b.model.lhs),
                 (a.model.rhs, b.model.rhs), (a.model.kind, b.model.kind)):
        assert np.array_equal(x, y)
    assert a.seed == b.seed


def test_sweep_rate_vectors():
    base = W.flat32x64(R=2, G=5)
    sw = W.sweep256x256(P=256, R=2, G=5)
    assert sw.rates.shape == (256, 64) and sw.P == 256
    assert np.array_equal(sw.model.lhs, base.model.lhs)
    ratio = np.log10(sw.rates / base.rates[0])
    # common two-decade factor times a per-rate jitter of +-1/4 decade
    assert np.all(ratio >= -1.25 - 1e-12) and np.all(ratio <= 1.25 + 1e-12)
    common = ratio.mean(axis=1)
    assert common.max() - common.min() > 1.6                   # points ~2 decades apart
    assert np.all(ratio.max(axis=1) - ratio.min(axis=1) <= 0.5 + 1e-12)
    assert np.all(ratio.max(axis=1) - ratio.min(axis=1) > 0.2)   # the vectors differ in shape


def test_cwc3x24_rules():
    b = W.cwc3x24(R=2, G=5)
    m = b.model
    assert (m.n_species, m.n_labels, m.max_compartments, m.n_rules) == (24, 4, 64, 48)
    kinds = np.bincount(m.kind, minlength=4)
    assert kinds.tolist() == [24, 12, 6, 6]
    for lab in range(4):
        assert np.sum((m.kind == W.LOCAL) & (m.ctx_label == lab)) == 6
    # containment: top holds labels 1 and 2, label 1 holds label 3
    allowed = {(0, 1), (0, 2), (1, 3)}
    for j in range(m.n_rules):
        if m.kind[j] != W.LOCAL:
            assert (int(m.ctx_label[j]), int(m.child_label[j])) in allowed
    pc = np.where(m.kind == W.PARENT_CHILD)[0]
    into = [j for j in pc if m.lhs[j, 0].sum() == 1 and m.rhs[j, 2].sum() == 1 and m.lhs[j, 1].sum() == 0]
    out = [j for j in pc if m.lhs[j, 2].sum() == 1 and m.rhs[j, 0].sum() == 1]
    wrap = [j for j in pc if m.lhs[j, 1].sum() == 1]
    assert (len(into), len(out), len(wrap)) == (6, 4, 2)
    # the token is touched only by CREATE (parent content -> new wrap) and DISSOLVE (wrap)
    tok = W.CWC_TOKEN
    for j in range(m.n_rules):
        uses = m.lhs[j, :, tok].any() or m.rhs[j, :, tok].any()
        assert uses == (m.kind[j] in (W.CREATE, W.DISSOLVE))
    for j in np.where(m.kind == W.CREATE)[0]:
        assert m.lhs[j, 0, tok] == 1 and m.rhs[j, 1, tok] == 1 and m.rhs[j, 2].sum() == 20
    for j in np.where(m.kind == W.DISSOLVE)[0]:
        assert m.lhs[j, 1, tok] == 1 and m.lhs[j].sum() == 1
    structural = np.isin(m.kind, [W.CREATE, W.DISSOLVE])
    assert np.all(b.rates[0, structural] >= 0.1 * (1 - 1e-12)) and np.all(b.rates[0, structural] <= 1.0)


def test_cwc3x24_initial_term():
    b = W.cwc3x24(R=2, G=5)
    S, tok = 24, W.CWC_TOKEN
    img = b.init[0]
    assert img.shape == (64, W.slot_image_width(S))
    alive = img[:, 0] == 1
    assert alive.sum() == 33 and np.all(alive[:33]) and not alive[33:].any()
    labels, parents = img[:33, 1], img[:33, 2]
    assert labels[0] == 0 and parents[0] == -1
    assert np.sum(labels == 1) == 8 and np.sum(labels == 2) == 8 and np.sum(labels == 3) == 16
    for c in range(1, 33):
        assert labels[parents[c]] == {1: 0, 2: 0, 3: 1}[int(labels[c])]
        assert img[c, 3 + tok] == 1                                 # one token in every wrap
    wrap, content = img[:, 3:3 + S], img[:, 3 + S:]
    assert wrap[:, tok].sum() + content[:, tok].sum() == 63          # so at most 64 compartments
    mol = content[:33, :tok]
    assert np.all(mol >= 10) and np.all(mol <= 200)
    assert np.all(wrap[:33, :tok] == 0)


@pytest.mark.parametrize("n", [2, 4, 32])
def test_lotka_volterra_chain(n):
    b = W.lotka_volterra(n, R=2, G=5)
    m = b.model
    assert m.n_species == n and m.n_rules == n + 1
    assert m.lhs[0, 0, 0] == 1 and m.rhs[0, 0, 0] == 2                # prey birth
    for i in range(n - 1):                                            # S_i + S_(i+1) -> 2 S_(i+1)
        assert m.lhs[i + 1, 0, i] == 1 and m.lhs[i + 1, 0, i + 1] == 1 and m.rhs[i + 1, 0, i + 1] == 2
    assert m.lhs[n, 0, n - 1] == 1 and m.rhs[n].sum() == 0            # last predator death
    assert np.all(b.init == 1000)
    assert b.rates[0, 0] == 10.0 and b.rates[0, -1] == 10.0 and np.all(b.rates[0, 1:-1] == 0.01)


def test_general_pattern_workload_recipe():
    """cwc_general: every rule kind present, FUSION with identical (cells) and
    different (vesicles) patterns, PAIR with ordered (cells) and unordered
    (vesicles) pairs, NESTED with its grandchild label; tokens
    M (cells) and V (vesicles): one in every wrap, conserved by every rule,
    so at most 18 compartments besides the root exist (24 slots)."""
    b = W.cwc_general()
    m = b.model
    assert set(m.kind.tolist()) == set(W.KIND_NAMES)
    lhs5, rhs5, grand = m.rows5()
    for j in range(m.n_rules):
        # token balance of every rule: matched tokens + released = produced
        for tok in (W.GEN_M, W.GEN_V):
            if m.kind[j] == W.DISSOLVE:
                continue                      # releases the whole wrap into the parent
            if m.kind[j] == W.FUSION:
                assert lhs5[j, :, tok].sum() == rhs5[j, :, tok].sum()
            elif m.kind[j] == W.CREATE:
                assert lhs5[j, 0, tok] == rhs5[j, 1, tok]
            else:
                assert lhs5[j, :, tok].sum() == rhs5[j, :, tok].sum()
        if m.kind[j] == W.NESTED:
            assert grand[j] == 2 and m.child_label[j] == 1 and m.ctx_label[j] == 0
    fus = np.nonzero(m.kind == W.FUSION)[0]
    sym = [np.array_equal(lhs5[j, 1:3], lhs5[j, 3:5]) for j in fus]
    assert sorted(sym) == [False, True]
    pair = np.nonzero(m.kind == W.PAIR)[0]
    sym = [np.array_equal(lhs5[j, 1:3], lhs5[j, 3:5]) and np.array_equal(rhs5[j, 1:3], rhs5[j, 3:5]) for j in pair]
    assert sorted(sym) == [False, True]
    img = b.init[0]
    S = m.n_species
    tokens_M = img[:, 3 + W.GEN_M].sum() + img[:, 3 + S + W.GEN_M].sum()
    tokens_V = img[:, 3 + W.GEN_V].sum() + img[:, 3 + S + W.GEN_V].sum()
    assert (tokens_M, tokens_V) == (10, 8)
    assert 1 + tokens_M + tokens_V <= m.max_compartments - 5


def test_michaelis_menten_cascade_recipe():
    """20 stages: species 0 the input kinase, stage i's inactive / active forms
    2i-1 / 2i; rule 2(i-1) activates stage i with enzyme 0 (i = 1) or the
    previous stage's active form, rule 2(i-1)+1 deactivates it without an
    enzyme; every rule Michaelis-Menten with K = 50 on its substrate;
    activation k = 1, deactivation k = 20; each stage conserves its 100
    molecules; P > 1 scales the activation constants by factors in [0.5, 2]."""
    b = W.mm_cascade(stages=20, R=8, P=5)
    m = b.model
    assert (m.n_species, m.n_rules) == (41, 40)
    lhs, rhs = m.lhs[:, 0, :], m.rhs[:, 0, :]
    for i in range(1, 21):
        x, xa, enz = 2 * i - 1, 2 * i, 0 if i == 1 else 2 * (i - 1)
        ja, jd = 2 * (i - 1), 2 * (i - 1) + 1
        assert set(np.nonzero(lhs[ja])[0]) == {x, enz} and m.rate_law[ja] == 1 + x
        assert rhs[ja, xa] == 1 and rhs[ja, enz] == 1 and rhs[ja, x] == 0
        assert set(np.nonzero(lhs[jd])[0]) == {xa} and m.rate_law[jd] == 1 + xa and rhs[jd, x] == 1
        assert (rhs[ja] - lhs[ja]).sum() == 0 and (rhs[jd] - lhs[jd]).sum() == 0
    assert np.all(m.rate_par == 50.0) and np.all((m.lhs[:, 0, :] <= 1))
    assert np.all(b.rates[:, 1::2] == 20.0)
    f = b.rates[:, 0::2]
    assert np.all(f == f[:, :1]) and np.all((f >= 0.5) & (f <= 2.0)) and len(set(f[:, 0])) == 5
    assert b.init[0, 0] == 10 and np.all(b.init[0, 1::2] == 100) and np.all(b.init[0, 2::2] == 0)
    b1 = W.mm_cascade(stages=20, R=8, P=1)
    assert np.all(b1.rates[0, 0::2] == 1.0)
    b2 = W.mm_cascade(stages=20, R=8, P=5)
    assert np.array_equal(b.rates, b2.rates)
