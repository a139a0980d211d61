"""Pins of the oracle's simulation against laws the mathematics fixes.

Gillespie's direct method (Sec. 2.2, two steps: tau ~ Exp(r), reaction i with
probability r_i / r) samples the continuous-time Markov chain exactly, so the
distribution of X(t) must match:
  * closed forms (birth-death: Poisson / binomial mixture; isomerisation:
    binomial mixture; CWC transport and create/dissolve: binomial);
  * the chemical master equation p(t) = expm(Q^T t) p0 on small state spaces.
All seeds are fixed, so every test is deterministic; thresholds are p > 1e-4.
"""
import math

import numpy as np
import pytest
from scipy import linalg, stats

import oracle
from paper_1010_2438_gb300 import workloads as W

P_MIN = 1e-4


def chi2_pvalue(samples, pmf, min_expected=5.0):
    """Chi-square goodness of fit of integer samples against pmf (array over 0..K)."""
    n = len(samples)
    K = len(pmf)
    obs = np.bincount(np.clip(samples, 0, K - 1), minlength=K).astype(np.float64)[:K]
    exp = np.asarray(pmf, np.float64) * n
    # merge bins from both ends until every bin has enough expected mass
    bins_o, bins_e = [], []
    acc_o = acc_e = 0.0
    for o, e in zip(obs, exp):
        acc_o += o
        acc_e += e
        if acc_e >= min_expected:
            bins_o.append(acc_o)
            bins_e.append(acc_e)
            acc_o = acc_e = 0.0
    if bins_e:
        bins_o[-1] += acc_o
        bins_e[-1] += acc_e
    bins_o = np.array(bins_o)
    bins_e = np.array(bins_e)
    bins_e *= bins_o.sum() / bins_e.sum()
    if len(bins_e) < 2:
        return 1.0
    chi2 = float(((bins_o - bins_e) ** 2 / bins_e).sum())
    return float(stats.chi2.sf(chi2, len(bins_e) - 1))


def run(model, rates, init, grid, R, seed, **kw):
    b = W.Batch(model, np.atleast_2d(np.asarray(rates, np.float64)), np.asarray(init, np.int32),
                np.asarray(grid, np.float64), R, seed)
    return oracle.simulate(b, threads=8, **kw)


# ----------------------------------------------------------------------------
# Birth-death 0 -> A (k1), A -> 0 (k2)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("x0", [0, 25])
def test_birth_death_transient_law(x0):
    k1, k2 = 12.0, 0.8
    grid = np.array([0.0, 0.3, 1.0, 2.5, 6.0])
    res = run(W.birth_death(), [k1, k2], [[x0]], grid, 20000, 1234 + x0)
    assert np.all(res["status"] == oracle.ST_OK)
    for g, t in enumerate(grid):
        x = res["states"][:, g, 0]
        q = math.exp(-k2 * t)
        lam = k1 / k2 * (1 - q)
        K = 120
        pmf = np.convolve(stats.binom.pmf(np.arange(K), x0, q), stats.poisson.pmf(np.arange(K), lam))[:K]
        assert chi2_pvalue(x, pmf) > P_MIN, (t, x.mean(), x0 * q + lam)


def test_birth_death_stationary_poisson():
    k1, k2 = 30.0, 1.5
    res = run(W.birth_death(), [k1, k2], [[0]], [40.0], 20000, 99)
    x = res["states"][:, 0, 0]
    pmf = stats.poisson.pmf(np.arange(100), k1 / k2)
    assert chi2_pvalue(x, pmf) > P_MIN


# ----------------------------------------------------------------------------
# Isomerisation A -> B (kf), B -> A (kb): A(t) binomial mixture, A + B conserved
# ----------------------------------------------------------------------------

def test_isomerisation_binomial_mixture_and_conservation():
    kf, kb = 1.3, 0.6
    A0, B0 = 30, 10
    grid = np.array([0.0, 0.2, 0.7, 1.5, 5.0])
    res = run(W.isomerisation(), [kf, kb], [[A0, B0]], grid, 20000, 77)
    st = res["states"]
    assert np.all(st.sum(axis=2) == A0 + B0)
    pinf = kb / (kf + kb)
    for g, t in enumerate(grid):
        e = math.exp(-(kf + kb) * t)
        pA = pinf + (1 - pinf) * e        # an A molecule is an A at time t
        pB = pinf * (1 - e)               # a B molecule has become an A
        K = A0 + B0 + 1
        pmf = np.convolve(stats.binom.pmf(np.arange(K), A0, pA), stats.binom.pmf(np.arange(K), B0, pB))[:K]
        assert chi2_pvalue(st[:, g, 0], pmf) > P_MIN


# ----------------------------------------------------------------------------
# Chemical master equation via matrix exponential
# ----------------------------------------------------------------------------

def cme_check(model, rates, x0, states_of, index_of, n_states, propensities, grid, R, seed, obs):
    """Build Q from the propensity list and compare the oracle's histogram of obs(X)."""
    Q = np.zeros((n_states, n_states))
    for i in range(n_states):
        x = states_of(i)
        for a, dx in propensities(x):
            if a > 0:
                jdx = index_of(tuple(np.add(x, dx)))
                Q[i, jdx] += a
                Q[i, i] -= a
    p0 = np.zeros(n_states)
    p0[index_of(tuple(x0))] = 1.0
    res = run(model, rates, [x0], grid, R, seed)
    for g, t in enumerate(grid):
        pt = p0 @ linalg.expm(Q * t)
        pmf = np.zeros(n_states)
        for i in range(n_states):
            pmf[obs(states_of(i))] += pt[i]
        samples = np.array([obs(s) for s in res["states"][:, g]])
        assert chi2_pvalue(samples, pmf) > P_MIN, t


def test_dimerisation_cme():
    """2A -> B (k1 C(A,2)), B -> 2A (k2 B); A + 2B = N."""
    k1, k2, N = 0.15, 1.0, 24
    nB = N // 2 + 1
    cme_check(
        W.dimerisation(), [k1, k2], [N, 0],
        states_of=lambda i: (N - 2 * i, i), index_of=lambda x: x[1], n_states=nB,
        propensities=lambda x: [(k1 * x[0] * (x[0] - 1) / 2, (-2, 1)), (k2 * x[1], (2, -1))],
        grid=np.array([0.05, 0.3, 1.0, 4.0]), R=20000, seed=5, obs=lambda x: x[1])


def test_heterodimer_cme():
    """A + B -> C (k1 A B), C -> A + B (k2 C)."""
    k1, k2, A0, B0 = 0.2, 0.7, 12, 9
    cme_check(
        W.heterodimer(), [k1, k2], [A0, B0, 0],
        states_of=lambda i: (A0 - i, B0 - i, i), index_of=lambda x: x[2], n_states=B0 + 1,
        propensities=lambda x: [(k1 * x[0] * x[1], (-1, -1, 1)), (k2 * x[2], (1, 1, -1))],
        grid=np.array([0.05, 0.4, 1.5, 5.0]), R=20000, seed=6, obs=lambda x: x[2])


# ----------------------------------------------------------------------------
# CWC laws: per-child transport; create / dissolve with a conserved token
# ----------------------------------------------------------------------------

def test_cwc_transport_two_children_binomial():
    """Each root molecule enters either child at rate k_in and leaves at k_out:
    root count ~ Bin(N, p(t)), p = p_inf + (1 - p_inf) e^{-(2 k_in + k_out) t}."""
    k_in, k_out, N = 0.4, 1.1, 40
    rules = [W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_ctx={0: 1}, rhs_child={0: 1}),
             W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_child={0: 1}, rhs_ctx={0: 1})]
    model = W.cwc_model(1, 2, 3, rules)
    img = W.empty_slot_image(model)
    img[0, 4] = N
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 1, 0]
    grid = np.array([0.0, 0.2, 0.6, 1.5, 6.0])
    res = run(model, [k_in, k_out], img[None], grid, 20000, 8)
    st = res["states"]
    # observables: [top A, label-1 content A, label-1 wrap A, alive top, alive label 1]
    assert np.all(st[:, :, 0] + st[:, :, 1] == N)
    assert np.all(st[:, :, 4] == 2)
    pinf = k_out / (2 * k_in + k_out)
    for g, t in enumerate(grid):
        p = pinf + (1 - pinf) * math.exp(-(2 * k_in + k_out) * t)
        assert chi2_pvalue(st[:, g, 0], stats.binom.pmf(np.arange(N + 1), N, p)) > P_MIN


def test_cwc_create_dissolve_token_law():
    """CREATE top: M X -> X (M | )^1 at k_c per free token; DISSOLVE of each
    label-1 compartment at k_d releases its wrap token: #compartments ~ Bin(m, q(t))."""
    k_c, k_d, m = 0.9, 0.5, 12
    rules = [W.RuleSpec(W.CREATE, 0, 1, lhs_ctx={0: 1}, rhs_wrap={0: 1}),
             W.RuleSpec(W.DISSOLVE, 0, 1)]
    model = W.cwc_model(1, 2, m + 1, rules)
    img = W.empty_slot_image(model)
    img[0, 4] = m
    grid = np.array([0.0, 0.3, 1.0, 3.0, 10.0])
    res = run(model, [k_c, k_d], img[None], grid, 20000, 9)
    st = res["states"]
    assert np.all(res["status"] == oracle.ST_OK)
    # tokens are conserved: free in the top content + held in label-1 wraps
    assert np.all(st[:, :, 0] + st[:, :, 2] == m)
    # alive label-1 compartments == tokens held in wraps
    assert np.all(st[:, :, 4] == st[:, :, 2])
    for g, t in enumerate(grid):
        q = k_c / (k_c + k_d) * (1 - math.exp(-(k_c + k_d) * t))
        assert chi2_pvalue(st[:, g, 4], stats.binom.pmf(np.arange(m + 1), m, q)) > P_MIN


def test_cwc_dissolve_reparents_children():
    """Dissolving a label-1 compartment moves its label-2 child to the top level,
    where a top <- label-2 transport rule can then drain it."""
    rules = [W.RuleSpec(W.DISSOLVE, 0, 1),
             W.RuleSpec(W.PARENT_CHILD, 0, 2, lhs_child={0: 1}, rhs_ctx={0: 1})]
    model = W.cwc_model(1, 3, 3, rules)
    img = W.empty_slot_image(model)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 2, 1]
    img[2, 4] = 5
    res = run(model, [1.0, 1.0], img[None], [0.0, 200.0], 64, 10, log_cap=8)
    st = res["states"]
    O = model.n_observables  # 3 + 2 + 3
    assert O == 8
    assert np.all(st[:, 0, 2] == 5)                    # label-2 content at t = 0
    assert np.all(st[:, -1, 0] == 5)                   # all drained into the top
    assert np.all(st[:, -1, 5:] == [1, 0, 1])          # alive: top, no label 1, label 2
    assert np.all(res["log_rule"][:, 0] == 0)          # the dissolve must come first
    assert np.all(res["events"] == 6)
    assert np.all(res["status"] == oracle.ST_ABSORBED)


def test_cwc_capacity_status():
    rules = [W.RuleSpec(W.CREATE, 0, 1, lhs_ctx={0: 1})]
    model = W.cwc_model(1, 2, 3, rules)
    img = W.empty_slot_image(model)
    img[0, 4] = 10
    res = run(model, [1.0], img[None], [0.0, 1e6], 4, 11)
    assert np.all(res["status"] == oracle.ST_CAPACITY)
    assert np.all(res["events"] == 2)
    assert np.all(res["states"][:, -1, 0] == 8)


# ----------------------------------------------------------------------------
# Invariants and statuses
# ----------------------------------------------------------------------------

def test_conserving_network_invariant_and_time_order():
    b = W.flat8x12(R=16)          # no inflow/outflow: molecule count conserved
    res = oracle.simulate(b, log_cap=20000, threads=8)
    tot = res["states"].sum(axis=2)
    assert np.all(tot == tot[:, :1])
    lt = res["log_t"]
    for q in range(16):
        n = min(res["events"][q], 20000)
        assert np.all(np.diff(lt[q, :n]) >= 0)
        assert lt[q, n - 1] <= b.grid[-1]
        assert res["final_t"][q] == lt[q, n - 1]


def test_replaying_event_log_reproduces_states():
    """Applying the logged reactions in order to x0 gives the grid states
    (state at g = state after all events with time <= g)."""
    b = W.flat8x12(R=4)
    res = oracle.simulate(b, log_cap=20000)
    delta = (b.model.rhs[:, 0] - b.model.lhs[:, 0]).astype(np.int64)
    for q in range(4):
        n = res["events"][q]
        x = b.init[0].astype(np.int64).copy()
        k = 0
        for g, t in enumerate(b.grid):
            while k < n and res["log_t"][q, k] <= t:
                x += delta[res["log_rule"][q, k]]
                k += 1
            assert np.array_equal(res["states"][q, g], x)


def test_event_limit_and_absorbed():
    b = W.flat8x12(R=3)
    res = oracle.simulate(b, max_events=50)
    assert np.all(res["status"] == oracle.ST_EVENT_LIMIT)
    assert np.all(res["events"] == 50)
    r0 = oracle.simulate(b, max_events=0)
    assert np.all(r0["events"] == 0)
    assert np.all(r0["states"] == b.init[0])
    # pure death is absorbed at zero
    m = W.flat_model(1, [({0: 1}, {})])
    bb = W.Batch(m, np.array([[2.0]]), np.array([[30]], np.int32), np.array([0.0, 100.0]), 8, 3)
    r = oracle.simulate(bb)
    assert np.all(r["status"] == oracle.ST_ABSORBED)
    assert np.all(r["events"] == 30)
    assert np.all(r["states"][:, -1, 0] == 0)


def test_bad_input_and_overflow_statuses():
    m = W.birth_death()
    grid = np.array([0.0, 1.0])
    for rates, grid_, init in (([-1.0, 1.0], grid, [[3]]), ([1.0, np.inf], grid, [[3]]),
                               ([1.0, 1.0], np.array([0.0, 0.0]), [[3]]),
                               ([1.0, 1.0], np.array([-1.0, 1.0]), [[3]]),
                               ([1.0, 1.0], grid, [[-4]])):
        b = W.Batch(m, np.array([rates]), np.array(init, np.int32), grid_, 2, 1)
        r = oracle.simulate(b)
        assert np.all(r["status"] == oracle.ST_BAD_INPUT)
        assert np.all(r["events"] == 0)
    # counts may not exceed INT32_MAX
    b = W.Batch(m, np.array([[1e6, 1e-9]]), np.array([[2 ** 31 - 3]], np.int32), np.array([0.0, 1.0]), 2, 1)
    r = oracle.simulate(b)
    assert np.all(r["status"] == oracle.ST_INT_OVERFLOW)
    assert np.all(r["events"] == 2)
    assert np.all(r["states"][:, -1, 0] == 2 ** 31 - 1)
    # total propensity overflowing to +inf
    b = W.Batch(W.dimerisation(), np.array([[1e300, 1.0]]), np.array([[2 ** 30, 0]], np.int32),
                np.array([0.0, 1.0]), 2, 1)
    r = oracle.simulate(b)
    assert np.all(r["status"] == oracle.ST_PROP_OVERFLOW)


def test_trajectories_are_independent_of_batch_layout():
    """The random stream is keyed by (event, purpose, replica, point): any
    subset or split of trajectories reproduces the same results."""
    b = W.sweep256x256(P=4, R=3)
    full = oracle.simulate(b, states=True, threads=1)
    part = oracle.simulate(b, 5, 9, states=True, threads=2)
    for k in ("states", "events", "hash", "status", "final_t"):
        assert np.array_equal(full[k][5:9], part[k])
