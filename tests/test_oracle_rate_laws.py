"""Pins of the oracle's non-mass-action rate law (Michaelis-Menten).

Sec. 2.2 takes the rate of a rule as its kinetic constant times the number of
reactant combinations (mass action) and notes that "more flexible approaches"
are used too.  The oracle's reading: a flat-network reaction may have the
Michaelis-Menten rate a = k n_E n_S / (K + n_S) (substrate S, enzyme E, the
Michaelis constant K in molecules), evaluated as RN(RN(n_E n_S) / RN(K +
n_S)) times k.  Since a = k h still holds, the likelihood-ratio score keeps
its form.  The pins:

* closed forms and exact values: n_S = K gives h = n_E / 2 exactly; h is
  within the three roundings of the exact rational n_E n_S / (K + n_S); the
  substrate index matters (swapping substrate and enzyme changes h);
* laws: an enzyme-catalysed conversion is a pure-death chain with rates
  k n_E n / (K + n), and a Michaelis-Menten conversion with a mass-action
  back reaction is a birth-death chain on a finite state space: chemical
  master equation via the matrix exponential, chi-square at fixed seeds;
* the sensitivity: LR gradient against central finite differences with
  common random numbers, within 3 standard errors.
"""
import math
from fractions import Fraction

import numpy as np
from scipy import linalg, stats

import oracle
from paper_1010_2438_gb300 import workloads as W

from test_oracle_sensitivity import check_z, fd_crn, lr_per_grid_point

P_MIN = 1e-4


def _mm_model(K=10.0, enzyme=True):
    """S (0) -> P (1) catalysed by E (2) with Michaelis-Menten kinetics."""
    reac = ({0: 1, 2: 1}, {1: 1, 2: 1}) if enzyme else ({0: 1}, {1: 1})
    return W.flat_model(3, [reac], michaelis_menten={0: (0, K)})


def test_michaelis_menten_value_closed_forms():
    m = _mm_model(K=12.0)
    assert oracle.rule_h(m, [12, 0, 5])[0] == 2.5            # n_S = K: h = n_E / 2
    assert oracle.rule_h(m, [0, 7, 5])[0] == 0.0              # no substrate
    assert oracle.rule_h(m, [9, 0, 0])[0] == 0.0              # no enzyme
    m1 = _mm_model(K=3.0, enzyme=False)
    assert oracle.rule_h(m1, [3, 0, 0])[0] == 0.5
    # the substrate index is part of the law: E and S swapped give another value
    ms = W.flat_model(3, [({0: 1, 2: 1}, {1: 1, 2: 1})], michaelis_menten={0: (2, 12.0)})
    assert oracle.rule_h(ms, [12, 0, 5])[0] == 60.0 / 17.0 != oracle.rule_h(m, [12, 0, 5])[0]


def test_michaelis_menten_value_within_three_roundings_of_the_exact_rational():
    rng = np.random.default_rng(3)
    for K in (0.37, 1.0, 12.5, 1e3, 7.7e6):
        m = _mm_model(K=K)
        for _ in range(200):
            nS, nE = int(rng.integers(0, 2 ** 31 - 1)), int(rng.integers(0, 2 ** 31 - 1))
            got = oracle.rule_h(m, [nS, 0, nE])[0]
            exact = Fraction(nE * nS) / (Fraction(K) + nS)
            if exact == 0:
                assert got == 0.0
                continue
            rel = abs(Fraction(got) - exact) / exact
            assert rel <= Fraction(301, 100 * 2 ** 53), (K, nS, nE, float(rel))   # 3 roundings


def _cme(Q, p0, grid):
    return [p0 @ linalg.expm(Q * t) for t in grid]


def _chi2(samples, pmf):
    K = len(pmf)
    obs = np.bincount(samples, minlength=K)[:K].astype(np.float64)
    exp = np.asarray(pmf) * len(samples)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    if len(e) < 2:
        return 1.0 if obs[~keep].sum() == 0 else 0.0
    e *= o.sum() / e.sum()
    return float(stats.chi2.sf(((o - e) ** 2 / e).sum(), len(e) - 1))


def test_enzyme_catalysed_conversion_follows_its_master_equation():
    """S + E -> P + E at k n_E n_S / (K + n_S), E = 4 fixed: S is a pure-death
    chain with rates lambda_n = 4 k n / (K + n); half-saturated at n = K."""
    k, K, n0, nE = 1.3, 10.0, 40, 4
    m = _mm_model(K=K)
    grid = np.array([0.0, 1.0, 3.0, 6.0, 12.0])
    b = W.Batch(m, np.array([[k]]), np.array([[n0, 0, nE]], np.int32), grid, 20000, 17)
    res = oracle.simulate(b, threads=8)
    st = res["states"]
    assert np.all(st[:, :, 0] + st[:, :, 1] == n0) and np.all(st[:, :, 2] == nE)
    Q = np.zeros((n0 + 1, n0 + 1))
    for n in range(1, n0 + 1):
        Q[n, n - 1] = nE * k * n / (K + n)
        Q[n, n] = -Q[n, n - 1]
    p0 = np.zeros(n0 + 1)
    p0[n0] = 1.0
    for g, pt in enumerate(_cme(Q, p0, grid)):
        assert _chi2(st[:, g, 0], pt) > P_MIN, (grid[g], st[:, g, 0].mean())


def test_michaelis_menten_with_mass_action_back_reaction():
    """S -> P (Michaelis-Menten, no enzyme: k1 n_S / (K + n_S)) and P -> S
    (mass action k2 n_P), N = 30 molecules: a birth-death chain on n_S."""
    k1, K, k2, N = 6.0, 5.0, 0.4, 30
    m = W.flat_model(2, [({0: 1}, {1: 1}), ({1: 1}, {0: 1})], michaelis_menten={0: (0, K)})
    grid = np.array([0.0, 0.5, 2.0, 8.0])
    b = W.Batch(m, np.array([[k1, k2]]), np.array([[N, 0]], np.int32), grid, 20000, 23)
    st = oracle.simulate(b, threads=8)["states"]
    assert np.all(st.sum(axis=2) == N)
    Q = np.zeros((N + 1, N + 1))
    for n in range(N + 1):
        if n > 0:
            Q[n, n - 1] = k1 * n / (K + n)
        if n < N:
            Q[n, n + 1] = k2 * (N - n)
        Q[n, n] = -Q[n].sum()
    p0 = np.zeros(N + 1)
    p0[N] = 1.0
    for g, pt in enumerate(_cme(Q, p0, grid)):
        assert _chi2(st[:, g, 0], pt) > P_MIN, (grid[g], st[:, g, 0].mean())


def test_michaelis_menten_lr_gradient_vs_central_fd():
    """d E[X(g)] / d k for the reversible system above (both rates), LR against
    central differences with common random numbers."""
    m = W.flat_model(2, [({0: 1}, {1: 1}), ({1: 1}, {0: 1})], michaelis_menten={0: (0, 5.0)})
    b = W.Batch(m, np.array([[6.0, 0.4]]), np.array([[30, 0]], np.int32), np.array([0.5, 2.0]), 20000, 29)
    est, se = lr_per_grid_point(b)
    z = []
    for j in range(2):
        fd, fse = fd_crn(b, j)
        z += list(((est[:, :, j] - fd) / np.sqrt(se[:, :, j] ** 2 + fse ** 2)).ravel())
    check_z(z)
