"""Pins of the oracle's replica statistics (mean, variance, 90 % interval)."""
import math

import numpy as np
from scipy import stats

import oracle
from paper_1010_2438_gb300 import workloads as W


def test_z90_is_the_normal_quantile():
    assert abs(oracle.Z90 - stats.norm.ppf(0.95)) <= 2 * np.spacing(oracle.Z90)


def test_variance_matches_library_and_exact_sums():
    rng = np.random.default_rng(7)
    for R in (2, 3, 17, 64):
        st = rng.integers(0, 2 ** 31 - 1, size=(R * 2, 5, 3)).astype(np.int32)
        s, q, var, ci = oracle.replica_stats(st, 2, R)
        x = st.reshape(2, R, 5, 3)
        assert np.array_equal(s.astype(np.int64), x.astype(np.int64).sum(axis=1))
        q_ref = [[[sum(int(v) ** 2 for v in x[p, :, g, o]) for o in range(3)] for g in range(5)] for p in range(2)]
        assert np.array_equal(q, np.array(q_ref, dtype=object))
        ref = x.astype(np.float64).var(axis=1, ddof=1)
        assert np.allclose(var, ref, rtol=1e-12, atol=0)
        assert np.allclose(ci, stats.norm.ppf(0.95) * np.sqrt(ref / R), rtol=1e-12)


def test_single_replica_and_constant_columns():
    st = np.full((4, 2, 2), 7, np.int32)
    _, _, var, ci = oracle.replica_stats(st, 1, 4)
    assert np.all(var == 0.0) and np.all(ci == 0.0)
    _, _, var, ci = oracle.replica_stats(st[:1], 1, 1)
    assert np.all(var == 0.0)


def test_interval_covers_the_birth_death_mean():
    """Coverage of the 90 % interval for the mean of Poisson X(t) (birth-death
    from 0): over 60 independent batches it covers the true mean in about 90 %."""
    k1, k2, t = 6.0, 1.0, 3.0
    mu = k1 / k2 * (1 - math.exp(-k2 * t))
    hits = 0
    for seed in range(60):
        b = W.Batch(W.birth_death(), np.array([[k1, k2]]), np.array([[0]], np.int32), np.array([t]), 200, seed)
        st = oracle.simulate(b)["states"]
        s, _, var, ci = oracle.replica_stats(st, 1, 200)
        m = float(s[0, 0, 0]) / 200
        hits += abs(m - mu) <= ci[0, 0, 0]
    assert 45 <= hits <= 59
