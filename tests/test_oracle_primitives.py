"""Pins of the oracle's building blocks against mathematics and library routines.

Philox4x32-10 (Salmon et al., SC'11) is pinned on the CPU by the algorithm's
published known-answer vectors (tests/golden/philox4x32_10_kat.json) and by
statistical tests; the GPU test-suite additionally checks it word for word
against cuRAND's Philox4_32_10 (test_oracle_philox_matches_curand in
tests/test_gpu_flat.py).
"""
import decimal
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

EPS = 2.0 ** -52


# ----------------------------------------------------------------------------
# Philox4x32-10
# ----------------------------------------------------------------------------

def test_philox_known_answer_vectors():
    """The published known-answer vectors: a wrong round multiplier, Weyl
    increment, word order or key schedule changes every output word, which
    the statistical tests below cannot see."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")
    with open(path) as f:
        kat = json.load(f)
    assert len(kat["vectors"]) == 3
    for v in kat["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["ctr"]]], np.uint32)
        key = tuple(int(x, 16) for x in v["key"])
        out = oracle.philox(ctr, key)
        assert [int(x) for x in out[0]] == [int(x, 16) for x in v["out"]]


def _stream(n, purpose=0, r=3, p=5, key=(0x01234567, 0x89ABCDEF)):
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 1] = purpose
    ctr[:, 2] = r
    ctr[:, 3] = p
    return oracle.philox(ctr, key)


def test_philox_bit_frequencies():
    w = _stream(1 << 16).ravel()
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.int64)
    ones = bits.sum(axis=0)
    n = w.size
    z = (ones - n / 2) / math.sqrt(n / 4)
    assert np.all(np.abs(z) < 5.0), z


def test_philox_byte_histogram_chi2():
    w = _stream(1 << 16)
    b = w.view(np.uint8).ravel()
    hist = np.bincount(b, minlength=256)
    chi2, p = stats.chisquare(hist)
    assert p > 1e-4


def test_philox_counter_neighbours_uncorrelated():
    a = _stream(1 << 15).astype(np.float64)
    for col in range(4):
        x = a[:-1, col]
        y = a[1:, col]
        rho = np.corrcoef(x, y)[0, 1]
        assert abs(rho) < 5 / math.sqrt(x.size)
    # different purpose / replica / point words give unrelated streams
    b = _stream(1 << 15, purpose=1).astype(np.float64)
    c = _stream(1 << 15, r=4).astype(np.float64)
    for other in (b, c):
        rho = np.corrcoef(a[:, 0], other[:, 0])[0, 1]
        assert abs(rho) < 5 / math.sqrt(a.shape[0])


def test_philox_key_and_counter_sensitivity():
    base = _stream(64)
    assert not np.array_equal(base, _stream(64, key=(0x01234566, 0x89ABCDEF)))
    assert not np.array_equal(base, _stream(64, key=(0x01234567, 0x89ABCDEE)))
    # a one-bit counter change flips about half of the 128 output bits
    ctr = np.array([[7, 0, 3, 5], [7 ^ 1, 0, 3, 5], [7, 1 << 31, 3, 5], [7, 0, 3, 5 ^ (1 << 17)]], np.uint32)
    out = oracle.philox(ctr, (1, 2))
    for i in range(1, 4):
        flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(out[0], out[i]))
        assert 40 <= flips <= 88


# ----------------------------------------------------------------------------
# u52
# ----------------------------------------------------------------------------

def test_u52_boundaries_and_exactness():
    assert oracle.u52(0, 0) == 2.0 ** -53
    assert oracle.u52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # the 6 low bits of each word are discarded
    assert oracle.u52(0x3F, 0x3F) == 2.0 ** -53
    assert oracle.u52(0, 0x40) == 3 * 2.0 ** -53
    assert oracle.u52(0x40, 0) == (2 * 2 ** 26 + 1) * 2.0 ** -53
    rng = np.random.default_rng(11)
    for wa, wb in rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64):
        u = oracle.u52(int(wa), int(wb))
        v = u * 2.0 ** 53
        assert 0.0 < u < 1.0
        assert v == math.floor(v) and int(v) % 2 == 1          # (2k+1) 2^-53 exactly
        k = ((int(wa) >> 6) << 26) | (int(wb) >> 6)
        assert int(v) == 2 * k + 1


# ----------------------------------------------------------------------------
# log_spec: within 2 ulp of the C library logarithm
# ----------------------------------------------------------------------------

def _ulp_err(x, ref):
    spacing = np.spacing(np.abs(ref))
    return np.abs(x - ref) / spacing


def test_log_spec_accuracy_random():
    rng = np.random.default_rng(12)
    u1 = rng.random(500_000)
    u1 = u1[u1 > 0]
    u2 = 10.0 ** rng.uniform(-16, 0, 500_000)
    u2 = u2[(u2 > 0) & (u2 < 1)]
    for u in (u1, u2):
        got = oracle.log_spec(u)
        ref = np.log(u)
        assert np.max(_ulp_err(got, ref)) <= 1.0


def test_log_spec_edges():
    sqrt2 = math.sqrt(2.0)
    edges = [2.0 ** -53, 2.0 ** -52, 3 * 2.0 ** -53, 0.5, 0.25, 1 - 2.0 ** -53, 1 - 2.0 ** -52,
             sqrt2 / 2, np.nextafter(sqrt2 / 2, 0), np.nextafter(sqrt2 / 2, 1), 1 / sqrt2,
             0.7071067811865475, 0.7071067811865476, 1e-10, 0.1, 0.9, 0.999999]
    edges += [2.0 ** -k for k in range(1, 54)]
    edges += [np.nextafter(2.0 ** -k, 1) for k in range(1, 53)]
    u = np.array(edges)
    got = oracle.log_spec(u)
    ref = np.log(u)
    assert np.max(_ulp_err(got, ref)) <= 1.0
    assert np.all(got < 0)
    # exact powers of two: the series contributes exactly 0, so the result is
    # k ln 2 rounded once to nearest
    decimal.getcontext().prec = 60
    ln2 = decimal.Decimal(2).ln()
    for k in range(1, 54):
        assert oracle.log_spec([2.0 ** -k])[0] == -float(k * ln2)


def _decimal_ulp_err(u, got):
    decimal.getcontext().prec = 60
    out = []
    for x, y in zip(u, got):
        r = decimal.Decimal(float(x)).ln()
        out.append(abs(float((decimal.Decimal(float(y)) - r) / decimal.Decimal(math.ulp(float(r))))))
    return np.array(out)


def test_log_spec_within_0p55_ulp_of_60_digit_logarithms():
    """Both series paths (near one, and the atanh path over every binade of
    the uniforms) against logarithms to 60 digits: the integer evaluation
    rounds once, so the error stays just above half an ulp."""
    rng = np.random.default_rng(31)
    k = (rng.integers(0, 1 << 26, 3000, dtype=np.int64) << 26) | rng.integers(0, 1 << 26, 3000, dtype=np.int64)
    u = list((2.0 * k + 1.0) * 2.0 ** -53)
    near = 1.0 - rng.integers(1, 1 << 47, 500) * 2.0 ** -53          # both sides of the 2^-7 switch
    u += list(near)
    u += [1 - 2.0 ** -53, 1 - 2.0 ** -7, 1 - 2.0 ** -7 - 2.0 ** -53, 1 - 2.0 ** -7 + 2.0 ** -53, 2.0 ** -53]
    for e in range(-53, 0):
        b = 2.0 ** e
        u += [np.nextafter(2 * b, 0), math.sqrt(2.0) * b, np.nextafter(math.sqrt(2.0) * b, 0), 1.5 * b]
    u = np.array([x for x in u if 2.0 ** -53 <= x < 1.0])
    err = _decimal_ulp_err(u, oracle.log_spec(u))
    assert err.max() < 0.55


def test_log_spec_monotone():
    u = np.sort(np.random.default_rng(13).random(200_000))
    u = u[u > 0]
    got = oracle.log_spec(u)
    assert np.all(np.diff(got) >= 0)


# ----------------------------------------------------------------------------
# 32-lane blocked tree
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M", [1, 2, 7, 12, 24, 31, 32, 33, 48, 64, 65, 100, 200])
def test_tree_sum_error_bound(M):
    rng = np.random.default_rng(M)
    for _ in range(50):
        a = rng.random(M) * 10.0 ** rng.uniform(-5, 5, M)
        a[rng.random(M) < 0.2] = 0.0
        got = oracle.tree_sum(a)
        exact = math.fsum(a)
        B = (M + 31) // 32
        depth = 5 + (B - 1)          # additions on any leaf-to-root path
        assert abs(got - exact) <= depth * EPS * math.fsum(np.abs(a)) + 0.0


def test_tree_sum_exact_cases():
    assert oracle.tree_sum(np.zeros(17)) == 0.0
    a = np.zeros(50)
    a[37] = 0.1234567890123
    assert oracle.tree_sum(a) == 0.1234567890123
    ints = np.arange(1, 101, dtype=np.float64) * 3.0
    assert oracle.tree_sum(ints) == 3.0 * 5050
    # the blocked order is not the naive left-to-right order
    a = np.array([1.0, 2.0 ** -53, 2.0 ** -53] + [0.0] * 29)
    assert oracle.tree_sum(a) == 1.0          # (1 + 2^-53) + 2^-53 pairwise at level 1..5
    b = np.array([1.0] + [0.0] * 31 + [2.0 ** -53] * 32)   # B = 2
    naive = 1.0
    for v in b[1:]:
        naive += v
    assert naive == 1.0
    assert abs(oracle.tree_sum(b) - math.fsum(b)) <= 6 * EPS * math.fsum(b)


# ----------------------------------------------------------------------------
# Guarded selection
# ----------------------------------------------------------------------------

def test_select_never_picks_zero():
    rng = np.random.default_rng(21)
    for M in (1, 3, 12, 32, 33, 64, 100):
        for _ in range(200):
            a = np.where(rng.random(M) < 0.6, 0.0, 10.0 ** rng.uniform(-300, 3, M))
            if not np.any(a > 0):
                a[rng.integers(M)] = 1e-300
            a0 = oracle.tree_sum(a)
            for x in (0.0, a0 * 0.5, np.nextafter(a0, 0), a0, a0 * 1.0000001, rng.random() * a0):
                j = oracle.select(a, x)
                assert 0 <= j < M and a[j] > 0


def test_select_extremes():
    a = np.array([0.0, 0.0, 2.0, 0.0, 3.0, 0.0])
    assert oracle.select(a, 0.0) == 2
    assert oracle.select(a, 1.9999) == 2
    assert oracle.select(a, 2.0) == 4
    assert oracle.select(a, 4.99) == 4
    assert oracle.select(a, 1e9) == 4


@pytest.mark.parametrize("M", [5, 12, 32, 40, 64, 97])
def test_select_frequencies_quadrature(M):
    """With x = u a0 on a fine uniform grid of u, the share of picks of j is a_j/a0."""
    rng = np.random.default_rng(100 + M)
    a = np.where(rng.random(M) < 0.3, 0.0, rng.random(M) * 10.0 ** rng.uniform(-2, 2, M))
    a[0] = max(a[0], 1e-3)
    a0 = oracle.tree_sum(a)
    N = 20000
    picks = np.array([oracle.select(a, ((i + 0.5) / N) * a0) for i in range(N)])
    freq = np.bincount(picks, minlength=M) / N
    assert np.all(np.abs(freq - a / a0) <= 2.0 / N + 1e-12)
