"""Pins of the oracle's likelihood-ratio sensitivities.

For a CTMC path with propensities a_j = k_j H_j(X), the score of rule j up to
time g is S_j(g) = N_j(g)/k_j - int_0^g H_j(X(s)) ds, and
d E[f(X(g))]/d k_j = E[(f(X(g)) - E f) S_j(g)].  With an upstream gradient
G[g, o] of L = sum_g,o G[g,o] E[X_o(g)], the oracle returns per trajectory
sum_g c(g) S_j(g), c(g) = sum_o G[g,o] (X_o(g) - mean_o(g)).

Tolerance, stated in Monte-Carlo standard errors (SE) of the estimates, with
fixed seeds: at least 99 % of the entries within 3 SE and none beyond 5 SE;
with fewer than 100 entries (where 99 % would allow no miss anyway) every
entry within 3 SE.  For a comparison with finite differences the SE is
sqrt(SE_LR^2 + SE_FD^2).  The same rule is used by the GPU tests
(tests/test_gpu_lr_fd.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1010_2438_gb300 import workloads as W


def lr_per_grid_point(batch, threads=8):
    """LR estimates and SEs of d E[X_o(g)] / d k_j for every g, o, j (small O, G)."""
    means = oracle.mean_observables(batch, threads=threads)
    P, G, O = means.shape
    M = batch.model.n_rules
    est = np.zeros((G, O, M))
    se = np.zeros((G, O, M))
    for g in range(G):
        for o in range(O):
            gm = np.zeros_like(means)
            gm[0, g, o] = 1.0
            grad, part = oracle.sensitivity(batch, means, gm, threads=threads)
            est[g, o] = grad[0]
            se[g, o] = part.std(axis=0, ddof=1) / math.sqrt(batch.R)
    return est, se


def check_z(z):
    """>= 99 % of |z| within 3 and none beyond 5; every |z| within 3 when
    there are fewer than 100 entries."""
    z = np.abs(np.asarray(z, np.float64)).ravel()
    print("z-scores:", np.round(z, 2))
    assert np.all(np.isfinite(z))
    if z.size < 100:
        assert np.all(z <= 3.0), z.max()
    else:
        assert np.mean(z <= 3.0) >= 0.99, np.mean(z <= 3.0)
        assert np.all(z <= 5.0), z.max()


def test_birth_death_lr_matches_analytic_gradient():
    k1, k2, x0 = 8.0, 0.7, 20
    grid = np.array([0.3, 1.0, 2.0, 4.0])
    b = W.Batch(W.birth_death(), np.array([[k1, k2]]), np.array([[x0]], np.int32), grid, 40000, 4242)
    est, se = lr_per_grid_point(b)
    z = []
    for g, t in enumerate(grid):
        e = math.exp(-k2 * t)
        d1 = (1 - e) / k2
        d2 = -x0 * t * e - k1 / k2 ** 2 * (1 - e) + k1 / k2 * t * e
        z += [(est[g, 0, 0] - d1) / se[g, 0, 0], (est[g, 0, 1] - d2) / se[g, 0, 1]]
    check_z(z)


def test_birth_death_lr_zero_at_time_zero():
    b = W.Batch(W.birth_death(), np.array([[3.0, 1.0]]), np.array([[5]], np.int32),
                np.array([0.0, 1.0]), 200, 1)
    means = oracle.mean_observables(b)
    gm = np.zeros_like(means)
    gm[0, 0, 0] = 1.0             # derivative of E X(0) = x0: exactly zero
    grad, part = oracle.sensitivity(b, means, gm)
    assert np.all(part == 0.0)


def fd_crn(batch, j, rel=0.05, G_up=None, threads=8):
    """Central finite difference of L (or of every mean) w.r.t. k_j with common random numbers."""
    k = batch.rates
    d = rel * k[0, j]
    outs = []
    for sgn in (1, -1):
        kk = k.copy()
        kk[:, j] += sgn * d
        st = oracle.simulate(batch, rates=kk, threads=threads)["states"].astype(np.float64)
        outs.append(st)
    diff = (outs[0] - outs[1]) / (2 * d)          # per trajectory [nq, G, O]
    if G_up is not None:
        per = np.einsum("qgo,go->q", diff, G_up)
        return per.mean(), per.std(ddof=1) / math.sqrt(per.size)
    return diff.mean(axis=0), diff.std(axis=0, ddof=1) / math.sqrt(diff.shape[0])


def test_isomerisation_lr_vs_central_fd_crn():
    kf, kb = 1.2, 0.5
    grid = np.array([0.4, 1.5])
    b = W.Batch(W.isomerisation(), np.array([[kf, kb]]), np.array([[25, 5]], np.int32), grid, 20000, 31)
    est, se = lr_per_grid_point(b)
    z = []
    for j in range(2):
        fd, fse = fd_crn(b, j)
        z += list(((est[:, :, j] - fd) / np.sqrt(se[:, :, j] ** 2 + fse ** 2)).ravel())
    check_z(z)


def test_network_lr_vs_fd_with_upstream_gradient():
    """A random 8x12 network and a random upstream gradient G[g, o]."""
    b0 = W.flat8x12(R=3000, G=6)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.1, b0.R, b0.seed)   # ~1e3 events each
    rng = np.random.default_rng(5)
    G_up = rng.standard_normal((b.G, b.model.n_observables))
    means = oracle.mean_observables(b, threads=8)
    grad, part = oracle.sensitivity(b, means, G_up[None], threads=8)
    se = part.std(axis=0, ddof=1) / math.sqrt(b.R)
    z = []
    for j in range(b.model.n_rules):
        fd, fse = fd_crn(b, j, G_up=G_up)
        z.append((grad[0, j] - fd) / math.sqrt(se[j] ** 2 + fse ** 2))
    check_z(z)
