"""The tail layout (CWC_LAYOUT_TAIL): the queue kernel hands its last
trajectories over to one warp each.  Whichever kernel finishes a trajectory,
its results must equal the oracle's and the other layouts' bit for bit.
tail_threshold >= the batch size hands every trajectory over at its first
1024-event boundary, so the warp kernel runs nearly all the events."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

from test_gpu_flat import assert_same, gpu_run

pytestmark = pytest.mark.gpu
KEYS = ("status", "events", "hash", "final_t", "states")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def tail_vs_oracle(batch, threshold, log_cap=0, **kw):
    g = gpu_run(batch, layout=capi.CWC_LAYOUT_TAIL, tail_threshold=threshold, log_cap=log_cap, **kw)
    o = oracle.simulate(batch, threads=8, log_cap=log_cap)
    assert_same(g, o)
    if log_cap:
        valid = np.arange(log_cap)[None, :] < np.minimum(o["events"], log_cap)[:, None]
        assert np.array_equal(g["log_rule"][valid], o["log_rule"][valid])
        assert np.array_equal(g["log_t"].view(np.int64)[valid], o["log_t"].view(np.int64)[valid])
    return g, o


@pytest.mark.parametrize("name", ["flat8x12", "flat16x24", "flat32x64", "lv32"])
def test_warp_kernel_finishes_every_trajectory_bit_exact(name):
    """Every trajectory handed over after 1024 events: B = 1 with idle leaves
    (M = 12, 24), B = 2 (M = 64), S = 32 and a Lotka-Volterra chain."""
    if name == "lv32":
        b = W.lotka_volterra(32, R=96, G=40, T=0.02)
    else:
        b0 = getattr(W, name)(R=96, G=40)
        scale = 0.05 if name == "flat32x64" else 0.2
        b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * scale, b0.R, b0.seed)
    g, o = tail_vs_oracle(b, threshold=1 << 20, log_cap=3000)
    assert np.mean(o["events"]) > 2000          # most of the events ran in the warp kernel


def test_tail_sweep_points_and_reductions_match_queue_layout():
    """Eight sweep points of uneven length, means / variance / interval over
    replicas, default and forced thresholds: identical to the queue layout."""
    b0 = W.sweep256x256(P=8, R=96, G=50)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.05, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    kw = dict(states=True, means=True, sums=True, variance=True, ci90=True)
    ref = api.simulate(cm, rates, init, grid, b.R, b.seed, layout=capi.CWC_LAYOUT_QUEUE, **kw)
    for thr in (0, 40, 1 << 20):
        got = api.simulate(cm, rates, init, grid, b.R, b.seed, layout=capi.CWC_LAYOUT_TAIL, tail_threshold=thr, **kw)
        torch.cuda.synchronize()
        for k in ("states", "means", "sums", "variance", "ci90", "status", "events", "hash", "final_t"):
            assert torch.equal(got[k], ref[k]), (thr, k)


def test_warp_kernel_statuses():
    """Event cap, absorption and count overflow reached inside the warp kernel."""
    b = W.flat8x12(R=40, G=20)
    tail_vs_oracle(W.Batch(b.model, b.rates, b.init, b.grid, b.R, b.seed, max_events=1500), threshold=1 << 20)
    m = W.flat_model(1, [({0: 1}, {})])                         # pure death from 5000: absorbed
    tail_vs_oracle(W.Batch(m, np.array([[1.0]]), np.array([[5000]], np.int32), np.array([0.0, 1e3]), 16, 4),
                   threshold=1 << 20)
    m = W.birth_death()                                          # births push past INT32_MAX
    g, _ = tail_vs_oracle(W.Batch(m, np.array([[1e9, 1e-12]]), np.array([[2 ** 31 - 1500]], np.int32),
                                  np.array([0.0, 1.0]), 8, 6), threshold=1 << 20)
    assert np.all(g["status"] == oracle.ST_INT_OVERFLOW)


def test_warp_kernel_large_network_multi_block_leaves():
    """M = 200 rules (B = 7 per leaf) over S = 100 species: leaf scans of
    several rules and records wider than a warp."""
    rng = W.SplitMix64(77)
    m = W.random_flat_network(rng, 100, 140, 40, 10)
    assert m.n_rules > 160 and m.n_species == 100
    x0 = np.array([[rng.randint(50, 300) for _ in range(100)]], np.int32)
    k = np.array([[rng.log_uniform(-3, 0) for _ in range(m.n_rules)]])
    b = W.Batch(m, k, x0, W.uniform_grid(0.5, 30), 48, 9)
    g, o = tail_vs_oracle(b, threshold=1 << 20)
    assert np.mean(o["events"]) > 1500


def test_tail_layout_argument_rules():
    b = W.cwc3x24(R=4, G=4)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    a = api._sim_args(cm, rates, init, grid, b.R, b.seed, 10, capi.CWC_LAYOUT_TAIL, 0, 0)
    assert capi.lib().cwc_simulate(cm.handle, ctypes.byref(a), None) == capi.CWC_ERR_INVALID_ARG
    b = W.flat8x12(R=4, G=4)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    a = api._sim_args(cm, rates, init, grid, b.R, b.seed, 10, capi.CWC_LAYOUT_TAIL, 0, 1000)   # deadline
    assert capi.lib().cwc_simulate(cm.handle, ctypes.byref(a), None) == capi.CWC_ERR_INVALID_ARG
    a = api._sim_args(cm, rates, init, grid, b.R, b.seed, 10, capi.CWC_LAYOUT_TAIL, 0, 0)
    a.tail_threshold = -1
    assert capi.lib().cwc_simulate(cm.handle, ctypes.byref(a), None) == capi.CWC_ERR_INVALID_ARG
