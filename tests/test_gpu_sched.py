"""Scheduling of uneven sweeps: the autotuner's choice, CUDA-graph replays
and every (layout, block size) give bit-identical trajectories."""
import numpy as np
import pytest
import torch

from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def _sweep():
    b0 = W.sweep256x256(P=32, R=64)
    return W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.05, b0.R, b0.seed)


def _same(x, y):
    for k in ("states", "events", "hash", "status", "final_t"):
        assert torch.equal(x[k], y[k]), k


def test_autotune_choice_and_all_candidates_agree():
    b = _sweep()
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    ref = api.simulate(cm, rates, init, grid, b.R, b.seed, layout=capi.CWC_LAYOUT_STATIC, block_threads=64)
    lay, thr, lanes, ms = api.autotune(cm, rates, init, grid, b.R, b.seed, tune_events=500)
    assert lay in (capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE) and 32 <= thr <= 256 and ms > 0 and lanes == 1
    auto = api.simulate(cm, rates, init, grid, b.R, b.seed)          # uses the cached choice
    torch.cuda.synchronize()
    _same(auto, ref)
    for lay in (capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE):
        for T in (32, 96, 256):
            got = api.simulate(cm, rates, init, grid, b.R, b.seed, layout=lay, block_threads=T)
            torch.cuda.synchronize()
            _same(got, ref)


def test_cuda_graph_replay_matches_direct_calls():
    b = _sweep()
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    g = api.GraphedSimulation(cm, rates, init, grid, b.R, b.seed, sums=True)
    for scale in (1.0, 0.5, 1.0):
        r2 = rates * scale
        out = g.replay(rates=r2)
        torch.cuda.synchronize()
        ref = api.simulate(cm, r2.contiguous(), init, grid, b.R, b.seed, sums=True)
        torch.cuda.synchronize()
        _same(out, ref)
        assert torch.equal(out["sums"], ref["sums"])


def test_cwc_model_autotune_and_graph():
    b0 = W.cwc3x24(R=256, G=20)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.3, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    ref = api.simulate(cm, rates, init, grid, b.R, b.seed, layout=capi.CWC_LAYOUT_STATIC, block_threads=32)
    lay, thr, lanes, _ = api.autotune(cm, rates, init, grid, b.R, b.seed, tune_events=200)
    assert lanes in (1, 4, 8)
    got = api.simulate(cm, rates, init, grid, b.R, b.seed)
    g = api.GraphedSimulation(cm, rates, init, grid, b.R, b.seed)
    out = g.replay()
    torch.cuda.synchronize()
    _same(got, ref)
    _same(out, ref)


def test_time_sliced_run_equals_one_launch():
    """simulate_sliced: many short device-time slices with checkpoints in
    between give the outputs of one launch, for a flat and a compartment
    model."""
    for b in (W.flat16x24(R=4096), W.cwc3x24(R=256, G=50)):
        cm = api.CompiledModel(b.model)
        rates, init, grid = api.device_inputs(b)
        ref = api.simulate(cm, rates, init, grid, b.R, b.seed)
        seen = []
        out, slices = api.simulate_sliced(cm, rates, init, grid, b.R, b.seed, slice_ns=1_000_000,
                                          on_slice=lambda i, rem: seen.append(rem))
        assert slices > 1 and seen[-1] == 0 and len(seen) == slices
        for k in ("states", "events", "hash", "status", "final_t"):
            assert torch.equal(out[k], ref[k]), k
