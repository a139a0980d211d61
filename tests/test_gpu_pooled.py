"""GPU parity of the flat kernel's pooled leaf rebuild (the warp rebuilds its
lanes' dirty leaves together; chosen for B > 1 networks whose events dirty
three leaves or more on average).

The pooled path must give the oracle's trajectories bit for bit, including
the two places where it differs in mechanism from a lane rebuilding its own
leaves: a count product that overflows int64 inside a leaf rebuilt by
another lane (written as +inf, which must end the trajectory with
PROP_OVERFLOW at its next step exactly as the overflow flag does), and the
score replay, whose leaves read the owner's h values.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

from test_gpu_flat import assert_same, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def _dirty_leaves_per_rule(model):
    M = model.n_rules
    B = (M + 31) // 32
    lhs = model.lhs[:, 0, :]
    delta = model.rhs[:, 0, :] - lhs
    tot = 0
    for j in range(M):
        changed = set(np.nonzero(delta[j])[0])
        deps = [i for i in range(M) if changed & set(np.nonzero(lhs[i])[0])]
        tot += len(set(i // B for i in deps))
    return B, tot / M


def _overflow_model():
    """34 rules (B = 2): a trimolecular A + B + C -> ... whose count A B C is
    just below 2^63 with C = 2, an inflow of C, and 32 conversions D <-> E
    that dirty 16 leaves per event (so the leaves are pooled).  When the
    inflow fires, C = 3 overflows the trimolecular rule's count."""
    reactions = [({0: 1, 1: 1, 2: 1}, {0: 1, 1: 1, 2: 1, 3: 1}), ({}, {2: 1})]
    for _ in range(16):
        reactions.append(({3: 1}, {4: 1}))
        reactions.append(({4: 1}, {3: 1}))
    model = W.flat_model(5, reactions, "overflow_pool")
    rates = np.ones((1, len(reactions)))
    rates[0, 0] = 1e-30
    rates[0, 1] = 0.05
    init = np.array([[2 ** 31 - 1, 2 ** 31 - 1, 2, 50, 50]], np.int32)
    return W.Batch(model, rates, init, W.uniform_grid(100.0, 11), 32, 77, max_events=200000)


def test_pooled_leaf_count_overflow_ends_with_prop_overflow():
    b = _overflow_model()
    B, dirty = _dirty_leaves_per_rule(b.model)
    assert B == 2 and dirty >= 3.0
    g = gpu_run(b)
    o = oracle.simulate(b, threads=8)
    assert_same(g, o)
    assert np.all(o["status"] == capi.CWC_TRAJ_PROP_OVERFLOW) and o["events"].min() > 100


@pytest.mark.parametrize("layout", [capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE])
@pytest.mark.parametrize("threads", [32, 96, 224])
def test_pooled_flat32x64_bit_exact_with_event_log(layout, threads):
    """64 rules, 4.45 dirty leaves per event; ragged R, several block sizes
    (a block of 32 is one warp), both layouts."""
    b0 = W.flat32x64(R=197)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.01, b0.R, b0.seed)
    assert _dirty_leaves_per_rule(b.model)[1] >= 3.0
    g = gpu_run(b, log_cap=256, layout=layout, block_threads=threads)
    o = oracle.simulate(b, threads=8, log_cap=256)
    assert_same(g, o)
    valid = np.arange(256)[None, :] < np.minimum(o["events"], 256)[:, None]
    assert np.array_equal(g["log_rule"][valid], o["log_rule"][valid])


def test_pooled_score_replay_partials_match_oracle():
    """The score replay with pooled leaves (owner's h read from shared
    memory): partials within the tolerance of the other replay tests."""
    b0 = W.flat32x64(R=64, G=12)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.004, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(8)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, b.model.n_observables))).cuda()
    res = api.sensitivity(cm, rates, init, grid, b.R, b.seed, means, gm, partials=True)
    torch.cuda.synchronize()
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    ograd, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert scale > 0
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))
    gg = res["grad_rates"].cpu().numpy()
    assert np.all(np.abs(gg - ograd) <= 1e-9 * (np.abs(ograd) + scale))
