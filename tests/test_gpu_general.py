"""GPU parity for the general CWC patterns: two compartments in one left-hand
side, merged (FUSION) or both kept (PAIR), and patterns of depth two (NESTED),
mixed with every other
rule kind, against the oracle bit for bit (observables, statuses, event
counts, (rule, context) hashes, final times, event logs); score partials
within the FP64 tolerance of the other compartment tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

from test_gpu_cwc import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


@pytest.mark.parametrize("layout,lanes", [(capi.CWC_LAYOUT_STATIC, 1), (capi.CWC_LAYOUT_QUEUE, 1),
                                          (capi.CWC_LAYOUT_QUEUE, 4), (capi.CWC_LAYOUT_STATIC, 8)])
def test_general_model_bit_exact_with_event_log(layout, lanes):
    """21 rules of all seven kinds, 256 replicas x ~1.2e3 events; every rule
    kind fires (checked on the oracle's log), the symmetric vesicle PAIR too."""
    b = W.cwc_general(R=256)
    g, o = check(b, log_cap=2048, layout=layout, lanes=lanes)
    fired = np.unique(o["log_rule"][o["log_rule"] >= 0])
    assert set(W.KIND_NAMES) == set(b.model.kind[fired].tolist())
    pairs = o["log_slot"][np.isin(o["log_rule"], np.nonzero(np.isin(b.model.kind, (W.FUSION, W.PAIR)))[0])]
    assert pairs.size > 0 and np.all(pairs >> 16 > 0)          # pair contexts were logged
    assert np.isin(np.nonzero(b.model.kind == W.PAIR)[0], fired).all()


def test_general_model_ragged_batch_and_sweep_points():
    """Two sweep points (rates x1 and x2) x 37 replicas: a ragged last block."""
    b0 = W.cwc_general(R=37)
    rates = np.concatenate([b0.rates, b0.rates * 2.0])
    b = W.Batch(b0.model, rates, b0.init, b0.grid * 0.5, b0.R, b0.seed)
    check(b, lanes=4)


@pytest.mark.parametrize("lanes", [1, 4])
def test_law_models_of_the_general_patterns_bit_exact(lanes):
    """The pinned oracle scenarios: fusion of six empty compartments (the
    pure-death chain), depth-two transport with a decoy, fusion that moves
    children followed by depth-two drainage."""
    m = W.cwc_model(1, 2, 7, [W.RuleSpec(W.FUSION, 0, 1)])
    img = W.empty_slot_image(m)
    for c in range(1, 7):
        img[c, :3] = [1, 1, 0]
        img[c, 4] = 1
    check(W.Batch(m, np.array([[0.7]]), img[None], np.array([0.0, 0.1, 0.3, 0.8, 2.0]), 500, 41), lanes=lanes)

    m = W.cwc_model(1, 3, 7, [W.RuleSpec(W.NESTED, 0, 1, grand_label=2, lhs_child2={0: 1}, rhs_ctx={0: 1})])
    img = W.empty_slot_image(m)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 2, 1]
    img[2, 4] = 20
    img[3, :3] = [1, 1, 0]
    img[4, :3] = [1, 2, 3]
    img[4, 4] = 20
    img[5, :3] = [1, 2, 0]
    img[5, 4] = 9
    check(W.Batch(m, np.array([[0.6]]), img[None], np.array([0.0, 0.5, 1.5, 4.0]), 500, 12), lanes=lanes)

    rules = [W.RuleSpec(W.FUSION, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_child={1: 3}),
             W.RuleSpec(W.NESTED, 0, 1, grand_label=2, lhs_child2={0: 1}, rhs_ctx={0: 1})]
    m = W.cwc_model(2, 3, 6, rules)
    img = W.empty_slot_image(m)
    img[1, :7] = [1, 1, 0, 2, 0, 4, 0]
    img[3, :7] = [1, 1, 0, 1, 5, 0, 7]
    img[2, :3] = [1, 2, 1]
    img[2, 5] = 3
    img[4, :3] = [1, 2, 3]
    img[4, 5] = 2
    g, o = check(W.Batch(m, np.array([[1e6, 1.0]]), img[None], np.array([0.0, 1e-3, 100.0]), 64, 3),
                 log_cap=8, lanes=lanes)
    assert np.all(g["log_slot"][:, 0] == (1 | (3 << 16)))


def test_general_model_capacity_and_int_overflow_statuses():
    """A fusion whose merged wrap would exceed INT32_MAX stops the trajectory
    with INT_OVERFLOW before anything changes, as in the oracle."""
    rules = [W.RuleSpec(W.FUSION, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={0: 2})]
    m = W.cwc_model(1, 2, 4, rules)
    img = W.empty_slot_image(m)
    img[1, :4] = [1, 1, 0, 2 ** 31 - 5]
    img[2, :4] = [1, 1, 0, 10]
    g, o = check(W.Batch(m, np.array([[1.0]]), img[None], np.array([0.0, 10.0]), 8, 5), lanes=4)
    assert np.all(g["status"] == oracle.ST_INT_OVERFLOW)


@pytest.mark.parametrize("lanes", [1, 4])
def test_general_model_sensitivity_partials_match_oracle(lanes):
    b0 = W.cwc_general(R=48, G=10)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.5, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(3)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, cm.n_observables)) * 1e-2).cuda()
    res = api.sensitivity(cm, rates, init, grid, b.R, b.seed, means, gm, partials=True, lanes=lanes)
    torch.cuda.synchronize()
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    ograd, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert scale > 0
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))


def test_general_model_checkpoint_resume_equals_one_launch():
    """Time-sliced with checkpoints (short deadlines) equals one launch."""
    b = W.cwc_general(R=128)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    one = api.simulate(cm, rates, init, grid, b.R, b.seed, lanes=4)
    sl, n = api.simulate_sliced(cm, rates, init, grid, b.R, b.seed, slice_ns=200_000, lanes=4)
    torch.cuda.synchronize()
    for k in ("states", "status", "events", "hash", "final_t"):
        assert torch.equal(one[k], sl[k]), k


def test_checkpoint_records_of_odd_length():
    """A term of 7 slots x (3 + 2 S) words makes 43-word checkpoint records,
    so every other record's 64-bit fields (time, hash) sit on a 4-byte
    boundary; time-sliced runs must still equal one launch."""
    m = W.cwc_model(1, 3, 7, [W.RuleSpec(W.NESTED, 0, 1, grand_label=2, lhs_child2={0: 1}, rhs_ctx={0: 1}),
                              W.RuleSpec(W.LOCAL, 0, lhs_ctx={0: 1}, rhs_ctx={0: 2})])
    img = W.empty_slot_image(m)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 2, 1]
    img[2, 4] = 3000
    img[3, :3] = [1, 1, 0]
    img[4, :3] = [1, 2, 3]
    img[4, 4] = 3000
    b = W.Batch(m, np.array([[1.0, 0.001]]), img[None], W.uniform_grid(2.0, 9), 33, 21)
    assert capi.cwc_checkpoint_words(api.CompiledModel(b.model).handle) % 2 == 1
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    one = api.simulate(cm, rates, init, grid, b.R, b.seed, lanes=1)
    sl, n = api.simulate_sliced(cm, rates, init, grid, b.R, b.seed, slice_ns=50_000, lanes=1)
    torch.cuda.synchronize()
    for k in ("states", "status", "events", "hash", "final_t"):
        assert torch.equal(one[k], sl[k]), k


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_pair_rules_bit_exact(lanes):
    """The pinned PAIR scenarios: sibling transport (the Ehrenfest model, both
    directions as ordered pairs) among three compartments, a symmetric rule
    (unordered pairs), a one-sided rule with identical left-hand patterns
    (ordered pairs) and a rewrite of the parent content with both children,
    and a PAIR whose second compartment would overflow: INT_OVERFLOW."""
    m = W.cwc_model(1, 2, 4, [W.RuleSpec(W.PAIR, 0, 1, lhs_child={0: 1}, rhs_child2={0: 1})])
    img = W.empty_slot_image(m)
    for c, n in ((1, 12), (2, 3), (3, 0)):
        img[c, :3] = [1, 1, 0]
        img[c, 4] = n
    g, o = check(W.Batch(m, np.array([[0.7]]), img[None], np.array([0.0, 0.2, 0.6, 1.5, 4.0]), 300, 41),
                 log_cap=64, lanes=lanes)
    assert len(set(o["log_slot"][o["log_rule"] >= 0].tolist())) == 6     # all six ordered pairs

    rules = [W.RuleSpec(W.PAIR, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_wrap2={1: 1}),
             W.RuleSpec(W.PAIR, 0, 1, lhs_wrap={0: 1}, lhs_wrap2={0: 1}, rhs_wrap={1: 1}, rhs_wrap2={0: 1}),
             W.RuleSpec(W.PAIR, 0, 1, lhs_ctx={2: 1}, lhs_child={0: 1}, lhs_wrap2={1: 1},
                        rhs_child={1: 1}, rhs_wrap2={0: 2}, rhs_child2={2: 1}),
             W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_child={1: 1}, rhs_child={0: 1})]
    m = W.cwc_model(3, 2, 6, rules)
    img = W.empty_slot_image(m)
    img[0, 3 + 3 + 2] = 40
    for c in range(1, 5):
        img[c, :3] = [1, 1, 0]
        img[c, 3:6] = [3, 1, 0]
        img[c, 6:9] = [2, 2, 0]
    check(W.Batch(m, np.array([[0.3, 0.2, 0.05, 0.4]]), img[None], np.array([0.0, 0.5, 2.0, 6.0]), 200, 17),
          log_cap=256, lanes=lanes)

    m = W.cwc_model(1, 2, 3, [W.RuleSpec(W.PAIR, 0, 1, lhs_child={0: 1}, rhs_child={0: 1}, rhs_child2={0: 3})])
    img = W.empty_slot_image(m)
    img[1, :4] = [1, 1, 0, 0]
    img[1, 4] = 5
    img[2, :3] = [1, 1, 0]
    img[2, 4] = 2 ** 31 - 2
    g, o = check(W.Batch(m, np.array([[1.0]]), img[None], np.array([0.0, 10.0]), 8, 5), lanes=lanes)
    assert np.all(g["status"] == oracle.ST_INT_OVERFLOW)
