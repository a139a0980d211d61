"""GPU parity of the Michaelis-Menten rate law (flat networks).

Sec. 2.2 takes mass action as the usual rate and allows other kinetics; the
library's reading is a per-reaction Michaelis-Menten law
h = RN(RN(n_E n_S) / RN(K + n_S)) (RN(n_S / RN(K + n_S)) without an enzyme),
a = RN(k h).  The GPU runs it in a separate instantiation of the flat kernel
and must give the oracle's trajectories bit for bit: statuses, event counts,
event hashes, final times, grid states and the event log; the score replay
within the tolerance of the mass-action replay.
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


def check(batch, **kw):
    g = gpu_run(batch, **kw)
    o = oracle.simulate(batch, threads=8, log_cap=kw.get("log_cap", 0))
    assert_same(g, o)
    cap = kw.get("log_cap", 0)
    if cap:
        valid = np.arange(cap)[None, :] < np.minimum(o["events"], cap)[:, None]
        assert np.array_equal(g["log_rule"][valid], o["log_rule"][valid])
        assert np.array_equal(g["log_t"].view(np.int64)[valid], o["log_t"].view(np.int64)[valid])
    return g, o


@pytest.mark.parametrize("layout", [capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE])
@pytest.mark.parametrize("stages", [3, 20])
def test_cascade_bit_exact_with_event_log(layout, stages):
    """6 rules (one leaf per rule) and 40 rules (leaf blocks of 2, whose scan
    evaluates h in the descent), ragged R."""
    b = W.mm_cascade(stages=stages, R=77, G=25, T=8.0)
    g, o = check(b, log_cap=256, layout=layout)
    assert np.all(o["status"] == oracle.ST_OK) and o["events"].min() > 100


def test_cascade_sweep_points_bit_exact():
    b = W.mm_cascade(stages=20, R=40, G=10, T=5.0, P=6)
    check(b, layout=capi.CWC_LAYOUT_QUEUE)


def test_mixed_mass_action_and_michaelis_menten_bit_exact():
    """Mass-action rules of order 0, 1 and 2 beside Michaelis-Menten rules
    with and without an enzyme, 36 rules (leaf blocks of 2)."""
    reactions, mm = [], {}
    S = 12
    rng = np.random.default_rng(11)
    for j in range(36):
        a, c = (int(v) for v in rng.choice(S, 2, replace=False))
        kind = j % 6
        if kind == 0:
            reactions.append(({}, {a: 1}))
        elif kind == 1:
            reactions.append(({a: 1}, {}))
        elif kind == 2:
            reactions.append(({a: 2}, {c: 2}))
        elif kind == 3:
            reactions.append(({a: 1, c: 1}, {c: 1, (a + 1) % S: 1}))
            mm[j] = (a, float(rng.uniform(0.5, 80.0)))
        elif kind == 4:
            reactions.append(({a: 1}, {c: 1}))
            mm[j] = (a, float(rng.uniform(0.5, 80.0)))
        else:
            reactions.append(({a: 1, c: 1}, {a: 1, (c + 1) % S: 1}))
    model = W.flat_model(S, reactions, "mixed", michaelis_menten=mm)
    # every reaction but the inflow conserves or lowers the molecule count;
    # bimolecular mass-action constants scaled down to per-molecule rates
    rates = rng.uniform(0.05, 3.0, (1, 36))
    for j in range(36):
        if j % 6 in (2, 5):
            rates[0, j] *= 0.01
    init = rng.integers(5, 60, (1, S)).astype(np.int32)
    b = W.Batch(model, rates, init, W.uniform_grid(2.0, 20), 96, 5, max_events=200000)
    g, o = check(b, log_cap=128)
    lr = o["log_rule"]
    fired = set(lr[lr >= 0].tolist())
    assert len(fired & set(mm)) >= 3


def test_underflowing_propensity_never_fires():
    """A Michaelis-Menten rule with h < 1 and a subnormal k has a = RN(k h) =
    0 although h > 0: the leaf scan must skip it (the oracle tests a > 0),
    so it never fires.  34 rules make leaf blocks of 2; the rule is the
    second of its block, where the scan's fallback (the last positive entry)
    would otherwise pick it."""
    S = 4
    reactions = [({1: 1}, {0: 1}), ({0: 1}, {1: 1})] + [({2: 1}, {3: 1}), ({3: 1}, {2: 1})] * 16
    mm = {1: (0, 1e6)}   # h = n / (1e6 + n) < 1
    model = W.flat_model(S, reactions, "underflow", michaelis_menten=mm)
    rates = np.full((1, len(reactions)), 1.0)
    rates[0, 1] = 5e-324
    init = np.array([[50, 50, 20, 20]], np.int32)
    b = W.Batch(model, rates, init, W.uniform_grid(1.0, 10), 64, 9)
    g, o = check(b, log_cap=512)
    lr = o["log_rule"]
    assert not np.any(lr == 1) and np.any(lr == 0)


def test_huge_counts_round_like_the_oracle():
    """Counts near 2^31: n_E n_S is not a double exactly, so the product's
    rounding and the division decide the propensities."""
    model = W.flat_model(3, [({0: 1, 2: 1}, {1: 1, 2: 1}), ({1: 1}, {0: 1})],
                         michaelis_menten={0: (0, 3.3e8), 1: (1, 7.0)})
    rates = np.array([[1e-9, 0.7]])
    init = np.array([[2 ** 31 - 9, 2 ** 30, 2 ** 31 - 101]], np.int32)
    b = W.Batch(model, rates, init, W.uniform_grid(20.0, 8), 64, 13)
    g, o = check(b, log_cap=64)
    assert o["events"].min() > 10


def test_michaelis_menten_sensitivity_partials_match_oracle():
    """Score replay (h kept as doubles, changes integrated lazily) against the
    oracle's per-event integrals: the tolerance of the mass-action case."""
    b = W.mm_cascade(stages=20, R=64, G=12, T=2.0)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(21)
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


def test_tail_layout_refused_for_michaelis_menten_models():
    b = W.mm_cascade(stages=3, R=8, G=4, T=1.0)
    with pytest.raises(RuntimeError, match="mass-action"):
        gpu_run(b, layout=capi.CWC_LAYOUT_TAIL)


def test_checkpoint_resume_equals_one_launch():
    b = W.mm_cascade(stages=20, R=64, G=10, T=20.0)
    one = gpu_run(b, layout=capi.CWC_LAYOUT_QUEUE)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    sl, slices = api.simulate_sliced(cm, rates, init, grid, b.R, b.seed, b.max_events, slice_ns=200_000)
    torch.cuda.synchronize()
    assert np.array_equal(sl["states"].cpu().numpy().reshape(one["states"].shape), one["states"])
    assert np.array_equal(sl["hash"].cpu().numpy().reshape(-1).view(np.uint64), one["hash"])
