"""GPU parity for compartmentalised CWC models (transport, wrap binding,
creation and dissolution of compartments) against the oracle, bit for bit:
label-aggregated observables, statuses, event counts, (rule, slot) hashes,
final times and event logs."""
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


def check(batch, threads=8, **kw):
    g = gpu_run(batch, **kw)
    o = oracle.simulate(batch, threads=threads, log_cap=kw.get("log_cap", 0))
    assert_same(g, o)
    cap = kw.get("log_cap", 0)
    if cap:
        # entries past a trajectory's last event are not written by the GPU
        valid = np.arange(cap)[None, :] < np.minimum(o["events"], cap)[:, None]
        assert np.array_equal(g["log_rule"][valid], o["log_rule"][valid])
        assert np.array_equal(g["log_slot"][valid], o["log_slot"][valid])
        assert np.array_equal(g["log_t"].view(np.int64)[valid], o["log_t"].view(np.int64)[valid])
    return g, o


@pytest.mark.parametrize("layout,lanes", [(capi.CWC_LAYOUT_STATIC, 1), (capi.CWC_LAYOUT_QUEUE, 1),
                                          (capi.CWC_LAYOUT_STATIC, 4), (capi.CWC_LAYOUT_QUEUE, 8)])
def test_cwc3x24_bit_exact_with_event_log(layout, lanes):
    """One lane or a group of 4 / 8 lanes per term give the oracle's events."""
    b = W.cwc3x24(R=48)
    g, o = check(b, log_cap=512, layout=layout, lanes=lanes)
    assert np.all(g["status"] == oracle.ST_OK)


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_cwc3x24_structural_events_occur_and_match(lanes):
    """Longer horizon so that creations and dissolutions certainly happen."""
    b0 = W.cwc3x24(R=24, G=50)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 3.0, b0.R, b0.seed)
    g, o = check(b, log_cap=40000, lanes=lanes)
    lr = o["log_rule"]
    kinds = b.model.kind[lr[lr >= 0]]
    assert np.sum(kinds == W.CREATE) > 0 and np.sum(kinds == W.DISSOLVE) > 0


def _transport(n_children=2):
    rules = [W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_ctx={0: 1}, rhs_child={0: 1}),
             W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_child={0: 1}, rhs_ctx={0: 1})]
    m = W.cwc_model(1, 2, 1 + n_children, rules)
    img = W.empty_slot_image(m)
    img[0, 4] = 40
    for d in range(1, n_children + 1):
        img[d, :3] = [1, 1, 0]
    return m, img


@pytest.mark.parametrize("lanes", [1, 8])
def test_law_models_bit_exact(lanes):
    m, img = _transport()
    check(W.Batch(m, np.array([[0.4, 1.1]]), img[None], np.array([0.0, 0.2, 0.6, 1.5, 6.0]), 300, 8), log_cap=64,
          lanes=lanes)
    # create / dissolve with a conserved token
    rules = [W.RuleSpec(W.CREATE, 0, 1, lhs_ctx={0: 1}, rhs_wrap={0: 1}), W.RuleSpec(W.DISSOLVE, 0, 1)]
    m = W.cwc_model(1, 2, 13, rules)
    img = W.empty_slot_image(m)
    img[0, 4] = 12
    check(W.Batch(m, np.array([[0.9, 0.5]]), img[None], np.array([0.0, 0.3, 1.0, 3.0, 10.0]), 300, 9), log_cap=64,
          lanes=lanes)
    # dissolution reparents a label-2 child to the top, which a transport rule then drains
    rules = [W.RuleSpec(W.DISSOLVE, 0, 1), W.RuleSpec(W.PARENT_CHILD, 0, 2, lhs_child={0: 1}, rhs_ctx={0: 1})]
    m = W.cwc_model(1, 3, 3, rules)
    img = W.empty_slot_image(m)
    img[1, :3] = [1, 1, 0]
    img[2, :3] = [1, 2, 1]
    img[2, 4] = 5
    g, _ = check(W.Batch(m, np.array([[1.0, 1.0]]), img[None], np.array([0.0, 200.0]), 64, 10), log_cap=8,
                 lanes=lanes)
    assert np.all(g["status"] == oracle.ST_ABSORBED)


@pytest.mark.parametrize("lanes", [1, 8])
def test_capacity_and_bad_slot_images(lanes):
    rules = [W.RuleSpec(W.CREATE, 0, 1, lhs_ctx={0: 1})]
    m = W.cwc_model(1, 2, 3, rules)
    img = W.empty_slot_image(m)
    img[0, 4] = 10
    g, _ = check(W.Batch(m, np.array([[1.0]]), img[None], np.array([0.0, 1e6]), 4, 11), lanes=lanes)
    assert np.all(g["status"] == oracle.ST_CAPACITY)
    m, good = _transport(2)
    bads = []
    x = good.copy(); x[0, 0] = 0; bads.append(x)            # root not alive
    x = good.copy(); x[1, 1] = 0; bads.append(x)            # child with the top label
    x = good.copy(); x[1, 1] = 5; bads.append(x)            # label out of range
    x = good.copy(); x[1, 2] = 2; x[2, 2] = 1; bads.append(x)   # parent cycle
    x = good.copy(); x[2, 4] = -1; bads.append(x)           # negative count
    x = good.copy(); x[0, 3] = 1; bads.append(x)            # root with a wrap
    x = good.copy(); x[1, 0] = 2; bads.append(x)            # alive flag not 0/1
    x = good.copy(); x[1, 2] = 7; bads.append(x)            # parent out of range
    for img in bads:
        g, _ = check(W.Batch(m, np.array([[0.4, 1.1]]), img[None], np.array([0.0, 1.0]), 3, 1), lanes=lanes)
        assert np.all(g["status"] == oracle.ST_BAD_INPUT)


def test_flat_network_through_the_compartment_kernel_matches_the_flat_kernel():
    """A flat network declared with a spare label and slot runs the
    compartment kernel; its top-level totals, events, hashes and times equal
    the flat kernel's."""
    b = W.flat8x12(R=40)
    mf = b.model
    mc = W.Model(mf.n_species, 2, 2, mf.kind, mf.ctx_label, mf.child_label, mf.lhs, mf.rhs)
    img = W.empty_slot_image(mc)
    img[0, 3 + mf.n_species:] = b.init[0]
    bc = W.Batch(mc, b.rates, img[None], b.grid, b.R, b.seed)
    gf = gpu_run(b)
    gc = gpu_run(bc)
    S = mf.n_species
    assert np.array_equal(gc["states"][:, :, :S], gf["states"])
    for k in ("events", "hash", "status"):
        assert np.array_equal(gc[k], gf[k])
    assert np.array_equal(gc["final_t"].view(np.int64), gf["final_t"].view(np.int64))
    assert_same(gc, oracle.simulate(bc, threads=8))


def test_cwc3x24_full_size_sampled():
    from test_gpu_fullsize import check_sampled, sample_indices
    b = W.cwc3x24()                          # 16,384 replicas, 500-point grid, 172 observables
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    res = api.simulate(cm, rates, init, grid, b.R, b.seed, b.max_events, states=True, sums=True)
    torch.cuda.synchronize()
    assert torch.all(res["status"] == 0)
    check_sampled(b, res, sample_indices(b.n_traj, 10, 7))
    col = res["states"].reshape(b.R, b.G, -1).sum(dim=0, dtype=torch.int64)
    assert torch.equal(col, res["sums"][0])


def test_cwc_replica_variance_and_interval_bit_exact():
    b0 = W.cwc3x24(R=40, G=10)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.2, b0.R, b0.seed)
    g = gpu_run(b, variance=True, ci90=True, means=True)
    o = oracle.simulate(b, threads=8)
    s, q, var, ci = oracle.replica_stats(o["states"], b.P, b.R)
    assert np.array_equal(g["variance"].view(np.int64), var.view(np.int64))
    assert np.array_equal(g["ci90"].view(np.int64), ci.view(np.int64))


@pytest.mark.parametrize("lanes", [1, 4])
def test_cwc_sensitivity_partials_match_oracle(lanes):
    """Score replay on a compartment model (structural events included):
    per-trajectory partials within 1e-9 * (|x| + mean |x|) of the oracle (the
    integral of H_j is accumulated lazily on the GPU and at every event in the
    oracle, so they differ by FP64 rounding only)."""
    b0 = W.cwc3x24(R=32, G=8)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.5, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(11)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, cm.n_observables)) * 1e-3).cuda()
    res = api.sensitivity(cm, rates, init, grid, b.R, b.seed, means, gm, partials=True, lanes=lanes)
    torch.cuda.synchronize()
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    ograd, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert scale > 0
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))
    gg = res["grad_rates"].cpu().numpy()
    assert np.all(np.abs(gg - ograd) <= 1e-9 * (np.abs(ograd) + scale))


@pytest.mark.parametrize("lanes", [1, 4])
def test_cwc_sensitivity_after_propensity_overflow_matches_oracle(lanes):
    """Every rate scaled by f and the grid by 1/f keeps the dynamics but puts
    a0 at ~60 % of the largest double, so that most terms overflow it part-way
    through the grid.  The score's integrals then stop at the last applied
    event and H counts as zero after it (the oracle's convention); partials
    within the tolerance of the test above."""
    b0 = W.cwc3x24(R=32, G=8)
    f = 0.6 * 1.7976931348623157e308 / (9.6e3 / float(b0.grid[-1]))   # a0 ~ 9.6e3 / horizon
    b = W.Batch(b0.model, b0.rates * f, b0.init, b0.grid * 0.5 / f, b0.R, b0.seed)
    st = oracle.simulate(b, states=False, threads=8)["status"]
    assert np.sum(st == capi.CWC_TRAJ_PROP_OVERFLOW) >= b.R // 2
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(13)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, cm.n_observables)) * 1e-3).cuda()
    res = api.sensitivity(cm, rates, init, grid, b.R, b.seed, means, gm, partials=True, lanes=lanes)
    torch.cuda.synchronize()
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    _, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert scale > 0
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))


def test_cwc_autograd_function():
    b0 = W.cwc3x24(R=64, G=6)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.2, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    k = rates.clone().requires_grad_(True)
    m = api.mean_observables(k, cm, init, grid, b.R, b.seed)
    om = oracle.mean_observables(b, threads=8)
    assert np.array_equal(m.detach().cpu().numpy().view(np.int64), om.view(np.int64))
    (m * 0.001).sum().backward()
    og, _ = oracle.sensitivity(b, om, np.full(om.shape, 0.001), threads=8)
    assert np.allclose(k.grad.cpu().numpy(), og, rtol=1e-9, atol=1e-9 * np.abs(og).max())


def test_cwc_checkpoint_resume_reproduces_the_uninterrupted_run():
    """Compartment terms stopped on a short deadline and resumed from their
    saved slot images, until none is left, end bit-identical to an
    uninterrupted run (Sec. 5.2: instances stopped and restarted); the saved
    image of a finished trajectory is its final term."""
    b0 = W.cwc3x24(R=512, G=50)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 1.5, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    ref = api.simulate(cm, rates, init, grid, b.R, b.seed)
    out = api.simulate(cm, rates, init, grid, b.R, b.seed, checkpoint=True, deadline_ns=2_000_000,
                       layout=capi.CWC_LAYOUT_QUEUE)
    torch.cuda.synchronize()
    assert int((out["status"] == capi.CWC_TRAJ_TIMEOUT).sum()) > 0
    rounds = 0
    while bool((out["status"] == capi.CWC_TRAJ_TIMEOUT).any()):
        out = api.simulate(cm, rates, init, grid, b.R, b.seed, resume=True, deadline_ns=2_000_000,
                           layout=capi.CWC_LAYOUT_QUEUE, out=out)
        torch.cuda.synchronize()
        rounds += 1
        assert rounds < 2000
    assert rounds > 0
    for k in ("states", "events", "hash", "status", "final_t"):
        assert torch.equal(out[k], ref[k]), k
    # the saved terms give the last grid point's observables
    S, C, L = b.model.n_species, b.model.max_compartments, b.model.n_labels
    img = out["checkpoint"].cpu().numpy().reshape(b.R, 8 + C * (3 + 2 * S))[:, 8:].reshape(b.R, C, 3 + 2 * S)
    alive = img[:, :, 0] == 1
    lab = img[:, :, 1]
    last = ref["states"].cpu().numpy()[0, :, -1, :] if ref["states"].dim() == 4 else ref["states"].cpu().numpy()[:, -1, :]
    for l in range(L):
        m = alive & (lab == l)
        content = (img[:, :, 3 + S:] * m[:, :, None]).sum(axis=1)
        assert np.array_equal(np.minimum(content, 2**31 - 1), last[:, l * S:(l + 1) * S])
        assert np.array_equal(m.sum(axis=1), last[:, L * S + (L - 1) * S + l])
