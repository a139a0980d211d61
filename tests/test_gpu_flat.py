"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Bit-exact on every integer and hash output and on the FP64 event times
(both sides follow the same written specification); the score replay is
compared within a tolerance derived from its FP64 rounding (see
test_sensitivity_partials_match_oracle).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def gpu_run(batch, **kw):
    cm = api.CompiledModel(batch.model)
    rates, init, grid = api.device_inputs(batch)
    res = api.simulate(cm, rates, init, grid, batch.R, batch.seed, batch.max_events, **kw)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items() if not k.startswith("_")}
    Q = batch.P * batch.R
    for k in ("status", "events", "final_t"):
        if k in out:
            out[k] = out[k].reshape(Q)
    if "hash" in out:
        out["hash"] = out["hash"].reshape(Q).view(np.uint64)
    if "states" in out:
        out["states"] = out["states"].reshape(Q, batch.G, -1)
    for k in ("log_rule", "log_slot", "log_t"):
        if k in out:
            out[k] = out[k].reshape(Q, -1)
    return out


def assert_same(g, o, keys=("status", "events", "hash", "final_t", "states")):
    for k in keys:
        a, b = g[k], o[k]
        if k == "final_t":
            assert np.array_equal(a.view(np.int64), b.view(np.int64)), k
        else:
            assert np.array_equal(a, b), (k, np.argwhere(a != b)[:5])


# ----------------------------------------------------------------------------

def _compile_curand_ref():
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "curand_philox_ref.so")
    src = os.path.join(ROOT, "tests", "cuda", "curand_philox_ref.cu")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", "-o", so, src], check=True)
    return ctypes.CDLL(so)


def test_oracle_philox_matches_curand():
    lib = _compile_curand_ref()
    rng = np.random.default_rng(1)
    n = 4096
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = rng.integers(0, 2, n)
    ctr[:, 2] = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    ctr[:, 3] = rng.integers(0, 2 ** 16, n)
    for seed in (0, 0x0123456789ABCDEF, 2 ** 64 - 1):
        out = np.zeros_like(ctr)
        assert lib.curand_ref(ctr.ctypes.data, ctypes.c_ulonglong(seed), out.ctypes.data, n) == 0
        ref = oracle.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
        assert np.array_equal(out, ref)


# ----------------------------------------------------------------------------

@pytest.mark.parametrize("layout", [capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE])
@pytest.mark.parametrize("threads", [32, 64, 128])
def test_flat8x12_bit_exact_with_event_log(layout, threads):
    b = W.flat8x12()                     # 64 replicas, ~1e4 events, 100-point grid
    cap = 256
    g = gpu_run(b, log_cap=cap, layout=layout, block_threads=threads)
    o = oracle.simulate(b, log_cap=cap, threads=8)
    assert_same(g, o)
    assert np.array_equal(g["log_rule"], o["log_rule"])
    assert np.array_equal(g["log_slot"], o["log_slot"])
    assert np.array_equal(g["log_t"].view(np.int64), o["log_t"].view(np.int64))
    assert np.all(g["status"] == oracle.ST_OK)


@pytest.mark.parametrize("name,R,scale", [("flat16x24", 333, 1.0), ("flat32x64", 97, 0.1)])
def test_flat_workloads_ragged_bit_exact(name, R, scale):
    """Several blocks and a ragged last block; flat32x64 with a tenth of its horizon."""
    b0 = getattr(W, name)(R=R)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * scale, R, b0.seed)
    for layout in (capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE):
        g = gpu_run(b, layout=layout)
        o = oracle.simulate(b, threads=8)
        assert_same(g, o)


def test_sweep_points_bit_exact():
    b0 = W.sweep256x256(P=7, R=9)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.05, b0.R, b0.seed)
    g = gpu_run(b, sums=True, means=True)
    o = oracle.simulate(b, threads=8)
    assert_same(g, o)
    sums = oracle.sums(o["states"], b.P, b.R)
    assert np.array_equal(g["sums"], sums)
    assert np.array_equal(g["means"].view(np.int64), (sums.astype(np.float64) / b.R).view(np.int64))


def test_init_per_sweep_point():
    b0 = W.flat8x12(R=5)
    P = 3
    rates = np.tile(b0.rates, (P, 1)) * np.array([[1.0], [0.5], [2.0]])
    init = np.stack([b0.init[0], b0.init[0] * 2, b0.init[0] // 2]).astype(np.int32)
    b = W.Batch(b0.model, rates, init, b0.grid * 0.2, 5, 77)
    assert_same(gpu_run(b), oracle.simulate(b))


# ----------------------------------------------------------------------------
# Edge cases and statuses
# ----------------------------------------------------------------------------

def test_single_trajectory_single_grid_point():
    b0 = W.flat8x12(R=1)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid[-1:].copy(), 1, 3)
    assert_same(gpu_run(b), oracle.simulate(b))
    b = W.Batch(b0.model, b0.rates, b0.init, np.array([0.0]), 1, 3)      # T = 0: no event
    g = gpu_run(b)
    assert_same(g, oracle.simulate(b))
    assert g["events"][0] == 0


def test_event_limit_zero_and_small():
    b0 = W.flat8x12(R=40)
    for me in (0, 1, 37):
        b = W.Batch(b0.model, b0.rates, b0.init, b0.grid, 40, b0.seed, max_events=me)
        g = gpu_run(b)
        assert_same(g, oracle.simulate(b))
        assert np.all(g["status"] == oracle.ST_EVENT_LIMIT)


def test_absorbed_int_overflow_prop_overflow_bad_input():
    death = W.flat_model(1, [({0: 1}, {})])
    cases = [
        W.Batch(death, np.array([[2.0]]), np.array([[30]], np.int32), np.array([0.0, 100.0]), 50, 3),
        W.Batch(W.birth_death(), np.array([[1e6, 1e-9]]), np.array([[2 ** 31 - 3]], np.int32),
                np.array([0.0, 1.0]), 10, 1),
        W.Batch(W.dimerisation(), np.array([[1e300, 1.0]]), np.array([[2 ** 30, 0]], np.int32),
                np.array([0.0, 1.0]), 10, 1),
        W.Batch(W.birth_death(), np.array([[-1.0, 1.0]]), np.array([[3]], np.int32), np.array([0.0, 1.0]), 4, 1),
        W.Batch(W.birth_death(), np.array([[1.0, np.nan]]), np.array([[3]], np.int32), np.array([0.0, 1.0]), 4, 1),
        W.Batch(W.birth_death(), np.array([[1.0, 1.0]]), np.array([[3]], np.int32), np.array([0.0, 0.0]), 4, 1),
        W.Batch(W.birth_death(), np.array([[1.0, 1.0]]), np.array([[3]], np.int32), np.array([-1.0, 1.0]), 4, 1),
        W.Batch(W.birth_death(), np.array([[1.0, 1.0]]), np.array([[-3]], np.int32), np.array([0.0, 1.0]), 4, 1),
        W.Batch(W.birth_death(), np.array([[1.0, 1.0]]), np.array([[3]], np.int32), np.array([0.0, np.inf]), 4, 1),
    ]
    expect = [oracle.ST_ABSORBED, oracle.ST_INT_OVERFLOW, oracle.ST_PROP_OVERFLOW] + [oracle.ST_BAD_INPUT] * 6
    for b, st in zip(cases, expect):
        g = gpu_run(b, sums=True)
        o = oracle.simulate(b)
        assert_same(g, o)
        assert np.all(g["status"] == st), (st, g["status"])
        assert np.array_equal(g["sums"], oracle.sums(o["states"], b.P, b.R))


def test_deadline_stops_with_timeout_status():
    b0 = W.flat32x64(R=4096)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 100.0, b0.R, b0.seed)   # ~1e7 events each
    g = gpu_run(b, deadline_ns=20_000_000, layout=capi.CWC_LAYOUT_QUEUE)
    assert np.all(g["status"] == capi.CWC_TRAJ_TIMEOUT)
    # the trajectories that ran are a prefix of the exact ones: oracle with the same event count
    q = int(np.argmax(g["events"]))
    o = oracle.simulate(b, q, q + 1, max_events=int(g["events"][q]))
    assert o["hash"][0] == g["hash"][q]


def test_argument_errors_do_not_launch():
    b = W.flat8x12(R=2)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    with pytest.raises(capi.CwcError):
        api.simulate(cm, rates, init, grid, 0, 1)
    with pytest.raises(capi.CwcError):
        api.simulate(cm, rates, init, grid, 2, 1, max_events=2 ** 32)
    a = api._sim_args(cm, rates, init, grid, 2, 1, 10, capi.CWC_LAYOUT_QUEUE, 0, 0)
    with pytest.raises(capi.CwcError, match="WORKSPACE"):
        capi.cwc_simulate(cm.handle, a, 0)


# ----------------------------------------------------------------------------
# Score replay
# ----------------------------------------------------------------------------

def test_sensitivity_partials_match_oracle():
    """Per-trajectory score contractions vs the oracle.  Both sides evaluate
    the same formula on the same path; the integral int H_j dt is accumulated
    lazily on the GPU (only when H_j changes) and at every event in the
    oracle, so values differ by FP64 rounding only: |d| <= 1e-9 * (|x| + s),
    s = the mean magnitude of the partials (~1e4 additions of terms of that
    size, each off by <= 1 ulp)."""
    b0 = W.flat8x12(R=96, G=12)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.25, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(3)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, b.model.n_observables))).cuda()
    res = api.sensitivity(cm, rates, init, grid, b.R, b.seed, means, gm, partials=True)
    torch.cuda.synchronize()
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    ograd, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))
    gg = res["grad_rates"].cpu().numpy()
    assert np.all(np.abs(gg - ograd) <= 1e-9 * (np.abs(ograd) + scale))


def test_sensitivity_after_propensity_overflow_matches_oracle():
    """A birth-death process whose total propensity overflows to +inf once the
    count reaches 2 (k_death = 1e308): most trajectories stop with
    PROP_OVERFLOW part-way through the grid.  The score's integrals then stop
    at the last applied event and H counts as zero after it (the oracle's
    convention); the partials must agree to the same tolerance as above."""
    model = W.birth_death()
    rates = np.array([[1e307, 1e308]])
    init = np.array([[1]], np.int32)
    b = W.Batch(model, rates, init, W.uniform_grid(1e-305, 9), 128, 23)
    cm = api.CompiledModel(b.model)
    rates_d, init_d, grid_d = api.device_inputs(b)
    means = torch.from_numpy(oracle.mean_observables(b, threads=8)).cuda()
    rng = np.random.default_rng(5)
    gm = torch.from_numpy(rng.standard_normal((1, b.G, b.model.n_observables))).cuda()
    res = api.sensitivity(cm, rates_d, init_d, grid_d, b.R, b.seed, means, gm, partials=True)
    torch.cuda.synchronize()
    st = oracle.simulate(b, states=False, threads=8)["status"]
    assert np.sum(st == capi.CWC_TRAJ_PROP_OVERFLOW) >= b.R // 2
    gp = res["partials"].cpu().numpy().reshape(b.R, -1)
    ograd, op = oracle.sensitivity(b, means.cpu().numpy(), gm.cpu().numpy(), threads=8)
    scale = np.mean(np.abs(op))
    assert scale > 0
    assert np.all(np.abs(gp - op) <= 1e-9 * (np.abs(op) + scale))


def test_autograd_function_forward_and_backward():
    b0 = W.flat8x12(R=256, G=10)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.1, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    k = rates.clone().requires_grad_(True)
    m = api.mean_observables(k, cm, init, grid, b.R, b.seed)
    om = oracle.mean_observables(b, threads=8)
    assert np.array_equal(m.detach().cpu().numpy().view(np.int64), om.view(np.int64))
    w = torch.linspace(-1, 1, m.numel(), dtype=torch.float64, device="cuda").reshape(m.shape)
    (m * w).sum().backward()
    direct = api.sensitivity(cm, rates, init, grid, b.R, b.seed, m.detach(), w)["grad_rates"]
    torch.cuda.synchronize()
    assert torch.equal(k.grad, direct)
    og, _ = oracle.sensitivity(b, om, w.cpu().numpy(), threads=8)
    assert np.allclose(k.grad.cpu().numpy(), og, rtol=1e-9, atol=1e-9 * np.abs(og).max())


def test_sensitivity_deterministic():
    b = W.flat16x24(R=2048, G=20)
    b = W.Batch(b.model, b.rates, b.init, b.grid * 0.1, b.R, b.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    m = api.simulate(cm, rates, init, grid, b.R, b.seed, states=False, means=True, traj=False)["means"]
    gm = torch.ones_like(m)
    g1 = api.sensitivity(cm, rates, init, grid, b.R, b.seed, m, gm)["grad_rates"]
    g2 = api.sensitivity(cm, rates, init, grid, b.R, b.seed, m, gm, layout=capi.CWC_LAYOUT_STATIC)["grad_rates"]
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)


def test_huge_counts_exercise_int64_to_double_rounding():
    """Combinatorial counts above 2^53 (C(n,2), n*m with n ~ 2^30): the
    propensity's int64 -> double conversion rounds, and any difference from
    round-to-nearest-even would change a0 and so every event time."""
    n = (1 << 30) + 12345
    cases = [
        W.Batch(W.dimerisation(), np.array([[1e-12, 1e-3]]), np.array([[n, 7]], np.int32), np.array([0.0, 1e9]), 64,
                11, max_events=300),
        W.Batch(W.heterodimer(), np.array([[3e-13, 2.5]]), np.array([[n, n - 999, 5]], np.int32),
                np.array([0.0, 1e9]), 64, 12, max_events=300),
        W.Batch(W.heterodimer(), np.array([[3e-13, 2.5]]), np.array([[(1 << 31) - 2, (1 << 31) - 5, 5]], np.int32),
                np.array([0.0, 1e9]), 64, 13, max_events=300),
    ]
    for b in cases:
        g = gpu_run(b, log_cap=300)
        o = oracle.simulate(b, log_cap=300)
        assert_same(g, o)
        assert np.array_equal(g["log_t"].view(np.int64), o["log_t"].view(np.int64))


def test_replica_offset_shards_reproduce_one_batch():
    b_full = W.flat8x12(R=96)
    o = oracle.simulate(b_full)
    for off, cnt in ((0, 40), (40, 56), (17, 9)):
        b = W.Batch(b_full.model, b_full.rates, b_full.init, b_full.grid, cnt, b_full.seed)
        g = gpu_run(b, replica_offset=off)
        sub = {k: v[off:off + cnt] for k, v in o.items()}
        assert_same(g, sub)


def test_replica_variance_and_interval_bit_exact():
    for b in (W.sweep256x256(P=3, R=50), W.flat8x12(R=1), W.flat8x12(R=33)):
        b = W.Batch(b.model, b.rates, b.init, b.grid * 0.05, b.R, b.seed)
        g = gpu_run(b, sums=True, means=True, sumsq=True, variance=True, ci90=True)
        o = oracle.simulate(b, threads=8)
        s, q, var, ci = oracle.replica_stats(o["states"], b.P, b.R)
        assert np.array_equal(g["sums"], s.astype(np.int64))
        qq = g["sumsq"].view(np.uint64)
        got_q = qq[..., 0].astype(object) + (qq[..., 1].astype(object) << 64)
        assert np.array_equal(got_q, q)
        assert np.array_equal(g["variance"].view(np.int64), var.view(np.int64))
        assert np.array_equal(g["ci90"].view(np.int64), ci.view(np.int64))
        # variance and the interval alone (sums and squares in the workspace)
        g2 = gpu_run(b, variance=True, ci90=True)
        assert np.array_equal(g2["variance"].view(np.int64), var.view(np.int64))


@pytest.mark.parametrize("n", [2, 5, 32, 33])
def test_lotka_volterra_chain_bit_exact(n):
    """The paper's n-species Lotka-Volterra family; n = 33 gives 34 rules,
    i.e. two-rule leaf blocks with a ragged last block."""
    b = W.lotka_volterra(n, R=48, G=20, T=0.05)
    g = gpu_run(b, log_cap=64)
    o = oracle.simulate(b, threads=8, log_cap=64)
    assert_same(g, o)
    assert np.array_equal(g["log_rule"], o["log_rule"])


def test_checkpoint_resume_reproduces_the_uninterrupted_run():
    """Stop every trajectory on a short deadline, then resume from the
    checkpoints until none is left: states, hashes, event counts and final
    times equal an uninterrupted run bit for bit (Sec. 5.2: instances that can
    be stopped and restarted)."""
    b0 = W.flat32x64(R=2048)
    b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.3, b0.R, b0.seed)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    ref = api.simulate(cm, rates, init, grid, b.R, b.seed)
    out = api.simulate(cm, rates, init, grid, b.R, b.seed, checkpoint=True, deadline_ns=3_000_000,
                       layout=capi.CWC_LAYOUT_QUEUE)
    torch.cuda.synchronize()
    first = int((out["status"] == capi.CWC_TRAJ_TIMEOUT).sum())
    assert first > 0
    rounds = 0
    while bool((out["status"] == capi.CWC_TRAJ_TIMEOUT).any()):
        out = api.simulate(cm, rates, init, grid, b.R, b.seed, resume=True, deadline_ns=3_000_000,
                           layout=capi.CWC_LAYOUT_QUEUE, out=out)
        torch.cuda.synchronize()
        rounds += 1
        assert rounds < 400
    assert rounds > 0
    for k in ("states", "events", "hash", "status", "final_t"):
        assert torch.equal(out[k], ref[k]), k


def test_checkpoint_argument_rules():
    b = W.flat8x12(R=4)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    with pytest.raises(capi.CwcError, match="reductions"):
        api.simulate(cm, rates, init, grid, b.R, b.seed, checkpoint=True, sums=True)
    a = api._sim_args(cm, rates, init, grid, b.R, b.seed, 10, capi.CWC_LAYOUT_STATIC, 0, 0)
    a.resume = 1
    with pytest.raises(capi.CwcError, match="checkpoint"):
        capi.cwc_simulate(cm.handle, a, 0)


def test_extreme_rate_spreads_bit_exact():
    """Rates from the smallest subnormal to 1e20 in one network: propensity
    sums with subnormal and huge terms, near-empty subtrees in the descent
    and an event cap (EVENT_LIMIT) all match the oracle bit for bit."""
    b0 = W.flat8x12(R=16)
    rng = np.random.default_rng(77)
    choices = np.array([5e-324, 1e-310, 1e-300, 1e-20, 1.0, 3.7, 1e20])
    rates = choices[rng.integers(0, len(choices), (3, b0.model.n_rules))]
    for p in range(3):
        if not np.any(rates[p] >= 1.0):
            rates[p, 0] = 1.0
    b = W.Batch(b0.model, rates, b0.init, b0.grid, b0.R, b0.seed, max_events=3000)
    g = gpu_run(b, log_cap=64)
    o = oracle.simulate(b, threads=8, log_cap=64)
    assert_same(g, o)
    valid = np.arange(64)[None, :] < np.minimum(o["events"], 64)[:, None]
    assert np.array_equal(g["log_rule"][valid], o["log_rule"][valid])
    assert np.any(o["status"] == oracle.ST_EVENT_LIMIT)
