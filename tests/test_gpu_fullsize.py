"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (automatic layout = device work queue, automatic block size): the GPU
runs the whole batch; the oracle recomputes sampled trajectories one by one
and they must agree bit for bit (grid states, hash, events, status, final
time).  Batch-wide outputs are checked through properties that hold at any
size (exact sums = column sums of the states; means = sums / R)."""
import numpy as np
import pytest
import torch

import oracle
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


def sample_indices(n, k, seed):
    rng = np.random.default_rng(seed)
    idx = set([0, n - 1]) | set(rng.integers(0, n, k - 2).tolist())
    return np.array(sorted(idx))


def check_sampled(batch, res, qs, threads=8):
    st = res["states"].reshape(batch.n_traj, batch.G, -1)
    q_t = torch.from_numpy(qs).cuda()
    g_states = st.index_select(0, q_t).cpu().numpy()
    g_hash = res["hash"].reshape(-1).index_select(0, q_t).cpu().numpy().view(np.uint64)
    g_ev = res["events"].reshape(-1).index_select(0, q_t).cpu().numpy()
    g_status = res["status"].reshape(-1).index_select(0, q_t).cpu().numpy()
    g_t = res["final_t"].reshape(-1).index_select(0, q_t).cpu().numpy()
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        outs = list(ex.map(lambda q: oracle.simulate(batch, int(q), int(q) + 1), qs))
    for i, o in enumerate(outs):
        assert np.array_equal(g_states[i], o["states"][0]), int(qs[i])
        assert g_hash[i] == o["hash"][0]
        assert g_ev[i] == o["events"][0]
        assert g_status[i] == o["status"][0]
        assert g_t[i].view(np.int64) == o["final_t"][0].view(np.int64)


def test_flat32x64_full_size_sampled():
    b = W.flat32x64()                       # 65,536 replicas x ~1e5 events, 1000-point grid
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    res = api.simulate(cm, rates, init, grid, b.R, b.seed, b.max_events, states=True, sums=True, means=True)
    torch.cuda.synchronize()
    assert torch.all(res["status"] == 0)
    ev = res["events"].double()
    assert 0.9e5 < ev.mean().item() < 1.1e5
    check_sampled(b, res, sample_indices(b.n_traj, 14, 1))
    # exact sums and means over the whole batch
    col = res["states"].reshape(b.R, b.G, -1).sum(dim=0, dtype=torch.int64)
    assert torch.equal(col, res["sums"][0])
    assert torch.equal(res["means"], res["sums"].double() / b.R)


def test_sweep256x256_full_size_sampled():
    b = W.sweep256x256()                    # 256 rate vectors x 256 replicas, lengths ~100x apart
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    res = api.simulate(cm, rates, init, grid, b.R, b.seed, b.max_events, states=True)
    torch.cuda.synchronize()
    ev = res["events"].double().mean(dim=1)
    assert ev.max().item() / ev.min().item() > 30.0
    # sample across sweep points, including the longest and shortest
    pmax, pmin = int(torch.argmax(ev)), int(torch.argmin(ev))
    qs = np.unique(np.concatenate([sample_indices(b.n_traj, 10, 2), [pmax * b.R + 3, pmin * b.R + 5]]))
    check_sampled(b, res, qs)
    # the tail layout (last trajectories finished by one warp each) gives the
    # whole batch bit for bit
    tail = api.simulate(cm, rates, init, grid, b.R, b.seed, b.max_events, states=True,
                        layout=capi.CWC_LAYOUT_TAIL)
    torch.cuda.synchronize()
    for k in ("states", "status", "events", "hash", "final_t"):
        assert torch.equal(tail[k], res[k]), k


def test_flat16x24_full_size_forward_and_score_properties():
    b = W.flat16x24()                       # 131,072 replicas x ~1e4 events, 100-point grid
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    res = api.simulate(cm, rates, init, grid, b.R, b.seed, b.max_events, states=True, means=True)
    torch.cuda.synchronize()
    check_sampled(b, res, sample_indices(b.n_traj, 12, 3))
    m = res["means"]
    gm = torch.linspace(-1.0, 1.0, m.numel(), dtype=torch.float64, device="cuda").reshape(m.shape)
    sens = api.sensitivity(cm, rates, init, grid, b.R, b.seed, m, gm, partials=True)
    torch.cuda.synchronize()
    part = sens["partials"].reshape(b.R, -1)
    # the reduction is the mean of the per-trajectory partials
    ref = part.sum(dim=0) / b.R
    assert torch.allclose(sens["grad_rates"][0], ref, rtol=1e-10, atol=1e-12 * part.abs().max().item())
    # sampled partials against the oracle's replay of the same trajectories
    qs = sample_indices(b.n_traj, 8, 4)
    for q in qs:
        o = oracle.simulate(b, int(q), int(q) + 1, states=False, means=m.cpu().numpy(), grad_means=gm.cpu().numpy())
        got = part[int(q)].cpu().numpy()
        scale = np.abs(o["partials"][0]).mean() + 1e-300
        assert np.all(np.abs(got - o["partials"][0]) <= 1e-9 * (np.abs(o["partials"][0]) + scale))
