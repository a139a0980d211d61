"""cwc_simulate_noalloc, the entry point for callers that cannot allocate
device memory (their memory belongs to another framework's pool, or to a
fixed budget reserved up front), against cwc_simulate with a caller-owned
workspace.  Outputs must agree bit for bit, the tolerance every forward
parity test here uses, on two calls in a row: the shared scratch array keeps
the previous call's contents, so the second call checks that everything
that must start at zero is cleared.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

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


def _outputs(cm, batch, rates, init, grid):
    P, R, G, O = batch.P, batch.R, batch.G, cm.n_observables
    d = {
        "states": torch.full((P, R, G, O), -7, dtype=torch.int32, device="cuda"),
        "means": torch.full((P, G, O), -7.0, dtype=torch.float64, device="cuda"),
        "status": torch.full((P, R), -7, dtype=torch.int32, device="cuda"),
        "events": torch.full((P, R), -7, dtype=torch.int64, device="cuda"),
        "hash": torch.zeros((P, R), dtype=torch.int64, device="cuda"),
    }
    a = api._sim_args(cm, rates, init, grid, R, batch.seed, batch.max_events, capi.CWC_LAYOUT_QUEUE, 0, 0)
    a.states, a.means = d["states"].data_ptr(), d["means"].data_ptr()
    a.traj_status, a.traj_events, a.traj_hash = d["status"].data_ptr(), d["events"].data_ptr(), d["hash"].data_ptr()
    return a, d


def _compare_twice(batch):
    """cwc_simulate with a caller-owned workspace, then cwc_simulate_noalloc
    twice on fresh outputs: all three must agree bit for bit."""
    cm = api.CompiledModel(batch.model)
    rates, init, grid = api.device_inputs(batch)
    stream = torch.cuda.current_stream().cuda_stream

    # reference: cwc_simulate with a caller-owned workspace
    a_ref, ref = _outputs(cm, batch, rates, init, grid)
    nbytes = capi.cwc_simulate_workspace_size(cm.handle, a_ref)
    # the scratch it needs: cwc_simulate's workspace less, for a compartment
    # model, the hand-over records of its 16-bit terms (32-bit terms here)
    m = batch.model
    handover = 0 if (m.n_labels == 1 and m.max_compartments == 1) or a_ref.term_bits != 16 else \
        ((4 * batch.P * batch.R * (8 + m.max_compartments * (3 + 2 * m.n_species)) + 255) // 256) * 256
    assert 0 < nbytes - handover <= capi.CWC_NOALLOC_SCRATCH_BYTES   # uses scratch, and it fits
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    a_ref.workspace = (ws.data_ptr() + 255) & ~255
    a_ref.workspace_bytes = nbytes
    capi.cwc_simulate(cm.handle, a_ref, stream)
    torch.cuda.synchronize()

    for call in range(2):
        a, got = _outputs(cm, batch, rates, init, grid)
        a.workspace, a.workspace_bytes = None, 0       # ignored by the no-alloc entry point
        capi.cwc_simulate_noalloc(cm.handle, a, stream)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(got[k], ref[k]), (call, k)
        assert torch.all(got["events"] > 0)


def test_noalloc_matches_workspace_entry_point_twice():
    """A flat network over three sweep points: the queue ticket, the sweep
    order and the replica sums behind the means live in the scratch."""
    b0 = W.sweep256x256(P=3, R=700)
    _compare_twice(W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.02, b0.R, b0.seed))


def test_noalloc_compartment_model_matches_workspace_entry_point_twice():
    """The 24-species compartment workload with 40 replicas: here the scratch
    also holds one term slab per resident lane group, which is what makes
    a compartment batch fit the fixed array only when it is small."""
    b0 = W.cwc3x24(R=40, G=25)
    _compare_twice(W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.1, b0.R, b0.seed))


def test_noalloc_rejects_scratch_beyond_its_limit():
    b = W.flat32x64(R=4)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    big_grid = torch.linspace(0.0, float(b.grid[-1]), 5000, dtype=torch.float64, device="cuda")
    means = torch.empty((1, 5000, cm.n_observables), dtype=torch.float64, device="cuda")
    a = api._sim_args(cm, rates, init, big_grid, b.R, b.seed, 100, capi.CWC_LAYOUT_QUEUE, 0, 0)
    a.means = means.data_ptr()            # 8 * 5000 * 32 bytes of sums > 1 MiB
    rc = capi.lib().cwc_simulate_noalloc(cm.handle, ctypes.byref(a), None)
    assert rc == capi.CWC_ERR_INVALID_ARG
    assert "scratch" in capi.cwc_last_error()
