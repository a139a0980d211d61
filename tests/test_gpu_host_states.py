"""Grid states written by the kernel straight into page-locked host memory.

The C ABI accepts page-locked host memory for the states: the kernel stores
them across the host link while it runs, so an end-to-end call needs no copy
afterwards.  The states must equal those written to device memory bit for
bit, for flat and compartment models, and pageable memory is refused before
any launch.
"""
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


def _host_inputs(b):
    return (torch.from_numpy(np.ascontiguousarray(b.rates)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(b.init)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(b.grid)).pin_memory())


@pytest.mark.parametrize("name", ["flat32x64", "cwc3x24", "mm_cascade"])
def test_direct_host_states_equal_device_states(name):
    if name == "flat32x64":
        b0 = W.flat32x64(R=3000)
        b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.05, b0.R, b0.seed)
    elif name == "cwc3x24":
        b0 = W.cwc3x24(R=500, G=40)
        b = W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.2, b0.R, b0.seed)
    else:
        b = W.mm_cascade(stages=20, R=2000, G=30, T=5.0)
    cm = api.CompiledModel(b.model)
    rates_h, init_h, grid_h = _host_inputs(b)
    direct = api.simulate_host(cm, rates_h, init_h, grid_h, b.R, b.seed, b.max_events, direct=True)
    torch.cuda.synchronize()
    copied = api.simulate_host(cm, rates_h, init_h, grid_h, b.R, b.seed, b.max_events, direct=False)
    torch.cuda.synchronize()
    assert direct.device.type == "cpu" and direct.is_pinned()
    assert torch.equal(direct, copied)
    # a second direct call into the same buffer (reused outputs) gives the same states
    again = api.simulate_host(cm, rates_h, init_h, grid_h, b.R, b.seed, b.max_events, host_out=direct.clone().pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(again, copied)


def test_pageable_host_states_are_refused():
    b = W.flat8x12(R=16, G=8)
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    pageable = torch.empty((b.P, b.R, b.G, cm.n_observables), dtype=torch.int32)
    assert not pageable.is_pinned()
    with pytest.raises(capi.CwcError, match="pageable"):
        api.simulate(cm, rates, init, grid, b.R, b.seed, out={"states": pageable})
