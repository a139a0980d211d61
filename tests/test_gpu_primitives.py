"""The kernels' fixed logarithm against the oracle's, bit for bit, on the
uniforms the simulation draws (Sec. 2.2 step 2: tau = -ln(u) / a0)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def gpu_log(u):
    ud = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).cuda()
    out = torch.empty_like(ud)
    capi.cwc_log_spec(ud.data_ptr(), out.data_ptr(), ud.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_log_spec_gpu_equals_oracle_on_random_uniforms():
    rng = np.random.default_rng(2024)
    n = 1 << 22
    k = (rng.integers(0, 1 << 26, n, dtype=np.int64) << 26) | rng.integers(0, 1 << 26, n, dtype=np.int64)
    u = (2.0 * k + 1.0) * 2.0 ** -53           # (k + 1/2) 2^-52, exact
    g = gpu_log(u)
    o = oracle.log_spec(u)
    assert np.array_equal(g.view(np.int64), o.view(np.int64))


def test_log_spec_gpu_edges_and_range():
    sqrt2_half = np.sqrt(2.0) / 2.0
    edges = [2.0 ** -53, 3 * 2.0 ** -53, 2.0 ** -52 + 2.0 ** -53, 0.25, 0.5, 0.5 + 2.0 ** -53,
             1.0 - 2.0 ** -53, 1.0 - 3 * 2.0 ** -53, np.nextafter(sqrt2_half, 0), sqrt2_half,
             np.nextafter(sqrt2_half, 1)]
    # every binade of the uniforms, at its ends and around sqrt(2) inside it
    for e in range(-53, 0):
        b = 2.0 ** e
        edges += [b, np.nextafter(2 * b, 0), np.sqrt(2.0) * b, np.nextafter(np.sqrt(2.0) * b, 0)]
    u = np.array([x for x in edges if 2.0 ** -53 <= x < 1.0])
    g = gpu_log(u)
    assert np.array_equal(g.view(np.int64), oracle.log_spec(u).view(np.int64))
    bad = gpu_log(np.array([0.0, 1.0, 2.0 ** -54, -0.5, 2.0]))
    assert np.all(np.isnan(bad))


def test_log_spec_argument_errors():
    with pytest.raises(capi.CwcError):
        capi.cwc_log_spec(0, 0, -1)
    with pytest.raises(capi.CwcError):
        capi.cwc_log_spec(0, 0, 4)
