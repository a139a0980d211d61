"""The oracle's thread schedules give the single-thread run bit for bit.

`oracle.simulate(threads=n)` splits the trajectories over threads either
statically (one contiguous range per thread) or on demand (schedule="farm":
a thread takes the next unstarted trajectory whenever it finishes one, the
farm of independent simulation instances of Sec. 5.2 that the CPU baseline
times).  Every trajectory is a function of its own index q = p R + r only
(its Philox stream is keyed by (r, p)), so any split must reproduce the
one-thread run exactly: states, statuses, event counts, hashes, final times,
event logs and score partials.
"""
import numpy as np
import pytest

import oracle
from paper_1010_2438_gb300 import workloads as W


def _assert_same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].dtype == b[k].dtype and a[k].shape == b[k].shape, k
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def _uneven_sweep():
    """Four rate vectors of the 64-rule network, two decades apart in scale,
    so trajectory lengths differ by ~100x across sweep points."""
    b0 = W.sweep256x256(P=4, R=5, G=12)
    return W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.004, b0.R, b0.seed)


@pytest.mark.parametrize("schedule", ["static", "farm"])
@pytest.mark.parametrize("threads", [2, 3, 64])
def test_flat_sweep_split_equals_one_thread(schedule, threads):
    b = _uneven_sweep()
    one = oracle.simulate(b, threads=1, log_cap=32)
    ev = one["events"].reshape(b.P, b.R).mean(axis=1)
    assert ev.max() > 5 * ev.min() > 0          # the split really is uneven
    many = oracle.simulate(b, threads=threads, log_cap=32, schedule=schedule)
    _assert_same(one, many)


@pytest.mark.parametrize("schedule", ["static", "farm"])
def test_sub_range_and_score_partials(schedule):
    b = W.flat8x12(R=24, G=20)
    b = W.Batch(b.model, b.rates, b.init, b.grid * 0.1, b.R, b.seed)
    full = oracle.simulate(b, threads=1)
    means = oracle.sums(full["states"], b.P, b.R).astype(np.float64) / b.R
    gm = np.random.default_rng(3).standard_normal(means.shape)
    one = oracle.simulate(b, 5, 19, threads=1, means=means, grad_means=gm)
    many = oracle.simulate(b, 5, 19, threads=4, means=means, grad_means=gm, schedule=schedule)
    _assert_same(one, many)
    assert np.array_equal(one["states"], full["states"][5:19])
    assert np.any(one["partials"] != 0.0)


@pytest.mark.parametrize("schedule", ["static", "farm"])
def test_compartment_batch_split_equals_one_thread(schedule):
    c0 = W.cwc3x24(R=12, G=10)
    c = W.Batch(c0.model, c0.rates, c0.init, c0.grid * 0.1, c0.R, c0.seed)
    one = oracle.simulate(c, threads=1, log_cap=16)
    assert one["events"].min() > 0
    many = oracle.simulate(c, threads=5, log_cap=16, schedule=schedule)
    _assert_same(one, many)


def test_unknown_schedule_is_rejected():
    b = W.flat8x12(R=4, G=5)
    with pytest.raises(ValueError):
        oracle.simulate(b, threads=2, schedule="round-robin")
