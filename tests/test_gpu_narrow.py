"""GPU parity of the compartment forward with 16-bit term counts (term_bits = 16).

Such a call runs its terms with 16-bit counts first (half the slab bytes, so
that a full GPU's terms stay in L2); a trajectory whose count
would leave int16's range, during the run or already in its initial term,
is saved in a checkpoint record and finished by a 32-bit launch that
redraws the same event.  The results must equal the oracle's bit for bit
whether or not, and wherever, the hand-over happens, and the replica sums,
means and variances must add up across the two launches.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_2438_gb300 import api, capi
from paper_1010_2438_gb300 import workloads as W

from test_gpu_cwc import check
from test_gpu_flat import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_2438_gb300 import build
    build.build()
    capi.lib()


def _growth_model():
    """Inflow of A into the root (fast) and into label-1 compartments, a
    transport of A into them, and a dissolution that releases a
    compartment's A into the root: root and compartment counts cross 32767
    at different times in different replicas."""
    rules = [W.RuleSpec(W.LOCAL, 0, rhs_ctx={0: 1}),
             W.RuleSpec(W.LOCAL, 1, rhs_ctx={0: 1}),
             W.RuleSpec(W.PARENT_CHILD, 0, 1, lhs_ctx={0: 1}, rhs_child={0: 1}),
             W.RuleSpec(W.DISSOLVE, 0, 1, lhs_wrap={1: 1})]
    m = W.cwc_model(2, 2, 5, rules)
    img = W.empty_slot_image(m)
    img[0, 3 + 2 + 0] = 30000
    for c, a in ((1, 20000), (2, 32000), (3, 100)):
        img[c, :3] = [1, 1, 0]
        img[c, 3 + 1] = 1          # wrap token for DISSOLVE
        img[c, 3 + 2 + 0] = a
    return m, img


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_counts_crossing_16_bits_hand_over_bit_exact(lanes):
    m, img = _growth_model()
    rates = np.array([[3000.0, 200.0, 0.01, 0.02]])
    b = W.Batch(m, rates, img[None], np.array([0.0, 0.2, 0.5, 1.0, 2.0]), 64, 19, max_events=100000)
    g, o = check(b, log_cap=512, lanes=lanes, term_bits=16)
    root_a = o["states"][:, :, 0]
    assert root_a.max() > 32767 and root_a[:, 0].max() <= 32767    # crossed during the run
    assert np.all(o["status"] == oracle.ST_OK)


@pytest.mark.parametrize("lanes", [1, 4])
def test_initial_counts_above_16_bits_bit_exact(lanes):
    """Every replica's initial term already holds 70,000 A in one compartment;
    in sweep point 2 two compartments also hold 2^31 - 5 and 10 B, and when
    both dissolve the root's B overflows int32 itself: INT_OVERFLOW, decided
    by the 32-bit launch."""
    m, img = _growth_model()
    img = np.stack([img, img])
    img[:, 3, 3 + 2 + 0] = 70000
    img[1, 2, 3 + 2 + 1] = 2 ** 31 - 5
    img[1, 3, 3 + 2 + 1] = 10
    b = W.Batch(m, np.array([[50.0, 20.0, 0.01, 5.0], [50.0, 20.0, 0.01, 5.0]]), img.astype(np.int32),
                np.array([0.0, 0.1, 0.3]), 40, 23, max_events=100000)
    g, o = check(b, lanes=lanes, term_bits=16)
    assert np.any(o["status"] == oracle.ST_OK) and np.any(o["status"] == oracle.ST_INT_OVERFLOW)


def test_replica_means_and_variance_add_up_across_the_hand_over():
    """Grid points recorded by the 16-bit launch and by the 32-bit one go into
    the same exact sums: sums, 128-bit sums of squares, means, variances and
    intervals equal the oracle's replica statistics bit for bit."""
    m, img = _growth_model()
    rates = np.array([[3000.0, 200.0, 0.01, 0.02]])
    b = W.Batch(m, rates, img[None], np.array([0.0, 0.2, 0.5, 1.0, 2.0]), 96, 5, max_events=100000)
    g = gpu_run(b, sums=True, means=True, sumsq=True, variance=True, ci90=True, term_bits=16)
    o = oracle.simulate(b, threads=8)
    assert np.array_equal(g["states"], o["states"])
    s, q, var, ci = oracle.replica_stats(o["states"], b.P, b.R)
    assert np.array_equal(g["sums"], s.astype(np.int64))
    qq = g["sumsq"].view(np.uint64)
    assert np.array_equal(qq[..., 0].astype(object) + (qq[..., 1].astype(object) << 64), q)
    assert np.array_equal(g["variance"].view(np.int64), var.view(np.int64))
    assert np.array_equal(g["ci90"].view(np.int64), ci.view(np.int64))
    assert o["states"][:, :, 0].max() > 32767


def test_compartment_workload_runs_on_16_bit_terms_unchanged():
    """cwc3x24's counts stay below 32767, so every trajectory finishes in the
    16-bit launch; results equal the oracle for a ragged batch."""
    b = W.cwc3x24(R=77, G=50)
    check(b, lanes=4, term_bits=16)


def test_term_bits_argument_checks():
    b = W.cwc3x24(R=4, G=5)
    with pytest.raises(capi.CwcError, match="term_bits"):
        gpu_run(b, term_bits=8)
