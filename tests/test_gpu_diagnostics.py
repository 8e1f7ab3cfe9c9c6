"""The GPU diagnostics behind the paper's qualitative experiments, against the
float64 CPU checker, through the C ABI.

  * Overlap (App. E.2): the library's estimates of tau from a run's trace
    equal the checker's plain restatement of the estimator on the same trace
    (integer counts and their averages exactly; the mean window to 1e-12).
  * Epochs against concurrency (App. D.2): below the stability frontier the
    number of passes needed for a given suboptimality does not depend on the
    number of concurrent updates (the paper's 1- and 10-core curves coincide
    per iteration); at one step, 8 and 64 warps reach 1e-6 within a band of
    20% (+1 epoch) of each other.
"""
import json
import os

import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


@pytest.mark.parametrize("warps", [1, 64, 512])
def test_overlap_estimates_match_the_checker_on_the_same_trace(warps):
    p = synth.rcv1_like(seed=30, n=40000, d=4000)
    count = 10000  # a quarter epoch
    with asaga.Context(p, seed=1, max_warps=warps, gamma=0.01) as c:
        est, times = asaga.asaga_measure_overlap_trace(c.ctx, count / p.n, count)
    assert np.all(times[1::2] >= times[0::2]) and np.all(times > 0)
    ref = R.overlap_estimates(times)
    assert est["updates"] == ref["updates"] == count
    assert est["tau_mean"] == ref["tau_mean"]
    assert est["tau_max"] == ref["tau_max"]
    assert est["tau_paper"] == ref["tau_paper"]
    assert est["window_ns_mean"] == pytest.approx(ref["window_ns_mean"], rel=1e-12)
    if warps == 1:
        assert ref["tau_max"] == 0  # one core never overlaps itself
    else:
        assert ref["tau_paper"] >= ref["tau_mean"] > 0


def test_trace_buffer_must_hold_the_trace():
    p = synth.small_logistic()
    with asaga.Context(p, seed=1) as c:
        with pytest.raises(asaga.AsagaError) as e:
            asaga.asaga_measure_overlap_trace(c.ctx, 1.0, p.n // 2)  # room for half the updates
        assert e.value.status == asaga.EINVAL


def test_epochs_to_target_do_not_depend_on_warps_below_the_frontier():
    p = synth.rcv1_like(seed=22, n=60000, d=6000)
    cert = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-10)
    epochs = {}
    for warps in (8, 64):
        with asaga.Context(p, seed=3, max_warps=warps, abar_recompute_every=5) as c:
            s, r = asaga.asaga_run(c.ctx, 150, 1e-6, cert["fstar"])
        assert s == asaga.OK, (warps, asaga.STATUS_NAMES[s], r.as_dict())
        epochs[warps] = r.epochs
    assert abs(epochs[8] - epochs[64]) <= 0.2 * max(epochs.values()) + 1, epochs
