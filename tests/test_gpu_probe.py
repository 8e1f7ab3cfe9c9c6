"""The line-rate probe (asaga_probe_line_rate) and the floor it sets.

Every update whose row holds column v reads v's 8-byte state and then adds
to it (Algorithm 2's read of x^_v and write of x_v, abar_v); the L2 slice
that owns the line serialises those pairs.  The probe measures the time
per pair once the line is saturated, so an epoch of a problem whose most
frequent column is in c rows cannot take less than c times that.
"""
import numpy as np
import pytest

from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


def test_one_warp_sees_latency_and_many_warps_saturate_the_line():
    single = asaga.asaga_probe_line_rate(1, 2000)
    many = asaga.asaga_probe_line_rate(2048, 500)
    assert np.isfinite(single) and np.isfinite(many) and many > 0
    # one warp waits a full round trip per pair; 2048 warps queue at the line
    assert single > 20 * many, (single, many)
    # the line's service time is at least a cycle or so, far below a round trip
    assert 0.2 < many < 50.0, many


def test_the_update_kernel_does_not_beat_the_line_floor():
    p = synth.rcv1_like(seed=3, n=60000, d=6000)
    c_max = int(np.bincount(p.col_idx, minlength=p.d).max())
    assert c_max > 0.95 * p.n  # the frequent column is in almost every row
    ns = asaga.asaga_probe_line_rate(2048, 500)
    floor_s = c_max * ns * 1e-9
    with asaga.Context(p, storage="f32", seed=1, max_warps=512, gamma=0.05) as c:
        asaga.asaga_run(c.ctx, 2)  # warm-up
        _, r = asaga.asaga_run(c.ctx, 6)
    per_epoch = r.solver_seconds / r.epochs
    # the update launches of an epoch cannot serve the hot line faster than
    # the probe's saturated rate (slack for run-to-run noise)
    assert floor_s <= 1.25 * per_epoch, (floor_s, per_epoch)
