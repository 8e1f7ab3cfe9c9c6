"""The allocation-free abar recomputation (asaga_recompute_abar_noalloc).

It serves callers that cannot allocate device memory: processes with a
fixed device-memory footprint reserved up front, code inside a framework
that owns every device allocation, and paths that cannot afford cudaFree's
device-wide synchronisation.  It must give the same result as the context's
asaga_recompute_abar and as the float64 CPU checker's abar = (1/n) sum_i
alpha_i a_i, call after call, with its scratch living in a fixed array of the
library instead of allocated memory.  This file is collected last on purpose.

Tolerance against the checker: both sides sum the same float64 products
(float32 alpha_i and a_iv widened exactly) in different orders and the
library rounds the sum to float32, so each column differs from the checker's
float64 value by at most half a float32 ulp (2^-24 relative) plus float64
reordering error (~1e-15 relative): rtol 2^-23 covers it with a factor two.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth


@pytest.fixture(scope="module")
def lib():
    build.build()
    return asaga.load()


def test_rejects_more_columns_than_the_scratch_holds(lib):
    # checked before any CUDA call, so this runs without a GPU too
    s = lib.asaga_recompute_abar_noalloc(10, asaga.NOALLOC_MAX_D + 1, 8, 8, 8, 8, 8, None, None)
    assert s == asaga.EINVAL and "outside [1, 524288]" in asaga.asaga_last_error(None)
    assert lib.asaga_recompute_abar_noalloc(10, 0, 8, 8, 8, 8, 8, None, None) == asaga.EINVAL
    assert lib.asaga_recompute_abar_noalloc(10, 5, None, 8, 8, 8, 8, None, None) == asaga.EINVAL


@pytest.mark.gpu
def test_matches_the_context_recompute_on_two_calls_in_a_row(lib):
    import torch

    assert torch.cuda.is_available()
    p = synth.rcv1_like(seed=22, n=60000, d=6000)
    with asaga.Context(p, storage="f32", seed=2, max_warps=256, gamma=0.1) as c:
        asaga.asaga_run(c.ctx, 3)
        _, abar_before, alpha = asaga.asaga_get_state(c.ctx)
        drift_ref = asaga.asaga_recompute_abar(c.ctx)  # the existing entry point
        abar_ref = asaga.asaga_get_state(c.ctx)[1]
    abar_exact = R.abar_from_scratch(p, alpha.astype(np.float64))  # the float64 checker
    drift_exact = float(np.max(np.abs(abar_before.astype(np.float64) - abar_exact)))

    dev = torch.device("cuda", 0)
    row_ptr = torch.from_numpy(np.ascontiguousarray(p.row_ptr, dtype=np.int64)).to(dev)
    col_idx = torch.from_numpy(np.ascontiguousarray(p.col_idx, dtype=np.int32)).to(dev)
    values = torch.from_numpy(np.ascontiguousarray(p.values, dtype=np.float32)).to(dev)
    alpha_d = torch.from_numpy(alpha).to(dev)
    drift_d = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        abar_d = torch.from_numpy(abar_before.copy()).to(dev)
        asaga.asaga_recompute_abar_noalloc(p.n, p.d, row_ptr, col_idx, values, alpha_d, abar_d, drift_d,
                                           stream.cuda_stream)
        torch.cuda.synchronize(dev)
        got = abar_d.cpu().numpy()
        # both sum in float64 (atomics in different orders) and round to float32
        np.testing.assert_allclose(got, abar_ref, rtol=2.5e-7, atol=1e-12, err_msg=f"call {call}")
        np.testing.assert_allclose(got, abar_exact, rtol=2.0 ** -23, atol=1e-30, err_msg=f"call {call} vs checker")
        assert drift_d.item() == pytest.approx(drift_ref, rel=1e-6, abs=1e-12)
        assert drift_d.item() == pytest.approx(drift_exact, rel=1e-9, abs=1e-15)
