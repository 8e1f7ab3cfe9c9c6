"""Compact storage of A (asaga_options.compact): uint16 column indices when
d <= 65536, one value per row when every stored value of each row is equal.

The kernels then read the same numbers in the same order, so a single-warp
in-order replay and the float64 objective must agree bit for bit with the
uncompacted layout (the float64 column scatters add atomics in no fixed
order: 1e-12); against the float64 oracle the replay tolerance is the usual
1e-4 relative l2."""
import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = {
    # binary rows scaled to unit norm, d <= 65536: one value per row and uint16 columns
    "binary_small_d": (lambda: synth.sparse_logistic(3000, 9000, k_mean=30, k_min=2, k_max=90, k_sigma=0.4,
                                                     zipf_s=1.1, values="binary", storage="bf16", seed=71),
                       "bf16", 2, 1),
    # binary rows, d > 65536: one value per row, int32 columns
    "binary_large_d": (lambda: synth.sparse_logistic(4000, 70000, k_mean=40, k_min=2, k_max=120, k_sigma=0.4,
                                                     zipf_s=1.1, values="binary", storage="bf16", seed=72),
                       "bf16", 4, 1),
    # general values, d <= 65536, rows beyond the 128 staged entries: uint16 columns only
    "long_rows_f32": (lambda: synth.sparse_logistic(2000, 4000, k_mean=120, k_min=1, k_max=900, k_sigma=1.0,
                                                    zipf_s=1.1, storage="f32", seed=73),
                      "f32", 2, 0),
    "fp16_values": (lambda: synth.sparse_logistic(3000, 2000, k_mean=25, k_min=1, k_max=200, k_sigma=0.6,
                                                  zipf_s=1.1, storage="f16", seed=74),
                    "f16", 2, 0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_compact_layout_replays_bit_for_bit(case):
    make, storage, want_idx_bytes, want_row_values = CASES[case]
    p = make()
    idx = synth.sample_indices(p.n, p.n, seed=75)
    out = {}
    for compact in (0, 1):
        with asaga.Context(p, storage=storage, compact=compact) as c:
            info = asaga.asaga_get_info(c.ctx)
            asaga.asaga_run_indices(c.ctx, idx)
            out[compact] = (asaga.asaga_get_state(c.ctx), asaga.asaga_objective(c.ctx),
                            asaga.asaga_full_grad(c.ctx), asaga.asaga_recompute_abar(c.ctx), info)
    (x0, ab0, al0), f0, (g0, n0), d0, i0 = out[0]
    (x1, ab1, al1), f1, (g1, n1), d1, i1 = out[1]
    assert (i0["col_index_bytes"], i0["row_values"]) == (4, 0)
    assert (i1["col_index_bytes"], i1["row_values"]) == (want_idx_bytes, want_row_values)
    assert i1["device_bytes"] < i0["device_bytes"]
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(ab1, ab0)
    np.testing.assert_array_equal(al1, al0)
    assert f1 == f0  # fixed-order reductions
    # the column scatters add float64 atomics in no fixed order
    np.testing.assert_allclose(g1, g0, rtol=1e-12, atol=1e-18)
    assert n1 == pytest.approx(n0, rel=1e-12)
    assert d1 == pytest.approx(d0, rel=1e-6, abs=1e-12)
    # and the oracle on the same rows
    st = R.sparse_saga(p, R.State.zeros(p), idx, i1["gamma"])
    assert rel(x1, st.x) <= 1e-4


def test_general_values_with_large_d_stay_uncompacted():
    p = synth.sparse_logistic(3000, 70000, k_mean=20, k_min=2, k_max=60, k_sigma=0.4, zipf_s=1.1,
                              storage="f32", seed=76)
    with asaga.Context(p, storage="f32", compact=1) as c:
        info = asaga.asaga_get_info(c.ctx)
    assert (info["col_index_bytes"], info["row_values"]) == (4, 0)


def test_compact_async_run_reaches_1e6():
    make = CASES["binary_small_d"][0]
    p = make()
    fs = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-11, max_epochs=3000,
                           check_every=5)
    with asaga.Context(p, storage="bf16", compact=1, seed=3, abar_recompute_every=5) as c:
        asaga.asaga_autotune(c.ctx)
        s, r = asaga.asaga_run(c.ctx, 500, 1e-6, fs["fstar"])
        x = asaga.asaga_get_state(c.ctx)[0]
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict())
    assert (R.objective(p, x.astype(np.float64)) - fs["fstar"]) / abs(fs["fstar"]) <= 1e-6 + fs["bound"]


def test_batch_compacts_what_every_instance_allows():
    ps = synth.logistic_batch(count=5, seed=77, n_range=(1500, 3000), d_range=(200, 1500),
                              density_range=(0.01, 0.03), lam_range=(1e-3, 1e-2), storage="bf16")
    fs = np.array([R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-11,
                                     max_epochs=2000, check_every=5)["fstar"] for p in ps])
    with asaga.Batch(ps, storage="bf16", compact=1, epochs_per_segment=2, abar_recompute_every=5) as b:
        for i in range(len(ps)):
            info = asaga.asaga_batch_get_info(b.b, i)
            assert (info["col_index_bytes"], info["row_values"]) == (2, 0)
        asaga.asaga_batch_autotune(b.b, b.count)
        s, res = asaga.asaga_batch_run(b.b, b.count, 600, 1e-6, fs)
        assert s == asaga.OK
        f_gpu = asaga.asaga_batch_objective(b.b, b.count)
        for i, p in enumerate(ps):
            x = asaga.asaga_batch_get_state(b.b, i, p.d, p.n)[0]
            assert f_gpu[i] == pytest.approx(R.objective(p, x.astype(np.float64)), rel=1e-12)
