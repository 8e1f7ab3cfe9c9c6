"""Parity of the CUDA solver (through its C ABI) with the float64 CPU checker.

Tolerances:
  * deterministic replay (one warp, updates in order, float32 state) vs the
    float64 serial Sparse SAGA on the same index sequence: relative l2 error
    <= 1e-4 on x, alpha and abar after one epoch, and per element
    max_v |x_v - x*_v| <= 1e-3 max_v |x*_v| (likewise for alpha and abar).
    The l2 bound limits the average error; each coordinate's float32 error is
    rounding of its sum of updates (about 6e-8 of their size) plus the error
    of the deltas, which reaches every coordinate in proportion to a_iv, so no
    coordinate should exceed ~1e-4 of the largest.  Ten times the l2
    tolerance keeps a margin and still fails a coordinate that is wrong by a
    sizeable part of itself unless it is below 1e-3 of the largest;
  * float64 evaluations (objective, gradient, abar recomputation) at the
    GPU's float32 iterate widened exactly: relative error <= 1e-12 (sums of
    at most ~1e3 terms per row in a different order give ~1e-14);
  * asynchronous runs: (f - f*)/|f*| <= 1e-6 against the checker's f*.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

DET_TOL = 1e-4
ELEM_TOL = 1e-3
EVAL_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def elem(a, b):
    """max_v |a_v - b_v| / max_v |b_v|"""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b)) if b.size else 0.0
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0) if b.size else 0.0


def quantized(p, storage):
    q = synth.Problem(**{**p.__dict__})
    q.values = synth.to_storage_grid(p.values, storage)
    q.storage = storage
    return q


def replay_pair(p, idx, storage, **opt):
    """Runs the index sequence on the GPU (one warp, in order) and in the checker."""
    with asaga.Context(p, storage=storage, **opt) as c:
        asaga.asaga_run_indices(c.ctx, idx)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        info = asaga.asaga_get_info(c.ctx)
    st = R.State.zeros(p)
    R.sparse_saga(p, st, idx, info["gamma"])
    return (x, abar, alpha), st, info


def assert_replay(p, idx, storage, tol=DET_TOL, **opt):
    (x, abar, alpha), st, _ = replay_pair(p, idx, storage, **opt)
    for name, a, b in (("x", x, st.x), ("alpha", alpha, st.alpha), ("abar", abar, st.abar)):
        assert rel(a, b) <= tol, (name, rel(a, b))
        assert elem(a, b) <= 10 * tol, (name, elem(a, b))
    return x, st


# ------------------------------------------------------------------ deterministic replay

def test_replay_one_epoch_small_logistic_float64_problem():
    """n=2000, d=500 logistic, float64 values stored as float32 on the GPU."""
    p = synth.small_logistic()
    idx = synth.sample_indices(p.n, p.n, seed=4)
    assert_replay(p, idx, "f32")


def test_replay_one_epoch_small_logistic_same_quantised_values():
    p = quantized(synth.small_logistic(), "f32")
    idx = synth.sample_indices(p.n, p.n, seed=5)
    assert_replay(p, idx, "f32")


def test_replay_long_rows_cross_the_register_tile():
    """Rows of 1..700 entries: the in-register part (up to 128) and the re-read tail."""
    p = synth.sparse_logistic(1500, 3000, k_mean=150, k_min=1, k_max=700, k_sigma=1.0, zipf_s=1.1,
                              values="abs_normal", storage="f32", seed=6)
    assert p.row_lengths().max() > 256
    idx = synth.sample_indices(p.n, p.n, seed=7)
    assert_replay(p, idx, "f32")


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_replay_half_precision_storage(storage):
    p = synth.sparse_logistic(4000, 20000, k_mean=40, k_min=4, k_max=200, k_sigma=0.5, zipf_s=1.1,
                              values="binary" if storage == "bf16" else "abs_normal", storage=storage, seed=8)
    idx = synth.sample_indices(p.n, p.n, seed=9)
    assert_replay(p, idx, storage)


def test_replay_dense_ridge_fp16():
    p = synth.dense_ridge(3000, 54, storage="f16", lam=1e-3, seed=10)
    idx = synth.sample_indices(p.n, p.n, seed=11)
    assert_replay(p, idx, "f16")


def test_replay_dense_small_d_with_packed_and_padded_state():
    p = synth.dense_ridge(800, 7, storage="f32", lam=1e-2, seed=12)
    idx = synth.sample_indices(p.n, 2 * p.n, seed=13)
    for stride in (1, 16):
        assert_replay(p, idx, "f32", column_stride=stride)


def test_replay_empty_rows_and_untouched_columns():
    g = np.random.default_rng(14)
    n, d = 300, 80
    lengths = g.integers(0, 6, n)
    lengths[:5] = 0
    row_ptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    cols = [np.sort(g.choice(60, size=k, replace=False)) for k in lengths]  # columns 60..79 untouched
    col_idx = np.concatenate(cols).astype(np.int32)
    values = synth.to_storage_grid(g.standard_normal(col_idx.size), "f32")
    labels = np.where(g.standard_normal(n) >= 0, 1.0, -1.0)
    p = synth.Problem("edge", n, d, row_ptr, col_idx, values, labels, "logistic", lam=1.0 / n, storage="f32")
    idx = np.concatenate([np.arange(5), synth.sample_indices(n, 3 * n, seed=15)])
    x, st = assert_replay(p, idx, "f32")
    assert np.all(x[60:] == 0.0)


def test_replay_single_row_single_column():
    p = synth.Problem("one", 1, 1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                      np.array([0.75]), np.array([-1.0]), "logistic", lam=0.5, storage="f32")
    assert_replay(p, np.zeros(50, dtype=np.int64), "f32")


def test_replay_is_bitwise_reproducible():
    p = synth.small_logistic()
    idx = synth.sample_indices(p.n, p.n, seed=16)
    a = replay_pair(p, idx, "f32")[0]
    b = replay_pair(p, idx, "f32")[0]
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_device_index_out_of_range_stops_at_the_bad_entry():
    import torch
    p = synth.small_logistic()
    idx = synth.sample_indices(p.n, 500, seed=17)
    bad = idx.copy()
    bad[300] = p.n  # out of range
    with asaga.Context(p, storage="f32") as c:
        didx = torch.from_numpy(bad).cuda()
        with pytest.raises(asaga.AsagaError) as e:
            asaga.asaga_run_indices(c.ctx, didx, on_device=True)
        assert e.value.status == asaga.EINVAL
        x = asaga.asaga_get_state(c.ctx)[0]
        gamma = asaga.asaga_get_info(c.ctx)["gamma"]
    st = R.sparse_saga(p, R.State.zeros(p), idx[:300], gamma)
    assert rel(x, st.x) <= DET_TOL


def test_host_index_out_of_range_is_rejected_before_any_update():
    p = synth.small_logistic()
    with asaga.Context(p, storage="f32") as c:
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_run_indices(c.ctx, np.array([0, 1, p.n + 3]))
        assert np.all(asaga.asaga_get_state(c.ctx)[0] == 0.0)


# ------------------------------------------------------------------ set-up and float64 evaluations

@pytest.mark.parametrize("maker", ["small", "dense", "bf16"])
def test_setup_constants_match(maker):
    p = {"small": lambda: quantized(synth.small_logistic(), "f32"),
         "dense": lambda: synth.dense_ridge(2000, 54, storage="f16", seed=18),
         "bf16": lambda: synth.sparse_logistic(3000, 9000, k_mean=30, k_min=2, k_max=90, k_sigma=0.4,
                                               zipf_s=1.1, values="binary", storage="bf16", seed=19)}[maker]()
    with asaga.Context(p) as c:
        info = asaga.asaga_get_info(c.ctx)
    # L carries lambda * D_v with D_v stored in float32 on the device (relative rounding <= 6e-8)
    assert info["L"] == pytest.approx(R.lipschitz(p), rel=1e-7)
    assert info["gamma"] == pytest.approx(1.0 / (3.0 * info["L"]), rel=1e-15)
    assert info["delta"] == pytest.approx(R.sparsity_delta(p), rel=1e-15)
    assert info["max_row_len"] == p.row_lengths().max()


@pytest.mark.parametrize("maker", ["small", "dense", "long", "hot"])
def test_float64_evaluations_match(maker):
    p = {"small": lambda: quantized(synth.small_logistic(), "f32"),
         "dense": lambda: synth.dense_ridge(5000, 54, storage="f16", seed=20),
         "long": lambda: synth.sparse_logistic(2000, 4000, k_mean=120, k_min=1, k_max=900, k_sigma=1.0,
                                               zipf_s=1.1, storage="f32", seed=21),
         "hot": lambda: synth.sparse_logistic(20000, 3000, k_mean=40, k_min=1, k_max=300, k_sigma=0.6,
                                              zipf_s=1.1, storage="f32", seed=28)}[maker]()
    with asaga.Context(p, seed=3) as c:
        asaga.asaga_run(c.ctx, 3)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        f = asaga.asaga_objective(c.ctx)
        g, n2 = asaga.asaga_full_grad(c.ctx)
        drift = asaga.asaga_recompute_abar(c.ctx)
        abar_new = asaga.asaga_get_state(c.ctx)[1]
    x64 = x.astype(np.float64)
    assert f == pytest.approx(R.objective(p, x64), rel=EVAL_TOL)
    g_ref = R.gradient(p, x64)
    assert rel(g, g_ref) <= 1e-11
    assert n2 == pytest.approx(float(np.dot(g_ref, g_ref)), rel=1e-11)
    exact = R.abar_from_scratch(p, alpha.astype(np.float64))
    assert drift == pytest.approx(float(np.max(np.abs(abar.astype(np.float64) - exact))), rel=1e-6, abs=1e-12)
    np.testing.assert_array_equal(abar_new, exact.astype(np.float32))


def test_objective_at_zero_is_log2():
    p = synth.small_logistic()
    with asaga.Context(p) as c:
        assert asaga.asaga_objective(c.ctx) == pytest.approx(np.log(2.0), rel=1e-15)


# ------------------------------------------------------------------ asynchronous runs

def test_async_small_logistic_reaches_1e6():
    p = quantized(synth.small_logistic(), "f32")
    fstar = R.objective(p, R.newton(p))
    with asaga.Context(p, seed=1, abar_recompute_every=5) as c:
        s, r = asaga.asaga_run(c.ctx, 300, 1e-6, fstar)
        info = asaga.asaga_get_info(c.ctx)
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict(), info)
    assert r.rel_subopt <= 1e-6 and r.rel_subopt > -1e-9


def test_async_rcv1_shaped_medium_reaches_1e6():
    p = synth.rcv1_like(seed=22, n=60000, d=6000)
    cert = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-10)
    with asaga.Context(p, seed=2, abar_recompute_every=5) as c:
        tune = asaga.asaga_autotune(c.ctx)
        s, r = asaga.asaga_run(c.ctx, 200, 1e-6, cert["fstar"])
        info = asaga.asaga_get_info(c.ctx)
        x = asaga.asaga_get_state(c.ctx)[0]
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict(), info, tune)
    assert info["warps"] == tune["warps"] and info["gamma"] == tune["gamma"]
    assert R.objective(p, x.astype(np.float64)) - cert["fstar"] <= 1e-6 * abs(cert["fstar"]) + cert["bound"]


def test_autotune_leaves_a_zero_state_and_rejects_deterministic_mode():
    p = synth.small_logistic()
    with asaga.Context(p, seed=3) as c:
        tune = asaga.asaga_autotune(c.ctx, 4)
        assert tune["trials"] >= 1 and tune["warps"] >= 1 and tune["gamma"] > 0
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        assert not x.any() and not abar.any() and not alpha.any()
    with asaga.Context(p, deterministic=1) as c:
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_autotune(c.ctx)


def test_a_tuned_schedule_transfers_to_a_new_context():
    p = synth.rcv1_like(seed=22, n=60000, d=6000)
    cert = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-10)
    with asaga.Context(p, seed=2) as c:
        asaga.asaga_autotune(c.ctx)
        tuned = asaga.asaga_get_info(c.ctx)
    with asaga.Context(p, seed=3, abar_recompute_every=5) as c:
        asaga.asaga_set_schedule(c.ctx, tuned["warps"], tuned["gamma"], tuned["warps_per_block"])
        info = asaga.asaga_get_info(c.ctx)
        assert (info["warps"], info["gamma"], info["warps_per_block"]) == \
            (tuned["warps"], tuned["gamma"], tuned["warps_per_block"])
        s, r = asaga.asaga_run(c.ctx, 200, 1e-6, cert["fstar"])
        assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict(), tuned)
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_set_schedule(c.ctx, 0, 0.1)
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_set_schedule(c.ctx, 64, -1.0)


def test_async_dense_ridge_reaches_closed_form():
    p = synth.dense_ridge(20000, 54, storage="f16", lam=1e-3, seed=23)
    xs = R.ridge_closed_form(p)
    fstar = R.objective(p, xs)
    with asaga.Context(p, seed=4, abar_recompute_every=5) as c:
        asaga.asaga_autotune(c.ctx)
        s, r = asaga.asaga_run(c.ctx, 300, 1e-6, fstar)
        x = asaga.asaga_get_state(c.ctx)[0]
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict())
    # strong convexity: |x - x*|^2 <= 2 (f - f*) / lambda
    assert np.sum((x - xs) ** 2) <= 2 * (1e-6 * abs(fstar)) / p.lam * 1.01


def test_async_untouched_columns_stay_zero():
    p = synth.sparse_logistic(5000, 2900, k_mean=8, k_min=1, k_max=20, zipf_s=None, storage="f32", seed=24)
    p.d = 3000  # columns 2900..2999 exist but no row touches them
    cnt = np.bincount(p.col_idx, minlength=p.d)
    assert (cnt[2900:] == 0).all()
    with asaga.Context(p, seed=5) as c:
        asaga.asaga_run(c.ctx, 5)
        x, abar, _ = asaga.asaga_get_state(c.ctx)
    assert np.all(x[cnt == 0] == 0.0) and np.all(abar[cnt == 0] == 0.0)
    assert np.any(x != 0.0)


def test_run_status_paths():
    p = synth.small_logistic()
    with asaga.Context(p, seed=6) as c:
        s, r = asaga.asaga_run(c.ctx, 0)  # zero epochs: evaluates f(0)
        assert s == asaga.OK and r.f_last == pytest.approx(np.log(2.0), rel=1e-15)
        s, r = asaga.asaga_run(c.ctx, 2, 1e-30, 0.4)  # unreachable target
        assert s == asaga.ENOTCONVERGED and r.epochs == 2 and r.segments == 2
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_run(c.ctx, 1, 1e-6, 0.0)  # target needs a nonzero f*


def test_timeout_returns_status_and_keeps_context_usable():
    p = synth.rcv1_like(seed=25, n=200000, d=20000)
    with asaga.Context(p, seed=7, timeout_s=0.002, epochs_per_segment=50) as c:
        s, r = asaga.asaga_run(c.ctx, 50)
        assert s == asaga.ETIMEOUT
        f = asaga.asaga_objective(c.ctx)
        assert np.isfinite(f)


def test_cancel_from_another_thread_stops_a_run_and_keeps_the_context_usable():
    import threading
    import time
    p = synth.rcv1_like(seed=22, n=60000, d=6000)
    with asaga.Context(p, seed=5, max_warps=256, gamma=0.05) as c:
        out = {}

        def run():
            t0 = time.perf_counter()
            out["res"] = asaga.asaga_run(c.ctx, 1e6)
            out["t"] = time.perf_counter() - t0

        th = threading.Thread(target=run)
        th.start()
        time.sleep(0.3)
        asaga.asaga_cancel(c.ctx)
        th.join(timeout=60)
        assert not th.is_alive()
        s, r = out["res"]
        assert s == asaga.ECANCELLED and 0 < r.epochs < 1e6 and out["t"] < 10
        # a new run starts clean and the state is finite
        s2, r2 = asaga.asaga_run(c.ctx, 2)
        assert s2 == asaga.OK and np.isfinite(r2.f_last)
        assert np.all(np.isfinite(asaga.asaga_get_state(c.ctx)[0]))


def test_state_roundtrip_and_resume():
    p = synth.small_logistic()
    with asaga.Context(p, seed=8) as c:
        asaga.asaga_run(c.ctx, 2)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        f1 = asaga.asaga_objective(c.ctx)
        with asaga.Context(p, seed=8) as d:
            asaga.asaga_set_state(d.ctx, x, abar, alpha, updates_done=2 * p.n)
            x2, abar2, alpha2 = asaga.asaga_get_state(d.ctx)
            assert np.array_equal(x, x2) and np.array_equal(abar, abar2) and np.array_equal(alpha, alpha2)
            assert asaga.asaga_objective(d.ctx) == f1


def test_torch_stream_is_used():
    import torch
    p = synth.small_logistic()
    s = torch.cuda.Stream()
    with asaga.Context(p, seed=9, cuda_stream=s.cuda_stream) as c:
        st, r = asaga.asaga_run(c.ctx, 2)
        assert st == asaga.OK and np.isfinite(r.f_last)


def test_overlap_is_zero_for_one_warp_and_grows_with_warps():
    """tau (App. E.2 estimator): a single warp never overlaps itself; W warps
    keep about W - 1 other updates in flight."""
    p = synth.rcv1_like(seed=30, n=40000, d=4000)
    with asaga.Context(p, seed=1, max_warps=1) as c:
        o = asaga.asaga_measure_overlap(c.ctx, 0.05)
        assert o["warps"] == 1 and o["updates"] == 2000
        assert o["tau_mean"] <= 0.05
    with asaga.Context(p, seed=1, max_warps=256) as c:
        o = asaga.asaga_measure_overlap(c.ctx, 1.0)
        assert o["warps"] == 256
        assert 0.3 * 255 <= o["tau_mean"] <= 3 * 256, o
        assert o["tau_paper"] >= o["tau_mean"] and o["tau_max"] >= o["tau_paper"]
        assert o["window_ns_mean"] > 0


def test_plain_writes_break_the_average_invariant():
    """App. G.2: without atomic adds, concurrent updates are lost, so abar no
    longer equals (1/n) sum_i alpha_i a_i (the bookkeeping behind the floor the
    paper observes); with atomic adds the gap is float32 rounding."""
    p = synth.rcv1_like(seed=31, n=60000, d=6000)
    drift = {}
    for plain in (0, 1):
        with asaga.Context(p, seed=4, max_warps=1024, gamma=0.05, plain_writes=plain) as c:
            asaga.asaga_run(c.ctx, 3)
            drift[plain] = asaga.asaga_recompute_abar(c.ctx)
    assert drift[0] < 1e-5
    assert drift[1] > 30 * drift[0]


def test_abar_recompute_cadence_counts_across_calls():
    """abar_recompute_every counts segments over the context's life, so a loop of
    one-epoch asaga_run calls recomputes abar every k-th call (and reports its
    drift then), not never; asaga_set_state restarts the count."""
    p = synth.rcv1_like(seed=23, n=20000, d=3000)
    with asaga.Context(p, storage="f32", seed=3, max_warps=128, gamma=0.1, abar_recompute_every=2) as c:
        drifts = [asaga.asaga_run(c.ctx, 1)[1].abar_drift for _ in range(5)]
        assert drifts[0] == 0.0 and drifts[2] == 0.0 and drifts[4] == 0.0, drifts
        assert drifts[1] > 0.0 and drifts[3] > 0.0, drifts  # float32 running sums drift after an epoch
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        asaga.asaga_set_state(c.ctx, x, abar, alpha, 5 * p.n)
        after = [asaga.asaga_run(c.ctx, 1)[1].abar_drift for _ in range(2)]
        assert after[0] == 0.0 and after[1] > 0.0, after
