"""The batched solver (many independent problems in one launch) against the
float64 CPU checker, through the C ABI."""
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


def small_batch(storage, count=6, seed=61):
    return synth.logistic_batch(count=count, seed=seed, n_range=(1500, 4000), d_range=(200, 1500),
                                density_range=(0.005, 0.03), lam_range=(1e-3, 1e-2), storage=storage)


def fstars(ps):
    out = []
    for p in ps:
        res = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-11,
                                max_epochs=2000, check_every=5)
        out.append(res)
    return out


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batch_reaches_each_instance_optimum(storage):
    ps = small_batch(storage)
    cert = fstars(ps)
    fs = np.array([c["fstar"] for c in cert])
    with asaga.Batch(ps, storage=storage, epochs_per_segment=2, abar_recompute_every=5) as b:
        tune = asaga.asaga_batch_autotune(b.b, b.count)
        assert all(t["warps"] >= 4 and t["gamma"] > 0 for t in tune)
        s, res = asaga.asaga_batch_run(b.b, b.count, 600, 1e-6, fs)
        assert s == asaga.OK, (asaga.STATUS_NAMES[s], [r.as_dict() for r in res])
        f_gpu = asaga.asaga_batch_objective(b.b, b.count)
        for i, p in enumerate(ps):
            x = asaga.asaga_batch_get_state(b.b, i, p.d, p.n)[0]
            f_ref = R.objective(p, x.astype(np.float64))
            assert f_gpu[i] == pytest.approx(f_ref, rel=1e-12)
            assert (f_ref - fs[i]) / abs(fs[i]) <= 1e-6 + cert[i]["bound"] / abs(fs[i])
            assert res[i].rel_subopt <= 1e-6


def test_batch_stops_finished_instances_and_reports_times():
    ps = small_batch("f32", count=4, seed=62)
    fs = np.array([c["fstar"] for c in fstars(ps)])
    with asaga.Batch(ps, storage="f32", epochs_per_segment=1) as b:
        asaga.asaga_batch_autotune(b.b, b.count)
        s, res = asaga.asaga_batch_run(b.b, b.count, 600, 1e-6, fs)
        assert s == asaga.OK
        # an instance that finished stops receiving updates: its update count matches its epochs
        for i, p in enumerate(ps):
            assert res[i].updates == round(res[i].epochs * p.n)
            assert 0 < res[i].solver_seconds <= max(r.solver_seconds for r in res)


def test_batch_schedule_and_errors():
    ps = small_batch("f32", count=3, seed=63)
    with asaga.Batch(ps, storage="f32") as b:
        asaga.asaga_batch_set_schedule(b.b, warps=[5, 8, 12], gamma=[0.5, 0.5, 0.5])
        assert [asaga.asaga_batch_get_info(b.b, i)["warps"] for i in range(3)] == [8, 8, 12]
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_batch_set_schedule(b.b, warps=[0, 4, 4])
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_batch_get_state(b.b, 3, 10, 10)
        s, res = asaga.asaga_batch_run(b.b, b.count, 3)
        assert s == asaga.OK and all(np.isfinite(r.f_last) for r in res)
    mixed = [ps[0], synth.dense_ridge(500, 10, storage="f32", seed=64)]
    with pytest.raises(asaga.AsagaError):
        asaga.Batch(mixed, storage="f32")


def test_batch_cancel_from_another_thread():
    import threading
    ps = small_batch("f32", count=3, seed=63)
    with asaga.Batch(ps, storage="f32", epochs_per_segment=1) as b:
        out = {}
        th = threading.Thread(target=lambda: out.setdefault("res", asaga.asaga_batch_run(b.b, b.count, 1e6)))
        th.start()
        import time
        time.sleep(0.3)
        asaga.asaga_batch_cancel(b.b)
        th.join(timeout=60)
        assert not th.is_alive()
        s, res = out["res"]
        assert s == asaga.ECANCELLED and all(0 < r.epochs < 1e6 for r in res)
        s2, res2 = asaga.asaga_batch_run(b.b, b.count, 2)
        assert s2 == asaga.OK and all(np.isfinite(r.f_last) for r in res2)


def test_batched_abar_recomputation_matches_the_checker():
    """Every 2nd segment recomputes abar = (1/n) sum_i alpha_i a_i of every
    instance in one batched float64 pass inside the segment's graph; each
    instance's abar then equals the checker's float64 sum rounded to float32
    (one ulp: the float64 column sums add atomics in no fixed order)."""
    ps = small_batch("f32", count=5, seed=65)
    with asaga.Batch(ps, storage="f32", epochs_per_segment=1, abar_recompute_every=2) as b:
        s, res = asaga.asaga_batch_run(b.b, b.count, 2)
        assert s == asaga.OK
        for i, p in enumerate(ps):
            _, abar, alpha = asaga.asaga_batch_get_state(b.b, i, p.d, p.n)
            exact = R.abar_from_scratch(p, alpha.astype(np.float64))
            np.testing.assert_array_max_ulp(abar, exact.astype(np.float32), maxulp=1)
            assert 0 < res[i].abar_drift < 1e-4
        # the cadence counts over the batch's life: the next call's first segment does not recompute
        s, res = asaga.asaga_batch_run(b.b, b.count, 1)
        assert s == asaga.OK and all(r.abar_drift == 0 for r in res)
        asaga.asaga_batch_reset(b.b)
        x, abar, alpha = asaga.asaga_batch_get_state(b.b, 0, ps[0].d, ps[0].n)
        assert not x.any() and not abar.any() and not alpha.any()
