"""The C generator of the full-size batch workload (synth_gen.c), on CPU.

It only makes inputs, but both sides of every parity check consume them, and
the stored f* values are keyed by its output: it must give the same bits for
any thread count (and, by construction, on any host), and the instances must
have the shapes the workload specifies.
"""
import math

import numpy as np
import pytest

from paper_1606_04809_gb300 import synth


def small_specs():
    return synth.batch_params(count=6, seed=9, n_range=(500, 3000), d_range=(200, 2000),
                              density_range=(0.005, 0.05), lam_range=(1e-4, 1e-2), storage="bf16")


def test_same_bits_for_any_thread_count():
    spec = small_specs()[3]
    a = synth.batch_instance(spec, values="f64", threads=1)
    b = synth.batch_instance(spec, values="f64", threads=7)
    c = synth.batch_instance(spec, values="bits", threads=3)
    for x in (b, c):
        assert np.array_equal(a.row_ptr, x.row_ptr) and np.array_equal(a.col_idx, x.col_idx)
        assert np.array_equal(a.labels, x.labels)
        assert a.fingerprint() == x.fingerprint()
    assert np.array_equal(a.values, c.values_f64())


def test_instance_shapes():
    for spec in small_specs():
        p = synth.batch_instance(spec, values="f64")
        assert (p.n, p.d, p.lam) == (spec["n"], spec["d"], spec["lam"])
        lens = np.diff(p.row_ptr)
        assert lens.min() >= spec["k_min"] and lens.max() <= spec["k_max"]
        assert abs(lens.mean() - spec["k_mean"]) <= 0.1 * spec["k_mean"] + 1
        for i in range(0, p.n, max(1, p.n // 50)):
            cols = p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]]
            assert np.all(np.diff(cols) > 0) and cols.min() >= 0 and cols.max() < p.d  # sorted, distinct
            v = p.values[p.row_ptr[i]:p.row_ptr[i + 1]]
            assert np.all(v > 0) and abs(np.sum(v * v) - 1.0) <= 2e-2  # unit rows up to bf16 rounding
        assert np.array_equal(p.values, synth.to_storage_grid(p.values, "bf16"))
        assert set(np.unique(p.labels)) <= {-1.0, 1.0}
        # Zipf(1.1) columns: the most frequent column is in far more rows than the median one
        cnt = np.bincount(p.col_idx, minlength=p.d)
        assert cnt.max() >= 10 * max(1, np.median(cnt))


def test_specified_batch_ranges():
    sp = synth.batch_params(**synth.FULL_BATCH)
    assert len(sp) == 256
    assert all(10_000 <= s["n"] <= 200_000 and 1_000 <= s["d"] <= 50_000 for s in sp)
    assert all(0.005 * s["d"] - 1e-9 <= s["k_mean"] <= 0.02 * s["d"] + 1e-9 or s["k_mean"] == 1.0 for s in sp)
    lams = np.array([s["lam"] for s in sp])
    assert lams[0] == pytest.approx(1e-6) and lams[-1] == pytest.approx(1e-2) and np.all(np.diff(lams) > 0)


def test_own_log_and_exp_agree_with_the_c_library():
    L = synth._generator()
    xs = np.concatenate([np.logspace(-300, 300, 601), np.random.default_rng(0).uniform(1e-3, 10, 2000)])
    for x in xs:
        if x != 1.0:
            assert abs(L.synth_gen_log(x) - math.log(x)) <= 4e-16 * abs(math.log(x)) + 1e-300
    for y in np.random.default_rng(1).uniform(-30, 30, 2000):
        assert abs(L.synth_gen_exp(y) - math.exp(y)) <= 4e-15 * math.exp(y)
