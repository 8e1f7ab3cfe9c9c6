"""The C ABI on the host: the library loads, exports what include/asaga.h
declares, and rejects invalid problems before touching the GPU (CPU only)."""
import ctypes

import numpy as np
import pytest

from paper_1606_04809_gb300 import asaga, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return asaga.load()


def test_exports_every_declared_function(lib):
    names = asaga.header_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = asaga.asaga_default_options()
    assert o.loss == 0 and o.lambda_ == 0.0 and o.gamma == 0.0 and o.storage_dtype == asaga.DTYPE["f32"]
    assert o.epochs_per_segment == 1 and o.deterministic == 0 and o.cuda_stream is None


def test_status_strings(lib):
    for s, name in enumerate(asaga.STATUS_NAMES):
        assert asaga.asaga_status_string(s) == name
    assert asaga.asaga_status_string(99) == "ASAGA_UNKNOWN"


def small_csr():
    row_ptr = np.array([0, 2, 3, 5], dtype=np.int64)
    col_idx = np.array([0, 2, 1, 0, 3], dtype=np.int32)
    values = np.array([1.0, -0.5, 2.0, 0.25, 1.0])
    labels = np.array([1.0, -1.0, 1.0])
    return row_ptr, col_idx, values, labels


def create(row_ptr, col_idx, values, labels, n=3, d=4, dtype="f64", dense=False, nnz=None, **opt):
    prob = asaga.Problem(n, d, row_ptr, col_idx, values, dtype, labels, dense=dense, nnz=nnz)
    o = asaga.asaga_default_options(**opt)
    ctx = ctypes.c_void_p()
    s = asaga.load().asaga_create(ctypes.byref(ctx), ctypes.byref(prob.struct), ctypes.byref(o))
    if ctx.value:
        asaga.asaga_destroy(ctx.value)
    return s, asaga.asaga_last_error(None)


@pytest.mark.parametrize("mutate,msg", [
    (lambda a: a[0].__setitem__(2, 1), "decreases"),
    (lambda a: a[0].__setitem__(1, 9), "passes nnz at row 0"),  # row 0 would run past col_idx
    (lambda a: a[0].__setitem__(3, 4), "end at nnz"),
    (lambda a: a[1].__setitem__(1, 4), "out of range"),
    (lambda a: a[1].__setitem__(1, -1), "out of range"),
    (lambda a: a[1].__setitem__(1, 0), "repeated column"),
    (lambda a: a[2].__setitem__(2, np.nan), "non-finite value"),
    (lambda a: a[2].__setitem__(2, np.inf), "non-finite value"),
    (lambda a: a[3].__setitem__(1, 0.0), "not +-1"),
    (lambda a: a[3].__setitem__(1, np.nan), "non-finite label"),
])
def test_invalid_csr_is_rejected(lib, mutate, msg):
    arrs = list(small_csr())
    mutate(arrs)
    s, err = create(*arrs)
    assert s == asaga.EINVAL and msg in err


@pytest.mark.parametrize("opt,msg", [
    (dict(lam=-1.0), "lambda"),
    (dict(lam=float("nan")), "lambda"),
    (dict(gamma=float("inf")), "gamma"),
    (dict(storage_dtype="f64"), "storage_dtype"),
    (dict(loss=7), "loss"),
    (dict(max_warps=-2), "negative"),
    (dict(sampling=5), "sampling"),
])
def test_invalid_options_are_rejected(lib, opt, msg):
    s, err = create(*small_csr(), **opt)
    assert s == asaga.EINVAL and msg in err


def test_invalid_shapes_are_rejected(lib):
    rp, ci, v, y = small_csr()
    assert create(rp, ci, v, y, n=0)[0] == asaga.EINVAL
    assert create(rp, ci, v, y, d=0)[0] == asaga.EINVAL
    assert create(None, ci, v, y)[0] == asaga.EINVAL
    assert create(rp, ci, v, None)[0] == asaga.EINVAL
    dense_vals = np.ones(12)
    assert create(None, None, dense_vals, y, dense=True, nnz=5)[0] == asaga.EINVAL


def test_bf16_and_f16_nonfinite_bit_patterns(lib):
    rp, ci, _, y = small_csr()
    bad16 = np.array([0x3C00, 0x7C00, 0x3C00, 0x3C00, 0x3C00], dtype=np.uint16)  # f16 +inf
    assert create(rp, ci, bad16, y, dtype="f16")[0] == asaga.EINVAL
    badbf = np.array([0x3F80, 0x3F80, 0x7FC0, 0x3F80, 0x3F80], dtype=np.uint16)  # bf16 NaN
    assert create(rp, ci, badbf, y, dtype="bf16")[0] == asaga.EINVAL


def test_null_context_calls(lib):
    L = asaga.load()
    assert L.asaga_run(None, 1.0, 0.0, 1.0, None) == asaga.EINVAL
    assert L.asaga_objective(None, None) == asaga.EINVAL
    L.asaga_destroy(None)  # no-op


def test_valid_problem_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s, err = create(*small_csr())
    assert s == asaga.ECUDA and err


def test_validation_of_a_large_problem_reports_the_first_bad_row(lib):
    """Validation runs on several host threads; the reported error is still the first one."""
    g = np.random.default_rng(0)
    n, d, k = 300_000, 5000, 4
    col = np.sort(g.integers(0, d // k, (n, k)) + np.arange(k) * (d // k), axis=1).astype(np.int32)
    row_ptr = np.arange(n + 1, dtype=np.int64) * k
    vals = np.ones(n * k)
    y = np.ones(n)
    assert create(row_ptr, col.ravel(), vals, y, n=n, d=d)[0] != asaga.EINVAL
    bad = col.copy()
    bad[250_000, 1] = bad[250_000, 0]
    bad[280_000, 2] = bad[280_000, 0]
    s, err = create(row_ptr, bad.ravel(), vals, y, n=n, d=d)
    assert s == asaga.EINVAL and "row 250000" in err
    bad2 = col.copy()
    bad2[299_999, 3] = d
    s, err = create(row_ptr, bad2.ravel(), vals, y, n=n, d=d)
    assert s == asaga.EINVAL and str(299_999 * k + 3) in err


def test_sampler_arguments_are_checked_before_any_cuda_call(lib):
    L = asaga.load()
    rows = np.empty(4, dtype=np.int64)
    p = rows.ctypes.data
    assert L.asaga_sample_rows(1, 0, 0, 0, 4, p) == asaga.EINVAL
    assert "n must be" in asaga.asaga_last_error(None)
    assert L.asaga_sample_rows(1, 10, 2, 0, 4, p) == asaga.EINVAL
    assert "sampling" in asaga.asaga_last_error(None)
    assert L.asaga_sample_rows(1, 10, 0, 0, -1, p) == asaga.EINVAL
    assert L.asaga_sample_rows(1, 10, 0, 0, 4, None) == asaga.EINVAL
    assert L.asaga_sample_rows(1, (1 << 62) + 1, 1, 0, 4, p) == asaga.EINVAL
    assert L.asaga_sample_rows(1, 10, 0, 0, 0, None) == asaga.OK  # nothing to do


def test_cancel_needs_a_context(lib):
    L = asaga.load()
    assert L.asaga_cancel(None) == asaga.EINVAL
    assert L.asaga_batch_cancel(None) == asaga.EINVAL
    assert asaga.asaga_status_string(asaga.ECANCELLED) == "ASAGA_ECANCELLED"


def test_set_schedule_needs_a_context(lib):
    assert asaga.load().asaga_set_schedule(None, 4, 0.1, 0) == asaga.EINVAL


def test_row_path_and_draw_placement_need_a_context(lib):
    L = asaga.load()
    assert L.asaga_set_row_path(None, 0, 2) == asaga.EINVAL
    assert L.asaga_set_draw_ahead(None, 1) == asaga.EINVAL


def test_line_probe_arguments_are_checked_before_any_cuda_call(lib):
    import ctypes

    L = asaga.load()
    ns = ctypes.c_double()
    assert L.asaga_probe_line_rate(0, 10, ctypes.byref(ns)) == asaga.EINVAL
    assert "warps must be" in asaga.asaga_last_error(None)
    assert L.asaga_probe_line_rate(70000, 10, ctypes.byref(ns)) == asaga.EINVAL
    assert L.asaga_probe_line_rate(4, 0, ctypes.byref(ns)) == asaga.EINVAL
    assert L.asaga_probe_line_rate(4, 10, None) == asaga.EINVAL


# a stamp array per thread (d <= 2^18); a per-row hash set beyond, with short rows and with long
# ones that outgrow its first 64 slots
@pytest.mark.parametrize("n,d,k", [(50_000, 3000, 6), (50_000, 400_000, 6), (2_000, 400_000, 300)])
def test_rows_in_any_column_order_are_checked_alike(lib, n, d, k):
    """Increasing rows take a fast path; other rows the general check, with the same verdicts."""
    g = np.random.default_rng(1)
    col = np.stack([g.choice(d, k, replace=False) for _ in range(n)]).astype(np.int32)  # unsorted, distinct
    row_ptr = np.arange(n + 1, dtype=np.int64) * k
    vals = np.ones(n * k)
    y = np.ones(n)
    assert create(row_ptr, col.ravel(), vals, y, n=n, d=d)[0] != asaga.EINVAL
    srt = np.sort(col, axis=1)
    assert create(row_ptr, srt.ravel(), vals, y, n=n, d=d)[0] != asaga.EINVAL
    r1, r2 = 3 * n // 5, 4 * n // 5
    for c in (col, srt):
        bad = c.copy()
        bad[r1, k - 2] = bad[r1, 1]  # a repeat (unsorted, or sorted then broken), far apart in long rows
        s, err = create(row_ptr, bad.ravel(), vals, y, n=n, d=d)
        assert s == asaga.EINVAL and f"repeated column in row {r1}" in err, err
        bad = c.copy()
        bad[r2, 2] = d  # out of range in the middle of a row
        s, err = create(row_ptr, bad.ravel(), vals, y, n=n, d=d)
        assert s == asaga.EINVAL and str(r2 * k + 2) in err, err


@pytest.mark.parametrize("gamma", [0.0, -1.0])
def test_a_step_of_zero_or_below_selects_the_default(lib, gamma):
    """options.gamma <= 0 means 1/(3L) (include/asaga.h), so it is not an input
    error: without a GPU the call gets past the checks to the CUDA error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s, err = create(*small_csr(), gamma=gamma)
    assert s == asaga.ECUDA, err
