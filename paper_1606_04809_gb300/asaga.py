"""Python binding of the C ABI in include/asaga.h (ctypes; argument
marshalling only -- every step of the solver runs in the CUDA library).

The functions carry the C names.  Host arrays are numpy arrays; device
arrays may be passed as torch CUDA tensors (their data pointers are used).
Calls that fail with ASAGA_EINVAL / ENOMEM / ECUDA raise AsagaError;
asaga_run returns its status, since ENOTCONVERGED, ETIMEOUT and EDIVERGED
are outcomes of a run rather than misuse.  Loading fails loudly when the
library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libasaga.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "asaga.h")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDIVERGED, ENOTCONVERGED, ECANCELLED = range(8)
STATUS_NAMES = ["ASAGA_OK", "ASAGA_EINVAL", "ASAGA_ENOMEM", "ASAGA_ECUDA", "ASAGA_ETIMEOUT",
                "ASAGA_EDIVERGED", "ASAGA_ENOTCONVERGED", "ASAGA_ECANCELLED"]
LOSS = {"logistic": 0, "squared": 1}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
SAMPLING = {"uniform": 0, "permutation": 1}


class AsagaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")
        self.status = status
        self.message = message


class asaga_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("values_dtype", ctypes.c_int), ("labels", ctypes.c_void_p), ("dense", ctypes.c_int),
                ("on_device", ctypes.c_int)]


class asaga_options(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_int), ("lambda_", ctypes.c_double), ("gamma", ctypes.c_double),
                ("storage_dtype", ctypes.c_int), ("max_warps", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("epochs_per_segment", ctypes.c_int),
                ("abar_recompute_every", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("column_stride", ctypes.c_int),
                ("plain_writes", ctypes.c_int), ("sampling", ctypes.c_int), ("compact", ctypes.c_int)]


class asaga_result(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_double), ("seconds", ctypes.c_double), ("solver_seconds", ctypes.c_double),
                ("eval_seconds", ctypes.c_double), ("f_last", ctypes.c_double), ("rel_subopt", ctypes.c_double),
                ("updates", ctypes.c_int64), ("abar_drift", ctypes.c_double), ("segments", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class asaga_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("nnz", ctypes.c_int64), ("L", ctypes.c_double),
                ("gamma", ctypes.c_double), ("delta", ctypes.c_double), ("warps", ctypes.c_int),
                ("column_stride", ctypes.c_int), ("device_bytes", ctypes.c_int64),
                ("max_row_len", ctypes.c_int64), ("n_hot", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("col_index_bytes", ctypes.c_int), ("row_values", ctypes.c_int),
                ("row_threshold", ctypes.c_int64), ("row_group", ctypes.c_int), ("draw_ahead", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class asaga_tune_result(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int), ("gamma", ctypes.c_double), ("score", ctypes.c_double),
                ("trials", ctypes.c_int), ("seconds", ctypes.c_double), ("row_threshold", ctypes.c_int64),
                ("row_group", ctypes.c_int), ("draw_ahead", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class asaga_overlap(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("warps", ctypes.c_int), ("tau_mean", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("tau_paper", ctypes.c_double), ("window_ns_mean", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib: Optional[ctypes.CDLL] = None


def header_functions() -> list:
    """Names of the functions include/asaga.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asaga_[a-z_]+)\s*\(", text)))


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Loads libasaga.so (built by paper_1606_04809_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libasaga.so not built ({path}); run paper_1606_04809_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, vp, i64, i32, dbl = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.asaga_default_options.argtypes = [P(asaga_options)]
    L.asaga_default_options.restype = None
    L.asaga_create.argtypes = [P(vp), P(asaga_problem), P(asaga_options)]
    L.asaga_run.argtypes = [vp, dbl, dbl, dbl, P(asaga_result)]
    L.asaga_run_indices.argtypes = [vp, vp, i64, i32]
    L.asaga_autotune.argtypes = [vp, dbl, P(asaga_tune_result)]
    L.asaga_measure_overlap.argtypes = [vp, dbl, P(asaga_overlap)]
    L.asaga_measure_overlap_trace.argtypes = [vp, dbl, P(asaga_overlap), vp, i64]
    L.asaga_measure_overlap_trace.restype = i32
    L.asaga_objective.argtypes = [vp, P(dbl)]
    L.asaga_full_grad.argtypes = [vp, vp, P(dbl)]
    L.asaga_recompute_abar.argtypes = [vp, P(dbl)]
    L.asaga_get_state.argtypes = [vp, vp, vp, vp]
    L.asaga_set_state.argtypes = [vp, vp, vp, vp, i64]
    L.asaga_get_info.argtypes = [vp, P(asaga_info)]
    L.asaga_last_error.argtypes = [vp]
    L.asaga_last_error.restype = ctypes.c_char_p
    L.asaga_status_string.argtypes = [i32]
    L.asaga_status_string.restype = ctypes.c_char_p
    L.asaga_recompute_abar_noalloc.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, vp]
    L.asaga_recompute_abar_noalloc.restype = i32
    L.asaga_sample_rows.argtypes = [ctypes.c_uint64, i64, i32, ctypes.c_uint64, i64, vp]
    L.asaga_sample_rows.restype = i32
    L.asaga_probe_line_rate.argtypes = [i32, i64, P(dbl)]
    L.asaga_probe_line_rate.restype = i32
    L.asaga_cancel.argtypes = [vp]
    L.asaga_cancel.restype = i32
    L.asaga_set_schedule.argtypes = [vp, i32, dbl, i32]
    L.asaga_set_schedule.restype = i32
    L.asaga_set_row_path.argtypes = [vp, i64, i32]
    L.asaga_set_row_path.restype = i32
    L.asaga_set_draw_ahead.argtypes = [vp, i32]
    L.asaga_set_draw_ahead.restype = i32
    L.asaga_batch_set_row_paths.argtypes = [vp, vp, vp]
    L.asaga_batch_set_row_paths.restype = i32
    L.asaga_batch_reset.argtypes = [vp]
    L.asaga_batch_reset.restype = i32
    L.asaga_batch_cancel.argtypes = [vp]
    L.asaga_batch_cancel.restype = i32
    L.asaga_destroy.argtypes = [vp]
    L.asaga_destroy.restype = None
    L.asaga_batch_create.argtypes = [P(vp), i32, P(asaga_problem), P(asaga_options)]
    L.asaga_batch_run.argtypes = [vp, dbl, dbl, vp, vp]
    L.asaga_batch_autotune.argtypes = [vp, dbl, vp]
    L.asaga_batch_set_schedule.argtypes = [vp, vp, vp]
    L.asaga_batch_get_state.argtypes = [vp, i32, vp, vp, vp]
    L.asaga_batch_get_info.argtypes = [vp, i32, P(asaga_info)]
    L.asaga_batch_objective.argtypes = [vp, vp]
    L.asaga_batch_last_error.argtypes = [vp]
    L.asaga_batch_last_error.restype = ctypes.c_char_p
    L.asaga_batch_destroy.argtypes = [vp]
    L.asaga_batch_destroy.restype = None
    for f in ("asaga_batch_create", "asaga_batch_run", "asaga_batch_autotune", "asaga_batch_set_schedule",
              "asaga_batch_get_state", "asaga_batch_get_info", "asaga_batch_objective"):
        getattr(L, f).restype = i32
    for f in ("asaga_create", "asaga_run", "asaga_run_indices", "asaga_autotune", "asaga_measure_overlap", "asaga_objective", "asaga_full_grad",
              "asaga_recompute_abar", "asaga_get_state", "asaga_set_state", "asaga_get_info"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):  # torch tensor
        assert a.is_contiguous()
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(type(a))


def _check(ctx, status: int):
    if status != OK:
        raise AsagaError(status, asaga_last_error(ctx))


# --------------------------------------------------------------------- calls

def asaga_default_options(**overrides) -> asaga_options:
    o = asaga_options()
    load().asaga_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "lam" or k == "lambda":
            k = "lambda_"
        if k == "loss" and isinstance(v, str):
            v = LOSS[v]
        if k == "storage_dtype" and isinstance(v, str):
            v = DTYPE[v]
        if k == "sampling" and isinstance(v, str):
            v = SAMPLING[v]
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Problem:
    """Holds the arrays of an asaga_problem alive while the struct is in use."""

    def __init__(self, n, d, row_ptr, col_idx, values, values_dtype, labels, dense=False, on_device=False,
                 nnz=None):
        self.keep = (row_ptr, col_idx, values, labels)
        self.struct = asaga_problem(
            n=n, d=d, nnz=(int(nnz) if nnz is not None else (0 if dense else int(len(col_idx)))),
            row_ptr=_ptr(row_ptr), col_idx=_ptr(col_idx), values=_ptr(values),
            values_dtype=DTYPE[values_dtype] if isinstance(values_dtype, str) else values_dtype,
            labels=_ptr(labels), dense=int(dense), on_device=int(on_device))


def host_problem(p, values_dtype: str = "f64") -> Problem:
    """asaga_problem over the host arrays of a generated problem (values sent
    as float64 by default; the library rounds them to the storage type)."""
    np_dt = {"f64": np.float64, "f32": np.float32, "f16": np.float16}
    if values_dtype == "bf16" and p.values.dtype == np.uint16:  # raw bfloat16 bits already
        vals = np.ascontiguousarray(p.values)
    elif p.values.dtype == np.uint16:  # raw bfloat16 bits, widened exactly
        vals = np.ascontiguousarray(p.values_f64(), dtype=np_dt[values_dtype])
    elif values_dtype == "bf16":  # values already on the bf16 grid: keep the top 16 bits
        v32 = np.ascontiguousarray(p.values, dtype=np.float32).view(np.uint32)
        if np.any(v32 & 0xFFFF):
            raise ValueError("values are not exactly representable in bf16")
        vals = (v32 >> 16).astype(np.uint16)
    else:
        vals = np.ascontiguousarray(p.values, dtype=np_dt[values_dtype])
    labels = np.ascontiguousarray(p.labels, dtype=np.float64)
    if p.dense:
        return Problem(p.n, p.d, None, None, vals, values_dtype, labels, dense=True)
    return Problem(p.n, p.d, np.ascontiguousarray(p.row_ptr, dtype=np.int64),
                   np.ascontiguousarray(p.col_idx, dtype=np.int32), vals, values_dtype, labels)


def asaga_create(problem: Problem, options: asaga_options) -> int:
    ctx = ctypes.c_void_p()
    _check(None, load().asaga_create(ctypes.byref(ctx), ctypes.byref(problem.struct), ctypes.byref(options)))
    return ctx.value


def asaga_run(ctx: int, max_epochs: float, target_rel_subopt: float = 0.0, f_star: float = float("nan")):
    """Returns (status, asaga_result); raises only on EINVAL / ENOMEM / ECUDA."""
    r = asaga_result()
    s = load().asaga_run(ctx, float(max_epochs), float(target_rel_subopt), float(f_star), ctypes.byref(r))
    if s in (EINVAL, ENOMEM, ECUDA):
        raise AsagaError(s, asaga_last_error(ctx))
    return s, r


def asaga_autotune(ctx: int, trial_epochs: float = 0.0) -> dict:
    r = asaga_tune_result()
    _check(ctx, load().asaga_autotune(ctx, float(trial_epochs), ctypes.byref(r)))
    return r.as_dict()


def asaga_set_schedule(ctx: int, warps: int, gamma: float, warps_per_block: int = 0) -> None:
    _check(ctx, load().asaga_set_schedule(ctx, int(warps), float(gamma), int(warps_per_block)))


def asaga_set_row_path(ctx: int, threshold: int, group: int) -> None:
    """Rows longer than `threshold` entries (0: all, -1: none) on cores of `group` warps."""
    _check(ctx, load().asaga_set_row_path(ctx, int(threshold), int(group)))


def asaga_set_draw_ahead(ctx: int, on: int) -> None:
    """1: each core draws its next row while an update's gathers are in flight."""
    _check(ctx, load().asaga_set_draw_ahead(ctx, int(on)))


def asaga_cancel(ctx: int) -> None:
    """Asks the asaga_run in progress on ctx (in another thread) to stop."""
    _check(ctx, load().asaga_cancel(ctx))


def asaga_measure_overlap_trace(ctx: int, epochs: float, count: int):
    """(estimates, times): times[2t], times[2t+1] = start and end (ns) of update t."""
    o = asaga_overlap()
    times = np.zeros(2 * count, dtype=np.uint64)
    _check(ctx, load().asaga_measure_overlap_trace(ctx, float(epochs), ctypes.byref(o), _ptr(times), times.size))
    return o.as_dict(), times


def asaga_measure_overlap(ctx: int, epochs: float = 1.0) -> dict:
    o = asaga_overlap()
    _check(ctx, load().asaga_measure_overlap(ctx, float(epochs), ctypes.byref(o)))
    return o.as_dict()


def asaga_run_indices(ctx: int, idx, on_device: bool = False) -> None:
    if not on_device:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
    count = idx.shape[0] if hasattr(idx, "shape") else len(idx)
    _check(ctx, load().asaga_run_indices(ctx, _ptr(idx), int(count), int(on_device)))


def asaga_objective(ctx: int) -> float:
    f = ctypes.c_double()
    _check(ctx, load().asaga_objective(ctx, ctypes.byref(f)))
    return f.value


def asaga_full_grad(ctx: int, want_grad: bool = True):
    """Returns (grad float64[d] or None, |grad|^2)."""
    info = asaga_get_info(ctx)
    g = np.empty(info["d"], dtype=np.float64) if want_grad else None
    n2 = ctypes.c_double()
    _check(ctx, load().asaga_full_grad(ctx, _ptr(g), ctypes.byref(n2)))
    return g, n2.value


def asaga_recompute_abar(ctx: int) -> float:
    drift = ctypes.c_double()
    _check(ctx, load().asaga_recompute_abar(ctx, ctypes.byref(drift)))
    return drift.value


NOALLOC_MAX_D = 524288


def asaga_recompute_abar_noalloc(n, d, row_ptr, col_idx, values, alpha, abar, drift=None, stream=None) -> None:
    """Device-pointer (torch CUDA tensor) form of the allocation-free abar
    recomputation; raises AsagaError on EINVAL / ECUDA."""
    s = load().asaga_recompute_abar_noalloc(int(n), int(d), _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                            _ptr(alpha), _ptr(abar), _ptr(drift), stream)
    _check(None, s)


def asaga_sample_rows(seed: int, n: int, t_begin: int, count: int, sampling="uniform") -> np.ndarray:
    """Rows of updates t_begin .. t_begin+count-1 from the device sampler (int64)."""
    rows = np.empty(max(int(count), 0), dtype=np.int64)
    smp = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    s = load().asaga_sample_rows(int(seed), int(n), smp, int(t_begin), int(count), _ptr(rows) if count else None)
    _check(None, s)
    return rows


def asaga_probe_line_rate(warps: int, pairs: int) -> float:
    """Device ns per (16-byte read, dependent 2-wide reduction) pair on one state line."""
    ns = ctypes.c_double()
    _check(None, load().asaga_probe_line_rate(int(warps), int(pairs), ctypes.byref(ns)))
    return ns.value


def asaga_get_state(ctx: int):
    """Returns (x float32[d], abar float32[d], alpha float32[n])."""
    info = asaga_get_info(ctx)
    x = np.empty(info["d"], dtype=np.float32)
    abar = np.empty(info["d"], dtype=np.float32)
    alpha = np.empty(info["n"], dtype=np.float32)
    _check(ctx, load().asaga_get_state(ctx, _ptr(x), _ptr(abar), _ptr(alpha)))
    return x, abar, alpha


def asaga_set_state(ctx: int, x=None, abar=None, alpha=None, updates_done: int = 0) -> None:
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    x, abar, alpha = conv(x), conv(abar), conv(alpha)
    _check(ctx, load().asaga_set_state(ctx, _ptr(x), _ptr(abar), _ptr(alpha), int(updates_done)))


def asaga_get_info(ctx: int) -> dict:
    i = asaga_info()
    _check(ctx, load().asaga_get_info(ctx, ctypes.byref(i)))
    return i.as_dict()


def asaga_last_error(ctx: Optional[int]) -> str:
    return load().asaga_last_error(ctx).decode()


def asaga_status_string(s: int) -> str:
    return load().asaga_status_string(int(s)).decode()


def asaga_destroy(ctx: Optional[int]) -> None:
    if ctx:
        load().asaga_destroy(ctx)


class Context:
    """Owning wrapper: creates a context from a generated problem and frees it."""

    def __init__(self, p, *, storage: Optional[str] = None, values_dtype: str = "f64", **options):
        opts = dict(loss=p.loss, lam=p.lam, storage_dtype=storage or p.storage)
        if opts["storage_dtype"] == "f64":
            opts["storage_dtype"] = "f32"
        opts.update(options)
        self.problem = host_problem(p, values_dtype)
        self.options = asaga_default_options(**opts)
        self.ctx = asaga_create(self.problem, self.options)

    def close(self):
        if self.ctx:
            asaga_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------- batches

def _bcheck(b, status: int):
    if status != OK:
        raise AsagaError(status, load().asaga_batch_last_error(b).decode())


def asaga_batch_create(problems, options) -> int:
    n = len(problems)
    P = (asaga_problem * n)(*[p.struct for p in problems])
    O = (asaga_options * n)(*options)
    b = ctypes.c_void_p()
    _bcheck(None, load().asaga_batch_create(ctypes.byref(b), n, P, O))
    return b.value


def asaga_batch_run(b: int, count: int, max_epochs: float, target: float = 0.0, f_star=None):
    """Returns (status, [asaga_result] * count); raises on EINVAL / ENOMEM / ECUDA."""
    res = (asaga_result * count)()
    fs = None if f_star is None else np.ascontiguousarray(f_star, dtype=np.float64)
    s = load().asaga_batch_run(b, float(max_epochs), float(target), _ptr(fs), ctypes.cast(res, ctypes.c_void_p))
    if s in (EINVAL, ENOMEM, ECUDA):
        raise AsagaError(s, load().asaga_batch_last_error(b).decode())
    return s, list(res)


def asaga_batch_cancel(b: int) -> None:
    """Asks the asaga_batch_run in progress (in another thread) to stop."""
    _bcheck(b, load().asaga_batch_cancel(b))


def asaga_batch_autotune(b: int, count: int, trial_epochs: float = 0.0) -> list:
    res = (asaga_tune_result * count)()
    _bcheck(b, load().asaga_batch_autotune(b, float(trial_epochs), ctypes.cast(res, ctypes.c_void_p)))
    return [r.as_dict() for r in res]


def asaga_batch_set_schedule(b: int, warps=None, gamma=None) -> None:
    w = None if warps is None else np.ascontiguousarray(warps, dtype=np.int32)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    _bcheck(b, load().asaga_batch_set_schedule(b, _ptr(w), _ptr(g)))


def asaga_batch_set_row_paths(b: int, threshold, group) -> None:
    t = np.ascontiguousarray(threshold, dtype=np.int64)
    g = np.ascontiguousarray(group, dtype=np.int32)
    _bcheck(b, load().asaga_batch_set_row_paths(b, _ptr(t), _ptr(g)))


def asaga_batch_reset(b: int) -> None:
    """Every instance back to x = 0 (the schedule stays)."""
    _bcheck(b, load().asaga_batch_reset(b))


def asaga_batch_get_state(b: int, i: int, d: int, n: int):
    x = np.empty(d, dtype=np.float32)
    abar = np.empty(d, dtype=np.float32)
    alpha = np.empty(n, dtype=np.float32)
    _bcheck(b, load().asaga_batch_get_state(b, int(i), _ptr(x), _ptr(abar), _ptr(alpha)))
    return x, abar, alpha


def asaga_batch_get_info(b: int, i: int) -> dict:
    info = asaga_info()
    _bcheck(b, load().asaga_batch_get_info(b, int(i), ctypes.byref(info)))
    return info.as_dict()


def asaga_batch_objective(b: int, count: int) -> np.ndarray:
    f = np.empty(count, dtype=np.float64)
    _bcheck(b, load().asaga_batch_objective(b, _ptr(f)))
    return f


def asaga_batch_destroy(b) -> None:
    if b:
        load().asaga_batch_destroy(b)


class Batch:
    """Owning wrapper over a batch of generated problems."""

    def __init__(self, problems, *, storage: str, values_dtype: str = "f64", per_instance=None, structs=None,
                 **options):
        """problems: generated problems (their loss and lambda set each
        instance's options); structs: prebuilt asaga.Problem objects for them
        (e.g. over device arrays), else host_problem(p, values_dtype)."""
        self.problems = problems
        self.structs = structs if structs is not None else [host_problem(p, values_dtype) for p in problems]
        opts = []
        for k, p in enumerate(problems):
            o = dict(loss=p.loss, lam=p.lam, storage_dtype=storage, seed=k)
            o.update(options)
            if per_instance:
                o.update(per_instance[k])
            opts.append(asaga_default_options(**o))
        self.b = asaga_batch_create(self.structs, opts)
        self.count = len(problems)

    def close(self):
        if self.b:
            asaga_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
