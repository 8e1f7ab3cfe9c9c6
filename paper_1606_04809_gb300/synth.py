"""Seeded synthetic inputs for the ASAGA solver and for its CPU checker.

This module only makes data: CSR matrices, labels and index streams. It holds
none of the solver's arithmetic (no loss, no gradient, no reweighting), so both
the CUDA path and the CPU checker can consume the same inputs without sharing
any of the method.

The shapes follow the workloads of the paper's experiments (Sec. 4.1 and the
dataset table of App. E.2): an RCV1-like sparse logistic problem, a URL-like
very sparse high-dimensional one with binary row-normalised features, and a
Covtype-like dense low-dimensional one (used here as a ridge problem). The
datasets themselves are not available; every generator here is a seeded
stand-in with the same n, d, support-size statistics and value distribution.

Values are emitted as float64 numbers that are exactly representable in the
problem's storage dtype (fp32, bf16 or fp16), so that the device copy and the
float64 checker see the same matrix bit for bit.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import dataclasses
import hashlib
import math
import os
import subprocess
import threading
from typing import Optional

import numpy as np

STORAGE_DTYPES = ("f64", "f32", "bf16", "f16")


@dataclasses.dataclass
class Problem:
    """A finite-sum problem min_x 1/n sum_i phi_i(a_i.x) + lam/2 |x|^2 in CSR form.

    row_ptr: int64[n+1]; col_idx: int32[nnz] (sorted within each row, distinct);
    values: float64[nnz], exactly representable in ``storage``;
    labels: float64[n] (+-1 for logistic, real targets for squared).
    ``dense`` marks a fully dense matrix (row i holds columns 0..d-1 in order);
    the CSR arrays are still filled so that every consumer can read it as CSR.
    """

    name: str
    n: int
    d: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    values: np.ndarray
    labels: np.ndarray
    loss: str  # "logistic" | "squared"
    lam: float
    storage: str = "f32"
    dense: bool = False
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def dense_values(self) -> np.ndarray:
        """Row-major n*d view of a dense problem's values."""
        assert self.dense
        return self.values.reshape(self.n, self.d)

    def values_f64(self) -> np.ndarray:
        """The values as float64 (bfloat16 bits widened exactly when the problem
        holds raw bits, meta['values_bits'] == 'bf16')."""
        if self.values.dtype == np.uint16:
            return (self.values.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return self.values

    def fingerprint(self) -> dict:
        """Platform-stable summary used to check that a stored result belongs to
        the same generated problem: exact integer structure plus value sums
        (for the C generator's problems: the digest of its per-row checksums,
        which cover lengths, columns, stored values and labels)."""
        if "row_digest" in self.meta:
            return {"row_digest": self.meta["row_digest"], "n": self.n, "d": self.d, "nnz": self.nnz}
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(self.row_ptr, dtype="<i8").tobytes())
        h.update(np.ascontiguousarray(self.col_idx, dtype="<i4").tobytes())
        if self.loss == "logistic":
            h.update(np.ascontiguousarray(self.labels > 0).tobytes())
        return {
            "structure_sha256": h.hexdigest(),
            "n": self.n,
            "d": self.d,
            "nnz": self.nnz,
            "sum_values": float(np.sum(self.values)),
            "sum_abs_values": float(np.sum(np.abs(self.values))),
            "sum_labels": float(np.sum(self.labels)),
        }


# --------------------------------------------------------------------------
# value quantisation to the storage grid (data preparation, not the method)
# --------------------------------------------------------------------------

def to_storage_grid(v: np.ndarray, storage: str) -> np.ndarray:
    """Round float64 values to the nearest number of the storage dtype and
    return them as float64 (exactly representable in that dtype)."""
    v = np.asarray(v, dtype=np.float64)
    if storage == "f64":
        return v.copy()
    if storage == "f32":
        return v.astype(np.float32).astype(np.float64)
    if storage == "f16":
        return v.astype(np.float16).astype(np.float64)
    if storage == "bf16":
        f = v.astype(np.float32)
        bits = f.view(np.uint32).astype(np.uint64)
        # round-to-nearest-even on the top 16 bits (no NaN/Inf in the data)
        bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
        return bits.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(f"unknown storage dtype {storage!r}")


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _clipped_lognormal_lengths(rng, n, mean, lo, hi, sigma) -> np.ndarray:
    mu = math.log(mean) - 0.5 * sigma * sigma
    k = np.rint(np.exp(mu + sigma * rng.standard_normal(n)))
    return np.clip(k, lo, hi).astype(np.int64)


def _zipf_cdf(d: int, s: float) -> np.ndarray:
    w = np.arange(1, d + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _inverse_cdf(cdf: np.ndarray, u: np.ndarray) -> np.ndarray:
    """First index k with cdf[k] > u (= searchsorted(side='right')), clipped to
    the last index, via a guide table followed by a short forward scan."""
    m = 16 * cdf.size
    guide = np.searchsorted(cdf, np.arange(m, dtype=np.float64) / m, side="right")
    k = guide[np.minimum((u * m).astype(np.int64), m - 1)]
    last = cdf.size - 1
    np.minimum(k, last, out=k)
    act = np.nonzero((cdf[k] <= u) & (k < last))[0]
    while act.size:
        k[act] += 1
        act = act[(cdf[k[act]] <= u[act]) & (k[act] < last)]
    return k


def _distinct_columns(lengths: np.ndarray, d: int, make_draw, chunk_rows: int = 32768):
    """For each row i draw columns one at a time (with replacement) and keep
    the first lengths[i] distinct ones; columns are returned sorted within each
    row.  Rows are processed in fixed chunks; chunk c draws from
    ``make_draw(c)``, its own seeded stream, so chunks can run on several
    threads with a result that does not depend on the thread count.
    Returns (row_ptr, col_idx)."""
    n = lengths.shape[0]
    if np.any(lengths > d):
        raise ValueError("a row is longer than d")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    col_idx = np.empty(int(row_ptr[-1]), dtype=np.int32)

    def one_chunk(c):
        draw = make_draw(c)
        todo = np.arange(c * chunk_rows, min(n, (c + 1) * chunk_rows))
        over = 1.25
        while todo.size:
            k = lengths[todo]
            m = np.ceil(k * over).astype(np.int64) + 4
            rows_local = np.repeat(np.arange(todo.size, dtype=np.int64), m)
            cols = draw(int(m.sum())).astype(np.int64)
            pbits = max(1, int(cols.size - 1).bit_length())
            key = (rows_local * d + cols).astype(np.uint64)
            comb = np.sort((key << np.uint64(pbits)) | np.arange(cols.size, dtype=np.uint64))
            ks = comb >> np.uint64(pbits)
            first = np.ones(ks.size, dtype=bool)
            first[1:] = ks[1:] != ks[:-1]
            keep = np.sort((comb[first] & np.uint64((1 << pbits) - 1)).astype(np.int64))
            kr = rows_local[keep]
            cnt = np.bincount(kr, minlength=todo.size)
            start = np.zeros(todo.size, dtype=np.int64)
            np.cumsum(cnt[:-1], out=start[1:])
            rank = np.arange(keep.size, dtype=np.int64) - start[kr]
            done = cnt >= k
            ok = (rank < k[kr]) & done[kr]
            rc = np.sort(kr[ok] * d + cols[keep[ok]])  # sort columns within each row
            kr_ok, cols_ok = rc // d, rc % d
            cs = np.zeros(todo.size + 1, dtype=np.int64)
            np.cumsum(np.where(done, k, 0), out=cs[1:])
            within = np.arange(kr_ok.size, dtype=np.int64) - cs[kr_ok]
            col_idx[row_ptr[todo[kr_ok]] + within] = cols_ok
            todo = todo[~done]
            over *= 2.0

    nchunks = (n + chunk_rows - 1) // chunk_rows
    workers = max(1, min(nchunks, os.cpu_count() or 1, 32))
    if workers == 1:
        for c in range(nchunks):
            one_chunk(c)
    else:
        with concurrent.futures.ThreadPoolExecutor(workers) as ex:
            list(ex.map(one_chunk, range(nchunks)))
    return row_ptr, col_idx


def _normalize_rows(values, row_ptr):
    n = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    ss = np.bincount(rows, weights=values * values, minlength=n)
    return values / np.sqrt(ss)[rows]


def _csr_matvec(row_ptr, col_idx, values, w):
    n = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return np.bincount(rows, weights=values * w[col_idx], minlength=n)


def _signs(v):
    return np.where(v >= 0.0, 1.0, -1.0)  # sign(0) = +1


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def sparse_logistic(
    n: int,
    d: int,
    *,
    k_mean: float,
    k_min: int,
    k_max: int,
    k_sigma: float = 0.0,
    zipf_s: Optional[float] = None,
    values: str = "abs_normal",
    storage: str = "f32",
    lam: Optional[float] = None,
    seed: int = 0,
    name: str = "sparse_logistic",
    permute_columns: bool = True,
) -> Problem:
    """Sparse l2-logistic problem.

    Row lengths: round(lognormal) with the given mean, clipped to [k_min,k_max]
    (k_sigma = 0 gives 1 + Poisson(k_mean - 1), clipped).  Columns: uniform, or
    Zipf(zipf_s) over ranks mapped through a seeded column permutation, drawn
    without replacement within a row.  Values: 'normal' (N(0,1)), 'abs_normal'
    (|N(0,1)|) or 'binary' (ones), each row scaled to unit l2 norm, then
    rounded to the storage grid.  Labels: sign(a_i.w* + 0.1 eps), w* ~ N(0,I).
    """
    r_len, r_col, r_val, r_w, r_eps = (_rng(seed, s) for s in range(1, 6))
    if k_sigma > 0:
        lengths = _clipped_lognormal_lengths(r_len, n, k_mean, k_min, k_max, k_sigma)
    else:
        lengths = np.clip(1 + r_len.poisson(max(k_mean - 1.0, 0.0), n), k_min, k_max).astype(np.int64)
    lengths = np.minimum(lengths, d)
    if zipf_s is None:
        def make_draw(c):
            g = _rng(seed, 100_000 + c)
            return lambda m: g.integers(0, d, m)
    else:
        cdf = _zipf_cdf(d, zipf_s)
        perm = r_col.permutation(d) if permute_columns else np.arange(d)

        def make_draw(c):
            g = _rng(seed, 100_000 + c)
            return lambda m: perm[_inverse_cdf(cdf, g.random(m))]
    row_ptr, col_idx = _distinct_columns(lengths, d, make_draw)
    nnz = int(row_ptr[-1])
    if values == "normal":
        v = r_val.standard_normal(nnz)
    elif values == "abs_normal":
        v = np.abs(r_val.standard_normal(nnz))
    elif values == "binary":
        v = np.ones(nnz)
    else:
        raise ValueError(values)
    v = _normalize_rows(v, row_ptr)
    v = to_storage_grid(v, storage)
    w_star = r_w.standard_normal(d)
    labels = _signs(_csr_matvec(row_ptr, col_idx, v, w_star) + 0.1 * r_eps.standard_normal(n))
    return Problem(
        name=name, n=n, d=d, row_ptr=row_ptr, col_idx=col_idx.astype(np.int32), values=v,
        labels=labels, loss="logistic", lam=(1.0 / n if lam is None else lam), storage=storage,
        meta={"seed": seed, "k_mean": k_mean, "zipf_s": zipf_s, "values": values},
    )


def dense_ridge(n: int, d: int, *, storage: str = "f16", lam: float = 1e-3, seed: int = 0,
                name: str = "dense_ridge") -> Problem:
    """Dense squared-loss problem: features N(0,1) standardised per column,
    rounded to the storage grid; y = A w* + 0.1 eps with w* ~ N(0,I)."""
    r_a, r_w, r_eps = (_rng(seed, s) for s in range(1, 4))
    a = r_a.standard_normal((n, d))
    a = (a - a.mean(axis=0)) / a.std(axis=0)
    a = to_storage_grid(a, storage)
    w_star = r_w.standard_normal(d)
    y = a @ w_star + 0.1 * r_eps.standard_normal(n)
    row_ptr = np.arange(n + 1, dtype=np.int64) * d
    col_idx = np.tile(np.arange(d, dtype=np.int32), n)
    return Problem(
        name=name, n=n, d=d, row_ptr=row_ptr, col_idx=col_idx, values=a.reshape(-1).copy(),
        labels=y, loss="squared", lam=lam, storage=storage, dense=True, meta={"seed": seed},
    )


def sample_indices(n: int, count: int, seed: int, offset: int = 0) -> np.ndarray:
    """Uniform indices in [0,n) drawn with replacement (the sampling the paper
    prescribes), as an int64 stream.  ``offset`` selects a later part of the
    same seeded stream in chunks of ``count``."""
    g = _rng(seed, 1000 + offset)
    return g.integers(0, n, count, dtype=np.int64)


# --------------------------------------------------------------------------
# the five named workloads
# --------------------------------------------------------------------------

def small_logistic(seed: int = 11) -> Problem:
    """n=2000, d=500, ~10 uniform columns per row, N(0,1) values, unit rows, fp64."""
    return sparse_logistic(2000, 500, k_mean=10, k_min=1, k_max=20, values="normal",
                           storage="f64", seed=seed, name="logistic_n2000_d500")


def rcv1_like(seed: int = 21, n: int = 700_000, d: int = 47_000, storage: str = "f32") -> Problem:
    """RCV1-shaped: n=700000, d=47000, row lengths mean 75 in [4,1224] (long
    tail), Zipf(1.1) columns, |N(0,1)| values, unit rows, fp32 storage."""
    return sparse_logistic(n, d, k_mean=75, k_min=4, k_max=1224, k_sigma=0.6, zipf_s=1.1,
                           values="abs_normal", storage=storage, seed=seed,
                           name=f"rcv1like_n{n}_d{d}_{storage}")


def url_like(seed: int = 31, n: int = 2_400_000, d: int = 3_200_000, storage: str = "bf16") -> Problem:
    """URL-shaped: n=2.4M, d=3.2M, row lengths mean 115 in [16,414], Zipf(1.1)
    columns, binary values scaled to unit rows, bf16 storage."""
    return sparse_logistic(n, d, k_mean=115, k_min=16, k_max=414, k_sigma=0.28, zipf_s=1.1,
                           values="binary", storage=storage, seed=seed,
                           name=f"urllike_n{n}_d{d}_{storage}")


def covtype_like(seed: int = 41, n: int = 581_000, d: int = 54, storage: str = "f16") -> Problem:
    """Covtype-shaped ridge: n=581000, d=54 dense, standardised N(0,1), fp16, lam=1e-3."""
    return dense_ridge(n, d, storage=storage, lam=1e-3, seed=seed, name=f"covtypelike_n{n}_d{d}_{storage}")


def logistic_batch(count: int = 256, seed: int = 51, n_range=(10_000, 200_000), d_range=(1_000, 50_000),
                   density_range=(0.005, 0.02), lam_range=(1e-6, 1e-2), storage: str = "bf16") -> list:
    """Independent l2-logistic instances of uneven shape, as in a
    regularisation path: n and d uniform in their ranges, density uniform
    (rows of 1 + Poisson(density*d - 1) entries), Zipf(1.1) columns, |N(0,1)|
    values row-normalised, lambda on a log grid over lam_range (instance k
    gets the k-th grid point), values on the storage grid."""
    g = _rng(seed, 0)
    ns = g.integers(n_range[0], n_range[1] + 1, count)
    ds = g.integers(d_range[0], d_range[1] + 1, count)
    dens = g.uniform(density_range[0], density_range[1], count)
    lams = np.logspace(math.log10(lam_range[0]), math.log10(lam_range[1]), count)
    out = []
    for k in range(count):
        n, d = int(ns[k]), int(ds[k])
        kmean = max(1.0, float(dens[k]) * d)
        out.append(sparse_logistic(n, d, k_mean=kmean, k_min=1, k_max=max(1, min(d, int(4 * kmean) + 4)),
                                   zipf_s=1.1, values="abs_normal", storage=storage, lam=float(lams[k]),
                                   seed=seed * 1000 + k, name=f"batch{seed}_{k}_n{n}_d{d}_{storage}"))
    return out


# --------------------------------------------------------------------------
# the C generator (synth_gen.c) for the full-size batch workload
# --------------------------------------------------------------------------

_GEN_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_gen.c")
_GEN_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libsynthgen.so")
_gen = None
_gen_lock = threading.Lock()


def build_generator(force: bool = False) -> str:
    """Compiles synth_gen.c with gcc (no fast-math, no contraction: the same
    bits on x86-64 and aarch64) into _build/libsynthgen.so."""
    if not force and os.path.exists(_GEN_LIB) and os.path.getmtime(_GEN_LIB) >= os.path.getmtime(_GEN_SRC):
        return _GEN_LIB
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    tmp = _GEN_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-pthread", _GEN_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _generator():
    global _gen
    with _gen_lock:
        if _gen is None:
            L = ctypes.CDLL(build_generator())
            i64, i32, u64, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            L.synth_gen_rows.argtypes = [u64, i64, i64, dbl, i64, i64, vp, i32]
            L.synth_gen_rows.restype = i64
            L.synth_gen_fill.argtypes = [u64, i64, i64, dbl, i64, i64, dbl, i32, vp, vp, vp, vp, vp, vp, i32]
            L.synth_gen_fill.restype = i32
            L.synth_gen_log.argtypes = [dbl]
            L.synth_gen_log.restype = dbl
            L.synth_gen_exp.argtypes = [dbl]
            L.synth_gen_exp.restype = dbl
            _gen = L
        return _gen


def fast_sparse_logistic(n: int, d: int, *, k_mean: float, k_min: int, k_max: int, zipf_s: float = 1.1,
                         storage: str = "bf16", lam: float, seed: int, name: str = "fast_sparse_logistic",
                         values: str = "f64", threads: Optional[int] = None) -> Problem:
    """Sparse l2-logistic problem from the C generator (synth_gen.c):
    row lengths round(k_mean + sqrt(k_mean) N(0,1)) clipped to [k_min, k_max],
    Zipf(zipf_s) columns (distinct within a row, through a seeded column
    permutation), |N(0,1)| values scaled to unit rows on the storage grid
    (f32 or bf16), labels sign(a.w* + 0.1 eps).  values='f64' keeps float64
    values; values='bits' keeps bfloat16 bits (uint16, half the host memory
    of float32; bf16 storage only).  The same bits on every host."""
    if storage not in ("f32", "bf16") or values not in ("f64", "bits") or (values == "bits" and storage != "bf16"):
        raise ValueError("storage f32 or bf16; values 'bits' needs bf16 storage")
    L = _generator()
    threads = int(threads or min(64, os.cpu_count() or 1))
    row_ptr = np.empty(n + 1, dtype=np.int64)
    nnz = L.synth_gen_rows(int(seed), n, d, float(k_mean), int(k_min), int(k_max), row_ptr.ctypes.data, threads)
    if nnz < 0:
        raise ValueError("bad generator arguments")
    col = np.empty(nnz, dtype=np.int32)
    labels = np.empty(n, dtype=np.float64)
    row_hash = np.empty(n, dtype=np.uint64)
    v64 = np.empty(nnz, dtype=np.float64) if values == "f64" else None
    v16 = np.empty(nnz, dtype=np.uint16) if values == "bits" else None
    rc = L.synth_gen_fill(int(seed), n, d, float(k_mean), int(k_min), int(k_max), float(zipf_s),
                          1 if storage == "f32" else 2, row_ptr.ctypes.data, col.ctypes.data,
                          None if v64 is None else v64.ctypes.data, None if v16 is None else v16.ctypes.data,
                          labels.ctypes.data, row_hash.ctypes.data, threads)
    if rc != 0:
        raise RuntimeError("synth_gen_fill failed")
    digest = hashlib.sha256(row_hash.astype("<u8").tobytes()).hexdigest()
    return Problem(name=name, n=n, d=d, row_ptr=row_ptr, col_idx=col, values=v64 if v64 is not None else v16,
                   labels=labels, loss="logistic", lam=float(lam), storage=storage,
                   meta={"seed": seed, "k_mean": k_mean, "zipf_s": zipf_s, "values": "abs_normal",
                         "generator": "synth_gen.c", "row_digest": digest,
                         "values_bits": "bf16" if values == "bits" else None})


# The batch workload at its full size: 256 l2-logistic instances with n
# uniform in [10000, 200000], d uniform in [1000, 50000], density uniform in
# [0.5%, 2%] (mean row length density * d), Zipf(1.1) columns and lambda on
# a log grid from 1e-6 to 1e-2 (instance k takes the k-th point), bf16 values.
FULL_BATCH = dict(count=256, seed=52, n_range=(10_000, 200_000), d_range=(1_000, 50_000),
                  density_range=(0.005, 0.02), lam_range=(1e-6, 1e-2), storage="bf16")


def batch_params(count: int = 256, seed: int = 52, n_range=(10_000, 200_000), d_range=(1_000, 50_000),
                 density_range=(0.005, 0.02), lam_range=(1e-6, 1e-2), storage: str = "bf16") -> list:
    """Shapes of the instances of a batch: n, d, mean row length, row length
    range, lambda and generator seed of each (drawn from a seeded PCG64
    stream; lambda on the log grid)."""
    g = _rng(seed, 0)
    ns = g.integers(n_range[0], n_range[1] + 1, count)
    ds = g.integers(d_range[0], d_range[1] + 1, count)
    dens = g.uniform(density_range[0], density_range[1], count)
    lams = np.logspace(math.log10(lam_range[0]), math.log10(lam_range[1]), count)
    out = []
    for k in range(count):
        n, d = int(ns[k]), int(ds[k])
        kmean = max(1.0, float(dens[k]) * d)
        out.append(dict(k=k, n=n, d=d, k_mean=kmean, k_min=1, k_max=max(1, min(d, int(4 * kmean) + 4)),
                        lam=float(lams[k]), seed=seed * 1000 + k, storage=storage,
                        name=f"batch{seed}_{k}_n{n}_d{d}_{storage}"))
    return out


def batch_instance(spec: dict, *, values: str = "f64", threads: Optional[int] = None) -> Problem:
    """One instance of batch_params, generated by the C generator."""
    return fast_sparse_logistic(spec["n"], spec["d"], k_mean=spec["k_mean"], k_min=spec["k_min"],
                                k_max=spec["k_max"], zipf_s=1.1, storage=spec["storage"], lam=spec["lam"],
                                seed=spec["seed"], name=spec["name"], values=values, threads=threads)
