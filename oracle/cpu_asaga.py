"""Multi-threaded lock-free ASAGA on the host cores (C file ``asaga_cpu.c``):
Algorithm 2 with compare-and-swap updates (App. G.2), the paper's own kind
of implementation, used as a CPU timing baseline.

TEST INFRASTRUCTURE ONLY: only the tests and the benchmark's CPU-baseline
leg may use it.  Its iterate depends on the thread interleaving, so it is
not a checker; with one thread it is the serial Sparse SAGA of
``reference.sparse_saga`` on the SplitMix64 row stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import reference as R

_fn = None


def _lib():
    global _fn
    if _fn is None:
        L = R.lib()
        i64, i32, dp, dbl, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64
        L.cpu_asaga.argtypes = [i64, i64, dp, dp, dp, dp, i32, dbl, dbl, dp, dp, dp, dp, u64, u64, i64, i32, dp, i64]
        L.cpu_asaga.restype = i32
        _fn = L.cpu_asaga
    return _fn


class Runner:
    """Holds the contiguous float64 copies of a problem and runs updates on
    a shared state (x, alpha, abar) in place."""

    def __init__(self, p, threads: int | None = None, D: np.ndarray | None = None):
        self.p = p
        self.threads = int(threads or os.cpu_count() or 1)
        self.rp = np.ascontiguousarray(p.row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(p.col_idx, dtype=np.int32)
        self.va = np.ascontiguousarray(p.values, dtype=np.float64)
        self.lb = np.ascontiguousarray(p.labels, dtype=np.float64)
        self.D = np.ascontiguousarray(R.reweighting(p) if D is None else D, dtype=np.float64)
        self.max_row = int(np.max(np.diff(self.rp))) if p.n > 0 else 0
        self.zbuf = np.empty(max(1, self.threads * max(1, self.max_row)))
        self.t = 0

    def run(self, state: R.State, count: int, gamma: float, seed: int) -> R.State:
        p = self.p
        for a in (state.x, state.alpha, state.abar):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        rc = _lib()(p.n, p.d, R._ptr(self.rp), R._ptr(self.ci), R._ptr(self.va), R._ptr(self.lb),
                    R.LOSS_CODES[p.loss], float(p.lam), float(gamma), R._ptr(self.D), R._ptr(state.x),
                    R._ptr(state.alpha), R._ptr(state.abar), int(seed) & ((1 << 64) - 1), self.t, int(count),
                    self.threads, R._ptr(self.zbuf), max(1, self.max_row))
        if rc != 0:
            raise RuntimeError("could not start the worker threads")
        self.t += int(count)
        return state
