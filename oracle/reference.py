"""Float64 CPU checker for the ASAGA solver (TEST INFRASTRUCTURE ONLY).

Everything here is a plain restatement of arXiv:1606.04809 in float64, written
for a reader to check by eye against the paper:

* ``objective`` / ``gradient`` / ``hessian`` -- the finite-sum objective of
  Eq. finiteSum with the l2-logistic model of Sec. 4.1 (and the squared loss
  used for the ridge workload);
* ``reweighting`` -- D = diag(1/p_v), p_v the fraction of rows whose support
  contains v (Sec. 2, Sparse SAGA);
* ``sparse_saga`` -- the serial Sparse SAGA iteration with the projected l2
  term (Eq. SparseSAGA and Sec. 4.2), run by the C file ``saga_ref.c``;
* ``dense_saga_step`` -- the original SAGA update (Eq. SAGAupdate), used only
  to check the sparse variant against it;
* ``lagged_saga`` -- the same dense SAGA iteration with lagged updates
  (App. F), the serial baseline the paper compares Sparse SAGA with;
* ``splitmix64`` / ``sampler_indices`` -- the published SplitMix64 generator
  and the row sampling built on it, written independently of the solver's;
* ``newton`` / ``ridge_closed_form`` -- exact minimisers used to certify f*.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may use
this module.  It shares no code with the solver.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.special

from . import build as _build

LOSS_CODES = {"logistic": 0, "squared": 1}

_lib = None


def lib():
    """The C part of the checker, built on first use."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.oracle_sparse_saga.argtypes = [i64, i64, dp, dp, dp, dp, i32, ctypes.c_double,
                                         ctypes.c_double, dp, dp, dp, dp, dp, i64]
        L.oracle_sparse_saga.restype = i32
        L.oracle_row_derivatives.argtypes = [i64, dp, dp, dp, dp, i32, dp, dp]
        L.oracle_row_derivatives.restype = None
        L.oracle_lagged_saga.argtypes = [i64, i64, dp, dp, dp, dp, i32, ctypes.c_double,
                                         ctypes.c_double, dp, dp, dp, dp, dp, i64, i64]
        L.oracle_lagged_saga.restype = i32
        L.oracle_lagged_catch_up.argtypes = [i64, ctypes.c_double, ctypes.c_double, dp, dp, dp, i64]
        L.oracle_lagged_catch_up.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# problem
# --------------------------------------------------------------------------

def csr(p) -> scipy.sparse.csr_matrix:
    return scipy.sparse.csr_matrix((p.values, p.col_idx, p.row_ptr), shape=(p.n, p.d))


def margins(p, x: np.ndarray) -> np.ndarray:
    """z_i = a_i . x for every row."""
    return csr(p) @ np.asarray(x, dtype=np.float64)


def phi(loss: str, z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-sample loss: logistic log(1 + exp(-y z)) (Sec. 4.1), squared (z-y)^2/2."""
    if loss == "logistic":
        return np.logaddexp(0.0, -y * z)
    return 0.5 * (z - y) ** 2


def phi_prime(loss: str, z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d phi / dz: logistic -y / (1 + exp(y z)) = -y sigmoid(-y z); squared z - y."""
    if loss == "logistic":
        return -y * scipy.special.expit(-y * z)
    return z - y


def phi_second(loss: str, z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d^2 phi / dz^2 (labels +-1 for logistic): s (1 - s), s = sigmoid(y z); squared 1."""
    if loss == "logistic":
        s = scipy.special.expit(y * z)
        return s * (1.0 - s)
    return np.ones_like(z)


def objective(p, x: np.ndarray) -> float:
    """f(x) = 1/n sum_i phi_i(a_i.x) + lambda/2 |x|^2 (Eq. finiteSum, Sec. 4.1)."""
    x = np.asarray(x, dtype=np.float64)
    z = margins(p, x)
    return float(np.mean(phi(p.loss, z, p.labels)) + 0.5 * p.lam * np.dot(x, x))


def gradient(p, x: np.ndarray) -> np.ndarray:
    """grad f(x) = 1/n A^T phi'(A x) + lambda x."""
    x = np.asarray(x, dtype=np.float64)
    z = margins(p, x)
    return csr(p).T @ phi_prime(p.loss, z, p.labels) / p.n + p.lam * x


def hessian(p, x: np.ndarray) -> np.ndarray:
    """Dense Hessian 1/n A^T diag(phi'') A + lambda I (small d only)."""
    A = csr(p)
    w = phi_second(p.loss, margins(p, x), p.labels) / p.n
    H = (A.T @ scipy.sparse.diags(w) @ A).toarray()
    H[np.diag_indices_from(H)] += p.lam
    return H


def lipschitz(p) -> float:
    """Smoothness constant of the components Sparse SAGA samples.

    With the l2 term projected as in Sec. 4.2, the update of row i is the
    gradient step of f_i(x) = phi_i(a_i.x) + lambda/2 sum_{v in S_i} D_v x_v^2
    (their mean over i is f, since E[D_i] = I on touched coordinates), whose
    Hessian is phi'' a_i a_i^T + lambda D_i with phi'' <= c (c = 1/4 logistic,
    1 squared).  So L = max_i (c |a_i|^2 + lambda max_{v in S_i} D_v).  With
    the paper's lambda = 1/n the second term is 1/|{j : v in S_j}| <= 1."""
    A = csr(p)
    r2 = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    D = reweighting(p)
    rows = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
    dmax = np.zeros(p.n)
    np.maximum.at(dmax, rows, D[p.col_idx])
    c = 0.25 if p.loss == "logistic" else 1.0
    return float(np.max(c * r2 + p.lam * dmax))


def column_counts(p) -> np.ndarray:
    """|{i : v in S_i}| for every column v, S_i the stored pattern of row i."""
    return np.bincount(p.col_idx, minlength=p.d).astype(np.int64)


def reweighting(p) -> np.ndarray:
    """Diagonal of D: 1/p_v with p_v = |{i : v in S_i}| / n (Sec. 2).  Columns
    that no row touches get 0 (they are never updated)."""
    cnt = column_counts(p)
    D = np.zeros(p.d)
    nz = cnt > 0
    D[nz] = p.n / cnt[nz]
    return D


def sparsity_delta(p) -> float:
    """Delta = max_v |{i : v in S_i}| / n (Sec. 3.4, Definition 'Sparsity')."""
    return float(column_counts(p).max() / p.n)


# --------------------------------------------------------------------------
# Sparse SAGA (C) and the original SAGA step (Python, for comparison)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class State:
    x: np.ndarray      # float64[d]
    alpha: np.ndarray  # float64[n]  (scalar memory per sample)
    abar: np.ndarray   # float64[d]  (running average of alpha_i a_i)

    @staticmethod
    def zeros(p) -> "State":
        return State(np.zeros(p.d), np.zeros(p.n), np.zeros(p.d))

    def copy(self) -> "State":
        return State(self.x.copy(), self.alpha.copy(), self.abar.copy())


def sparse_saga(p, state: State, idx: np.ndarray, gamma: float, D: Optional[np.ndarray] = None) -> State:
    """Runs len(idx) serial Sparse SAGA iterations in place (row idx[t] at
    iteration t) and returns the state."""
    L = lib()
    if D is None:
        D = reweighting(p)
    rp = np.ascontiguousarray(p.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(p.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(p.values, dtype=np.float64)
    lb = np.ascontiguousarray(p.labels, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    for a in (state.x, state.alpha, state.abar):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    rc = L.oracle_sparse_saga(p.n, p.d, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lb), LOSS_CODES[p.loss],
                              float(p.lam), float(gamma), _ptr(D), _ptr(state.x), _ptr(state.alpha),
                              _ptr(state.abar), _ptr(ix), ix.size)
    if rc != 0:
        raise ValueError("index out of range")
    return state


def lagged_saga(p, state: State, idx: np.ndarray, gamma: float) -> State:
    """Runs len(idx) steps of dense SAGA (Eq. SAGAupdate) in place with the
    lagged-update scheme of App. F (C file ``saga_ref.c``): per step only the
    sampled support is touched, the other coordinates catch up in closed
    form when next read, and all of them at the end.  For comparison with
    Sparse SAGA only; the solver has no counterpart."""
    rp = np.ascontiguousarray(p.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(p.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(p.values, dtype=np.float64)
    lb = np.ascontiguousarray(p.labels, dtype=np.float64)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    last = np.zeros(p.d, dtype=np.int64)
    for a in (state.x, state.alpha, state.abar):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    L = lib()
    rc = L.oracle_lagged_saga(p.n, p.d, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lb), LOSS_CODES[p.loss],
                              float(p.lam), float(gamma), _ptr(state.x), _ptr(state.alpha),
                              _ptr(state.abar), _ptr(last), _ptr(ix), ix.size, 0)
    if rc != 0:
        raise ValueError("index out of range")
    L.oracle_lagged_catch_up(p.d, float(p.lam), float(gamma), _ptr(state.x), _ptr(state.abar),
                             _ptr(last), ix.size)
    return state


# --------------------------------------------------------------------------
# row sampling: Algorithm 2 draws i uniformly (with replacement) before it
# reads anything.  The stream is the published SplitMix64 generator (Steele,
# Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
# 2014); update t takes the generator's (t+1)-th output u_t for a given seed
# and the row floor(u_t n / 2^64).
# --------------------------------------------------------------------------
_SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> list:
    """The first `count` outputs of SplitMix64 seeded with `seed` (plain
    Python integers, one step at a time)."""
    out, state = [], seed & _M64
    for _ in range(count):
        state = (state + _SPLITMIX_GAMMA) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def sampler_indices(seed: int, n: int, t_begin: int, count: int) -> np.ndarray:
    """Rows of updates t_begin .. t_begin+count-1 (int64), computed with exact
    integer arithmetic per update."""
    rows = np.empty(count, dtype=np.int64)
    for j in range(count):
        state = (seed + (t_begin + j + 1) * _SPLITMIX_GAMMA) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        rows[j] = ((z ^ (z >> 31)) * n) >> 64
    return rows


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def permutation_indices(seed: int, n: int, t_begin: int, count: int) -> np.ndarray:
    """Rows of updates t_begin .. t_begin+count-1 when every epoch visits each
    row once (a sampling variant the paper does not use; the solver's
    specification of it is restated here): epoch e = t // n sends position
    p = t - e n through a 4-round balanced Feistel network on 2h bits
    (4^h >= n, h >= 1), keyed by the (e+1)-th SplitMix64 output for seed xor
    0xD1B54A32D192ED03, repeating the network until the value is below n."""
    b = (n - 1).bit_length()
    h = max(1, (b + 1) // 2)
    mask = (1 << h) - 1
    rows = np.empty(count, dtype=np.int64)
    keys = {}
    for j in range(count):
        t = t_begin + j
        e, pos = divmod(t, n)
        if e not in keys:
            keys[e] = _mix64(((seed ^ 0xD1B54A32D192ED03) + (e + 1) * _SPLITMIX_GAMMA) & _M64)
        key = keys[e]
        x = pos
        while True:
            left, right = x >> h, x & mask
            for r in range(4):
                f = _mix64(((key ^ right) + (r + 1) * _SPLITMIX_GAMMA) & _M64) & mask
                left, right = right, left ^ f
            x = (left << h) | right
            if x < n:
                break
        rows[j] = x
    return rows


def row_derivatives(p, x: np.ndarray) -> np.ndarray:
    """phi'_i(a_i.x) for every i, row by row in float64 (C)."""
    out = np.empty(p.n)
    rp = np.ascontiguousarray(p.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(p.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(p.values, dtype=np.float64)
    lb = np.ascontiguousarray(p.labels, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    lib().oracle_row_derivatives(p.n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lb), LOSS_CODES[p.loss],
                                 _ptr(xx), _ptr(out))
    return out


def abar_from_scratch(p, alpha: np.ndarray) -> np.ndarray:
    """abar = 1/n sum_i alpha_i a_i (Sec. 2)."""
    return csr(p).T @ np.asarray(alpha, dtype=np.float64) / p.n


def dense_saga_step(p, state: State, i: int, gamma: float) -> State:
    """One step of the original, dense SAGA update (Eq. SAGAupdate) in place:
    x+ = x - gamma (f'_i(x) - alpha_i a_i + abar) with f'_i(x) = phi'_i a_i +
    lambda x, i.e. the data term remembered as the scalar alpha_i (App. G.2)
    and the l2 term's gradient taken exactly and unprojected.  This is the
    D = I counterpart of the Sec. 4.2 update; it serves only to check the
    sparse variant against it."""
    A = csr(p)
    a = A.getrow(i).toarray().ravel()
    g = float(phi_prime(p.loss, np.array([a @ state.x]), p.labels[i : i + 1])[0])
    fprime_i = g * a + p.lam * state.x
    memory_i = state.alpha[i] * a
    state.x = state.x - gamma * (fprime_i - memory_i + state.abar)
    state.abar = state.abar + (g - state.alpha[i]) * a / p.n
    state.alpha[i] = g
    return state


# --------------------------------------------------------------------------
# exact minimisers and f* certification
# --------------------------------------------------------------------------

def ridge_closed_form(p) -> np.ndarray:
    """x* = (A^T A / n + lambda I)^{-1} A^T y / n (squared loss, textbook normal equations)."""
    assert p.loss == "squared"
    A = csr(p)
    M = (A.T @ A).toarray() / p.n
    M[np.diag_indices_from(M)] += p.lam
    rhs = A.T @ p.labels / p.n
    c = scipy.linalg.cho_factor(M)
    return scipy.linalg.cho_solve(c, rhs)


def newton(p, x0: Optional[np.ndarray] = None, tol: float = 1e-14, max_iter: int = 100) -> np.ndarray:
    """Newton's method with Cholesky solves (small d only), until |grad f| <= tol."""
    x = np.zeros(p.d) if x0 is None else np.array(x0, dtype=np.float64)
    for _ in range(max_iter):
        g = gradient(p, x)
        if np.linalg.norm(g) <= tol:
            break
        H = hessian(p, x)
        step = scipy.linalg.cho_solve(scipy.linalg.cho_factor(H), g)
        # damped step: backtrack on f (needed only far from the optimum)
        f0, s = objective(p, x), 1.0
        while s > 1e-8 and objective(p, x - s * step) > f0 + 1e-16 * abs(f0):
            s *= 0.5
        x = x - s * step
    return x


def suboptimality_bound(p, x: np.ndarray) -> float:
    """f(x) - f* <= |grad f(x)|^2 / (2 mu) with mu >= lambda (strong convexity)."""
    g = gradient(p, x)
    return float(np.dot(g, g) / (2.0 * p.lam))


def certified_fstar(p, index_stream, *, gamma: Optional[float] = None, rel_tol: float = 1e-9,
                    max_epochs: int = 400, check_every: int = 2, log=None) -> dict:
    """f* of ``p`` in float64: serial Sparse SAGA epochs until the strong-
    convexity bound certifies f(x) - f* <= rel_tol |f(x)|.

    ``index_stream(epoch)`` returns the n row indices of that epoch (sampled by
    the caller).  Returns {'fstar', 'bound', 'epochs', 'x'}; fstar = f(x) at the
    certified x, which exceeds the true minimum by at most ``bound``."""
    L = lipschitz(p)
    gamma = 1.0 / (3.0 * L) if gamma is None else gamma
    D = reweighting(p)
    st = State.zeros(p)
    for ep in range(1, max_epochs + 1):
        sparse_saga(p, st, index_stream(ep), gamma, D)
        if ep % check_every == 0 or ep == max_epochs:
            f = objective(p, st.x)
            b = suboptimality_bound(p, st.x)
            if log:
                log(f"epoch {ep}: f={f:.17g} bound={b:.3e}")
            if not (np.isfinite(f) and np.isfinite(b)):
                raise RuntimeError(f"serial Sparse SAGA diverged at epoch {ep}")
            if b <= rel_tol * abs(f):
                return {"fstar": f, "bound": b, "epochs": ep, "x": st.x.copy()}
    raise RuntimeError("f* not certified within max_epochs")


def overlap_estimates(times: np.ndarray) -> dict:
    """The overlap tau of Assumption 1 estimated from a run's trace as App. E.2
    does, written out plainly (O(count^2) comparisons: small traces only).

    times[2t], times[2t+1]: when update t started (before its reads) and
    ended (after its writes).  Iterations r and t overlap when at some point
    they are processed concurrently, i.e. their closed intervals intersect;
    overlap(t) counts the other updates that do.  App. E.2 averages the
    overlap over 100 iterations (here: consecutive windows of 100 updates in
    start order, ties in update order, a trailing partial window dropped) and
    takes the largest such average; tau_mean and tau_max are the plain mean
    and maximum over all updates."""
    t = np.asarray(times, dtype=np.uint64).reshape(-1, 2)
    start, end = t[:, 0], t[:, 1]
    count = start.size
    ov = np.empty(count, dtype=np.int64)
    for u in range(count):
        hits = (start <= end[u]) & (end >= start[u])
        ov[u] = int(np.count_nonzero(hits)) - 1  # not itself
    order = np.lexsort((np.arange(count), start))
    ov_sorted = ov[order]
    paper = 0.0
    for w in range(count // 100):
        paper = max(paper, float(np.sum(ov_sorted[100 * w:100 * (w + 1)])) / 100.0)
    return {"updates": count, "tau_mean": float(np.sum(ov)) / count, "tau_max": float(np.max(ov)),
            "tau_paper": paper, "window_ns_mean": float(np.mean((end - start).astype(np.float64))),
            "overlaps": ov}
