"""Pins for the float64 CPU checker, against facts the paper and the
mathematics fix independently of the checker's own code (CPU only)."""
import math

import numpy as np
import pytest
import scipy.optimize

from oracle import reference as R
from paper_1606_04809_gb300 import synth


def tiny_sparse(n=8, d=6, loss="logistic", seed=0, k=3, lam=None):
    g = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    row_ptr = [0]
    for i in range(n):
        c = np.sort(g.choice(d, size=k, replace=False))
        rows.append(c)
        vals.append(g.standard_normal(k))
        row_ptr.append(row_ptr[-1] + k)
    col_idx = np.concatenate(rows).astype(np.int32)
    values = np.concatenate(vals)
    labels = np.where(g.standard_normal(n) >= 0, 1.0, -1.0) if loss == "logistic" else g.standard_normal(n)
    return synth.Problem("tiny", n, d, np.array(row_ptr, dtype=np.int64), col_idx, values, labels, loss,
                         lam=(1.0 / n if lam is None else lam), storage="f64")


def tiny_dense(n=7, d=4, loss="squared", seed=1, lam=0.1):
    g = np.random.default_rng(seed)
    a = g.standard_normal((n, d))
    labels = g.standard_normal(n) if loss == "squared" else np.where(g.standard_normal(n) >= 0, 1.0, -1.0)
    return synth.Problem("tinydense", n, d, np.arange(n + 1, dtype=np.int64) * d,
                         np.tile(np.arange(d, dtype=np.int32), n), a.ravel(), labels, loss, lam=lam,
                         storage="f64", dense=True)


def consistent_state(p, seed=3):
    """Random x (zero on untouched columns), random alpha, abar = 1/n sum alpha_i a_i
    accumulated row by row with plain loops."""
    g = np.random.default_rng(seed)
    cnt = np.bincount(p.col_idx, minlength=p.d)
    x = g.standard_normal(p.d) * (cnt > 0)
    alpha = g.standard_normal(p.n)
    abar = np.zeros(p.d)
    for i in range(p.n):
        for k in range(p.row_ptr[i], p.row_ptr[i + 1]):
            abar[p.col_idx[k]] += alpha[i] * p.values[k] / p.n
    return R.State(x, alpha, abar)


# ------------------------------------------------------------ objective pins

def test_logistic_objective_at_zero_is_log2():
    p = tiny_sparse(loss="logistic")
    assert R.objective(p, np.zeros(p.d)) == pytest.approx(math.log(2.0), abs=1e-15)


def test_squared_objective_at_zero():
    p = tiny_sparse(loss="squared")
    assert R.objective(p, np.zeros(p.d)) == pytest.approx(sum(y * y for y in p.labels) / (2 * p.n), rel=1e-15)


def test_logistic_gradient_at_zero():
    # phi'(0) = -b/2 for log(1+exp(-b z)), so grad f(0) = -(1/2n) sum_i b_i a_i
    p = tiny_sparse(loss="logistic", seed=5)
    expect = np.zeros(p.d)
    for i in range(p.n):
        for k in range(p.row_ptr[i], p.row_ptr[i + 1]):
            expect[p.col_idx[k]] -= p.labels[i] * p.values[k] / (2 * p.n)
    np.testing.assert_allclose(R.gradient(p, np.zeros(p.d)), expect, rtol=0, atol=1e-16)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_gradient_matches_finite_differences(loss):
    p = tiny_sparse(loss=loss, seed=7)
    x = np.random.default_rng(8).standard_normal(p.d)
    h = 1e-6
    fd = np.array([(R.objective(p, x + h * e) - R.objective(p, x - h * e)) / (2 * h) for e in np.eye(p.d)])
    np.testing.assert_allclose(R.gradient(p, x), fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_hessian_matches_finite_differences(loss):
    p = tiny_sparse(loss=loss, seed=9)
    x = np.random.default_rng(10).standard_normal(p.d)
    h = 1e-6
    fd = np.array([(R.gradient(p, x + h * e) - R.gradient(p, x - h * e)) / (2 * h) for e in np.eye(p.d)])
    np.testing.assert_allclose(R.hessian(p, x), fd, rtol=1e-6, atol=1e-8)


def test_ridge_closed_form_against_least_squares():
    # (A^T A/n + lam I) x = A^T y/n  <=>  least squares on [A/sqrt(n); sqrt(lam) I] x = [y/sqrt(n); 0]
    p = tiny_dense(n=30, d=5, lam=0.05)
    A = p.dense_values()
    M = np.vstack([A / math.sqrt(p.n), math.sqrt(p.lam) * np.eye(p.d)])
    rhs = np.concatenate([p.labels / math.sqrt(p.n), np.zeros(p.d)])
    x_ls = np.linalg.lstsq(M, rhs, rcond=None)[0]
    x_cf = R.ridge_closed_form(p)
    np.testing.assert_allclose(x_cf, x_ls, rtol=1e-12, atol=1e-13)
    assert np.linalg.norm(R.gradient(p, x_cf)) < 1e-14


def test_newton_matches_derivative_free_minimiser():
    p = tiny_sparse(n=12, d=4, k=2, loss="logistic", seed=11)
    xs = R.newton(p)
    assert np.linalg.norm(R.gradient(p, xs)) < 1e-14
    res = scipy.optimize.minimize(lambda x: R.objective(p, x), np.zeros(p.d), method="Nelder-Mead",
                                  options={"xatol": 1e-10, "fatol": 1e-15, "maxiter": 20000, "maxfev": 40000})
    np.testing.assert_allclose(res.x, xs, atol=1e-6)


def test_one_sample_logistic_optimum_by_bisection():
    # f(x) = log(1+exp(-x)) + lam x^2/2 with a=1, b=+1: optimum solves lam x = 1/(1+exp(x))
    lam = 0.3
    p = synth.Problem("one", 1, 1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                      np.array([1.0]), np.array([1.0]), "logistic", lam=lam, storage="f64")
    lo, hi = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lam * mid - 1.0 / (1.0 + math.exp(mid)) > 0:
            hi = mid
        else:
            lo = mid
    assert R.newton(p)[0] == pytest.approx(lo, abs=1e-14)


# ------------------------------------------------------------ reweighting pins

def test_reweighting_counts_rows():
    p = tiny_sparse(n=9, d=7, k=3, seed=12)
    D = R.reweighting(p)
    for v in range(p.d):
        rows_with_v = sum(1 for i in range(p.n) if v in p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]])
        if rows_with_v == 0:
            assert D[v] == 0.0
        else:
            assert D[v] * rows_with_v == pytest.approx(p.n, rel=1e-15)


def test_expected_projected_reweighting_is_identity():
    # E_i[D_i 1] = 1 on every touched coordinate (App. B, Eq. apxBias)
    p = tiny_sparse(n=10, d=8, k=3, seed=13)
    D = R.reweighting(p)
    acc = np.zeros(p.d)
    for i in range(p.n):
        for k in range(p.row_ptr[i], p.row_ptr[i + 1]):
            acc[p.col_idx[k]] += D[p.col_idx[k]] / p.n
    touched = np.bincount(p.col_idx, minlength=p.d) > 0
    np.testing.assert_allclose(acc[touched], 1.0, rtol=1e-15)


# ------------------------------------------------------------ Sparse SAGA pins

def one_step(p, st, i, gamma, D=None):
    s = st.copy()
    return R.sparse_saga(p, s, np.array([i]), gamma, D)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_sparse_step_is_unbiased(loss):
    """E_i[x+ - x] = -gamma grad f(x) over a uniform i, and equals the mean of the
    original (dense) SAGA step (Sec. 2: E D_i abar = abar; App. B)."""
    p = tiny_sparse(n=8, d=6, k=3, loss=loss, seed=14)
    st = consistent_state(p)
    gamma = 0.37
    mean_sparse = np.mean([one_step(p, st, i, gamma).x - st.x for i in range(p.n)], axis=0)
    mean_dense = np.mean([R.dense_saga_step(p, st.copy(), i, gamma).x - st.x for i in range(p.n)], axis=0)
    np.testing.assert_allclose(mean_sparse, -gamma * R.gradient(p, st.x), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(mean_dense, -gamma * R.gradient(p, st.x), rtol=1e-13, atol=1e-15)


def test_unbiasedness_pin_catches_a_wrong_reweighting():
    """The unbiasedness pin is sharp: the same step with D = I (a plausible
    mistake on sparse data) is biased."""
    p = tiny_sparse(n=8, d=6, k=3, seed=14)
    st = consistent_state(p)
    gamma = 0.37
    mean_wrong = np.mean([one_step(p, st, i, gamma, D=np.ones(p.d)).x - st.x for i in range(p.n)], axis=0)
    assert np.max(np.abs(mean_wrong + gamma * R.gradient(p, st.x))) > 1e-3


def test_sparse_step_equals_dense_step_when_D_is_identity():
    """Fully dense rows give p_v = 1, D = I, and Eq. SparseSAGA reduces to Eq. SAGAupdate."""
    for loss in ("squared", "logistic"):
        p = tiny_dense(n=7, d=4, loss=loss)
        np.testing.assert_array_equal(R.reweighting(p), np.ones(p.d))
        st = consistent_state(p, seed=15)
        for i in range(p.n):
            a = one_step(p, st, i, 0.2)
            b = R.dense_saga_step(p, st.copy(), i, 0.2)
            np.testing.assert_allclose(a.x, b.x, rtol=1e-15, atol=1e-16)
            np.testing.assert_allclose(a.abar, b.abar, rtol=1e-15, atol=1e-17)
            np.testing.assert_allclose(a.alpha, b.alpha, rtol=1e-15, atol=0)


def test_memory_takes_the_new_derivative():
    p = tiny_sparse(seed=16)
    st = consistent_state(p, seed=17)
    i = 5
    z = sum(p.values[k] * st.x[p.col_idx[k]] for k in range(p.row_ptr[i], p.row_ptr[i + 1]))
    s = one_step(p, st, i, 0.1)
    assert s.alpha[i] == pytest.approx(-p.labels[i] / (1.0 + math.exp(p.labels[i] * z)), rel=1e-15)
    assert np.array_equal(np.delete(s.alpha, i), np.delete(st.alpha, i))
    # coordinates outside S_i are untouched
    outside = np.setdiff1d(np.arange(p.d), p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]])
    np.testing.assert_array_equal(s.x[outside], st.x[outside])
    np.testing.assert_array_equal(s.abar[outside], st.abar[outside])


def test_variance_identity():
    """E||alpha_i - D_i abar - f'_i(x*)||^2 = E||alpha_i - f'_i(x*)||^2 - abar^T D abar
    (App. B, Eq. alphaiBarVariance), with vector memories alpha_i a_i and
    f'_i(x) = phi'_i a_i + lambda D_i x (the Sec. 4.2 split of the l2 term, whose
    mean over i is grad f)."""
    p = tiny_sparse(n=10, d=7, k=3, seed=18)
    xs = R.newton(p)
    D = R.reweighting(p)
    st = consistent_state(p, seed=19)
    A = R.csr(p).toarray()
    mask = (A != 0).astype(float)
    zs = A @ xs
    lhs = rhs = 0.0
    for i in range(p.n):
        mem = st.alpha[i] * A[i]
        fstar_i = R.phi_prime(p.loss, zs[i:i + 1], p.labels[i:i + 1])[0] * A[i] + p.lam * mask[i] * D * xs
        lhs += np.sum((mem - mask[i] * D * st.abar - fstar_i) ** 2) / p.n
        rhs += np.sum((mem - fstar_i) ** 2) / p.n
    rhs -= np.dot(st.abar, D * st.abar)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_abar_stays_the_average_of_the_memory():
    p = synth.small_logistic()
    st = R.State.zeros(p)
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    D = R.reweighting(p)
    for ep in range(3):
        R.sparse_saga(p, st, synth.sample_indices(p.n, p.n, 4, ep), gamma, D)
        ref = R.abar_from_scratch(p, st.alpha)
        assert np.max(np.abs(st.abar - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_sparse_saga_reaches_the_newton_optimum():
    p = synth.small_logistic()
    xs = R.newton(p)
    res = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 4, ep), rel_tol=1e-12, max_epochs=200)
    assert abs(res["fstar"] - R.objective(p, xs)) <= 1e-12 * abs(R.objective(p, xs))
    assert np.linalg.norm(res["x"] - xs) <= 1e-5 * np.linalg.norm(xs)


def test_sparse_saga_reaches_the_ridge_closed_form():
    p = tiny_dense(n=200, d=5, lam=0.01, seed=20)
    xs = R.ridge_closed_form(p)
    st = R.State.zeros(p)
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    for ep in range(300):
        R.sparse_saga(p, st, synth.sample_indices(p.n, p.n, 5, ep), gamma)
    np.testing.assert_allclose(st.x, xs, rtol=1e-9, atol=1e-11)


def test_theorem1_rate_bound_holds():
    """Theorem 1: with gamma = a/(5L), E|x_t - x*|^2 <= (1-rho)^t C0,
    rho = min(1/n, a/kappa)/5, C0 = |x0-x*|^2 + sum_i |alpha0_i - f'_i(x*)|^2/(5L^2).
    Checked on the average over seeds (a weak, one-sided pin)."""
    p = tiny_sparse(n=30, d=8, k=3, seed=21, lam=0.05)
    xs = R.newton(p)
    L = R.lipschitz(p)
    kappa = L / p.lam
    a = 1.0
    gamma, rho = a / (5 * L), min(1.0 / p.n, a / kappa) / 5.0
    A = R.csr(p).toarray()
    mask = (A != 0).astype(float)
    D = R.reweighting(p)
    zs = A @ xs
    fi = [R.phi_prime(p.loss, zs[i:i + 1], p.labels[i:i + 1])[0] * A[i] + p.lam * mask[i] * D * xs
          for i in range(p.n)]
    C0 = np.dot(xs, xs) + sum(np.dot(f, f) for f in fi) / (5 * L * L)
    T = 40 * p.n
    errs = []
    for s in range(8):
        st = R.State.zeros(p)
        R.sparse_saga(p, st, synth.sample_indices(p.n, T, 100 + s), gamma, D)
        errs.append(np.sum((st.x - xs) ** 2))
    assert np.mean(errs) <= (1 - rho) ** T * C0


def test_lipschitz_is_the_largest_curvature_of_a_sample():
    """For logistic phi'' peaks at z = 0 with value 1/4, so the largest Hessian
    eigenvalue of a one-sample problem at x = 0 is |a|^2/4 + lambda = L."""
    a = np.array([0.5, -1.5, 2.0])
    p = synth.Problem("one", 1, 3, np.array([0, 3], dtype=np.int64), np.arange(3, dtype=np.int32), a,
                      np.array([-1.0]), "logistic", lam=0.07, storage="f64")
    assert np.linalg.eigvalsh(R.hessian(p, np.zeros(3))).max() == pytest.approx(R.lipschitz(p), rel=1e-14)
    q = tiny_dense(n=5, d=3, loss="squared", lam=0.07)
    worst = max(np.linalg.eigvalsh(np.outer(r, r)).max() for r in q.dense_values()) + q.lam
    assert R.lipschitz(q) == pytest.approx(worst, rel=1e-13)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_row_derivatives_match_finite_differences(loss):
    p = tiny_sparse(loss=loss, seed=22)
    x = np.random.default_rng(23).standard_normal(p.d)
    z = R.margins(p, x)
    h = 1e-6
    fd = (R.phi(loss, z + h, p.labels) - R.phi(loss, z - h, p.labels)) / (2 * h)
    np.testing.assert_allclose(R.row_derivatives(p, x), fd, rtol=1e-8, atol=1e-10)


def test_sparsity_delta_brute_force():
    p = tiny_sparse(n=9, d=5, k=2, seed=24)
    best = max(sum(1 for i in range(p.n) if v in set(p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]]))
               for v in range(p.d))
    assert R.sparsity_delta(p) == best / p.n


def test_lipschitz_bounds_every_sampled_component():
    """L bounds the largest Hessian eigenvalue of every sampled component
    phi_i(a_i.x) + lambda/2 sum_{v in S_i} D_v x_v^2 (logistic curvature peaks
    at z = 0 with 1/4) and is attained on a row whose heaviest term dominates:
    here a row made of one column that no other row touches."""
    p = tiny_sparse(n=12, d=9, k=3, seed=25, lam=0.3)
    D = R.reweighting(p)
    L = R.lipschitz(p)
    A = R.csr(p).toarray()
    worst = 0.0
    for i in range(p.n):
        mask = A[i] != 0
        H = 0.25 * np.outer(A[i], A[i]) + p.lam * np.diag(D * mask)
        worst = max(worst, np.linalg.eigvalsh(H).max())
    assert worst <= L * (1 + 1e-12)
    # a row of a single, otherwise unused column: eigenvalue = c a^2 + lambda n, exactly L
    q = synth.Problem("rare", 3, 2, np.array([0, 1, 2, 3], dtype=np.int64), np.array([0, 0, 1], dtype=np.int32),
                      np.array([0.5, 0.5, 0.1]), np.array([1.0, -1.0, 1.0]), "logistic", lam=0.5, storage="f64")
    assert R.lipschitz(q) == pytest.approx(0.25 * 0.01 + 0.5 * 3, rel=1e-14)


def test_serial_sparse_saga_is_stable_with_heavy_reweighting():
    """With lambda n large and rare columns, gamma = 1/(3L) must account for
    lambda D_v: the run converges to the Newton optimum."""
    p = tiny_sparse(n=40, d=30, k=2, seed=26, lam=0.05)
    assert p.lam * R.reweighting(p).max() > 0.25
    xs = R.newton(p)
    res = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 9, ep), rel_tol=1e-12, max_epochs=3000)
    assert abs(res["fstar"] - R.objective(p, xs)) <= 1e-11 * abs(R.objective(p, xs))


# ------------------------------------------------------------ lagged updates (App. F)

@pytest.mark.parametrize("lam", [0.05, 0.0])
def test_lagged_saga_equals_dense_saga(lam):
    """The lagged scheme defers the steps x_v <- (1 - gamma lambda) x_v - gamma abar_v
    of coordinates outside the sampled support; after the final catch-up it is
    the dense SAGA iterate (Eq. SAGAupdate), step for step."""
    p = tiny_sparse(n=30, d=12, k=3, seed=40, lam=lam)
    st0 = consistent_state(p, seed=41)
    idx = np.random.default_rng(42).integers(0, p.n, 90)
    dense = st0.copy()
    for i in idx:
        R.dense_saga_step(p, dense, int(i), 0.15)
    lag = R.lagged_saga(p, st0.copy(), idx, 0.15)
    np.testing.assert_allclose(lag.x, dense.x, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(lag.abar, dense.abar, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(lag.alpha, dense.alpha, rtol=1e-12, atol=0)


def test_lagged_pin_catches_a_missing_catch_up():
    """A lagged step that forgot the deferred regulariser steps differs from
    dense SAGA (the pin above can fail)."""
    p = tiny_sparse(n=30, d=12, k=3, seed=40, lam=0.05)
    st0 = consistent_state(p, seed=41)
    idx = np.random.default_rng(42).integers(0, p.n, 90)
    dense = st0.copy()
    for i in idx:
        R.dense_saga_step(p, dense, int(i), 0.15)
    sparse_only = R.sparse_saga(p, st0.copy(), idx, 0.15, D=np.ones(p.d))
    assert np.max(np.abs(sparse_only.x - dense.x)) > 1e-3


def test_lagged_and_sparse_saga_converge_alike():
    """App. F.1: on sparse data Sparse SAGA and lagged-update SAGA need about
    the same number of passes over the data."""
    p = synth.sparse_logistic(3000, 600, k_mean=8, k_min=2, k_max=30, zipf_s=1.1, values="abs_normal",
                              storage="f64", seed=5, name="appC")
    fs = R.objective(p, R.newton(p))
    f0 = R.objective(p, np.zeros(p.d))
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    sub = {}
    for name, run in (("sparse", R.sparse_saga), ("lagged", R.lagged_saga)):
        st = R.State.zeros(p)
        curve = []
        for ep in range(30):
            run(p, st, synth.sample_indices(p.n, p.n, 7, ep), gamma)
            curve.append((R.objective(p, st.x) - fs) / (f0 - fs))
        sub[name] = np.array(curve)
    assert sub["sparse"][-1] < 1e-7 and sub["lagged"][-1] < 1e-7
    ratio = sub["sparse"][[9, 19, 29]] / sub["lagged"][[9, 19, 29]]
    assert np.all((ratio > 0.1) & (ratio < 10)), ratio


# ------------------------------------------------------------ row sampling

def test_splitmix64_matches_its_published_outputs():
    """The first outputs of the reference SplitMix64 for seed 1234567."""
    assert R.splitmix64(1234567, 5) == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                        4593380528125082431, 16408922859458223821]


def test_sampler_takes_the_generator_outputs_in_order():
    seed, n = 99, 1000
    u = R.splitmix64(seed, 40)
    rows = R.sampler_indices(seed, n, 0, 40)
    assert rows.tolist() == [(v * n) >> 64 for v in u]
    # a later window of the same stream
    np.testing.assert_array_equal(R.sampler_indices(seed, n, 25, 15), rows[25:])


def test_sampler_is_uniform_over_rows():
    n, count = 50, 50000
    rows = R.sampler_indices(7, n, 0, count)
    assert rows.min() >= 0 and rows.max() < n
    c = np.bincount(rows, minlength=n)
    chi2 = np.sum((c - count / n) ** 2 / (count / n))
    # chi-square with 49 degrees of freedom: P(chi2 > 90) < 1e-3
    assert chi2 < 90, chi2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 1000, 4097])
def test_permutation_sampling_visits_every_row_once_per_epoch(n):
    rows = R.permutation_indices(12, n, 0, 3 * n)
    for e in range(3):
        assert sorted(rows[e * n:(e + 1) * n].tolist()) == list(range(n))
    if n >= 16:  # the epochs differ from each other and from the identity
        assert not np.array_equal(rows[:n], rows[n:2 * n])
        assert not np.array_equal(rows[:n], np.arange(n))
    # a window that starts mid-epoch is the same stream
    np.testing.assert_array_equal(R.permutation_indices(12, n, n // 2 + 1, n), rows[n // 2 + 1:n // 2 + 1 + n])


def test_permutation_positions_are_spread_over_rows():
    """Over many epochs, the row at a fixed position is close to uniform."""
    n, epochs = 20, 4000
    first = np.array([R.permutation_indices(5, n, e * n, 1)[0] for e in range(epochs)])
    c = np.bincount(first, minlength=n)
    chi2 = np.sum((c - epochs / n) ** 2 / (epochs / n))
    assert chi2 < 50, chi2  # 19 degrees of freedom: P(chi2 > 50) < 1e-3


# ------------------------------------------------------------ multi-threaded CPU ASAGA (timing baseline)

def test_cpu_asaga_on_one_thread_is_serial_sparse_saga():
    from oracle import cpu_asaga
    p = synth.small_logistic()
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    run = cpu_asaga.Runner(p, threads=1)
    st = run.run(R.State.zeros(p), 2 * p.n, gamma, seed=17)
    ref = R.sparse_saga(p, R.State.zeros(p), R.sampler_indices(17, p.n, 0, 2 * p.n), gamma)
    # alpha_i += delta instead of alpha_i = phi'_i: equal up to one rounding per visit
    np.testing.assert_allclose(st.x, ref.x, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(st.abar, ref.abar, rtol=1e-10, atol=1e-14)


def test_cpu_asaga_with_threads_reaches_the_optimum():
    from oracle import cpu_asaga
    p = synth.small_logistic()
    fs = R.objective(p, R.newton(p))
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    run = cpu_asaga.Runner(p, threads=4)
    st = R.State.zeros(p)
    for _ in range(60):
        run.run(st, p.n, gamma, seed=3)
    assert (R.objective(p, st.x) - fs) / abs(fs) < 1e-8
    assert np.max(np.abs(st.abar - R.abar_from_scratch(p, st.alpha))) < 1e-10


# ------------------------------------------------------------ mixed precision: drift of the optimum

@pytest.mark.parametrize("values,storage", [("binary", "bf16"), ("abs_normal", "bf16"), ("abs_normal", "f16")])
def test_quantisation_moves_the_optimum_by_a_reported_amount(values, storage):
    """The solver's f* is the optimum of the stored (quantised) matrix; the
    float64 matrix's optimum differs.  This reports the relative gap (it is
    not a tolerance of the solver: the 1e-6 target is measured against the
    quantised problem's own f*) and bounds it loosely."""
    p = synth.sparse_logistic(3000, 800, k_mean=20, k_min=2, k_max=60, zipf_s=1.1, storage="f64", seed=9,
                              values=values)
    q = synth.Problem(**{**p.__dict__})
    q.values = synth.to_storage_grid(p.values, storage)
    q.storage = storage
    f64 = R.objective(p, R.newton(p))
    fq = R.objective(q, R.newton(q))
    drift = abs(fq - f64) / abs(f64)
    print(f"{values} {storage}: f*(float64 A) = {f64:.12f}, f*(stored A) = {fq:.12f}, relative gap {drift:.2e}")
    assert 0 < drift < 1e-3


# ---------------------------------------------------------------- overlap estimator (App. E.2)

def _trace(intervals):
    return np.array([v for iv in intervals for v in iv], dtype=np.uint64)


def test_overlap_of_identical_and_of_disjoint_intervals():
    """p updates processed at the same time overlap p - 1 others each; updates
    one after the other overlap none."""
    est = R.overlap_estimates(_trace([(5, 9)] * 150))
    assert est["tau_mean"] == 149 and est["tau_max"] == 149 and est["tau_paper"] == 149
    est = R.overlap_estimates(_trace([(10 * k, 10 * k + 9) for k in range(250)]))
    assert est["tau_mean"] == 0 and est["tau_max"] == 0 and est["tau_paper"] == 0
    assert est["window_ns_mean"] == 9


def test_overlap_of_a_staircase_has_its_closed_form():
    """Update k runs over [k, k + w] (closed): it overlaps the updates r with
    |k - r| <= w, i.e. min(k, w) + min(N - 1 - k, w) others."""
    N, w = 1000, 37
    est = R.overlap_estimates(_trace([(k, k + w) for k in range(N)]))
    want = np.array([min(k, w) + min(N - 1 - k, w) for k in range(N)])
    assert np.array_equal(est["overlaps"], want)
    assert est["tau_mean"] == want.sum() / N and est["tau_max"] == 2 * w
    # windows of 100 in start order: the interior windows see 2w each
    assert est["tau_paper"] == 2 * w


def test_overlap_windows_follow_start_order_and_drop_a_partial_window():
    """Window averages are taken over consecutive updates in start order, not
    in update order; the last, partial window is left out."""
    busy = [(0, 100)] * 100                      # 100 updates at once: 99 each
    idle = [(200 + 10 * k, 205 + 10 * k) for k in range(100)]  # one after another: 0 each
    tail = [(10_000, 10_001)] * 50               # a partial window of 49s
    est = R.overlap_estimates(_trace(idle + tail + busy))  # listed out of start order
    assert est["tau_paper"] == 99.0
    est = R.overlap_estimates(_trace(idle + tail))
    assert est["tau_paper"] == 0.0 and est["tau_max"] == 49
