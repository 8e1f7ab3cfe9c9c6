"""The device row sampler against the checker's independent restatement of
it, and single-warp runs that draw their own rows against the serial
float64 Sparse SAGA on the same rows (through the C ABI).

Integer work is compared bit for bit; iterates after one in-order epoch in
float32 within the replay tolerance of 1e-4 relative l2 (as in
test_gpu_parity)."""
import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

DET_TOL = 1e-4


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


@pytest.mark.parametrize("n,t_begin", [(1, 0), (7, 0), (1000, 12345), (700000, 0), (2_400_000, 2**40 + 3),
                                       (2**40 + 17, 99)])
def test_uniform_sampler_is_the_splitmix64_stream(n, t_begin):
    dev = asaga.asaga_sample_rows(2024, n, t_begin, 3000, "uniform")
    np.testing.assert_array_equal(dev, R.sampler_indices(2024, n, t_begin, 3000))


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 4097, 65536, 700000])
def test_permutation_sampler_matches_its_specification(n):
    count = min(3 * n, 6000)
    t0 = 0 if n > 2000 else 5
    dev = asaga.asaga_sample_rows(77, n, t0, count, "permutation")
    np.testing.assert_array_equal(dev, R.permutation_indices(77, n, t0, count))


@pytest.mark.parametrize("n", [1000, 65537, 700000])
def test_permutation_sampler_visits_every_row_once_per_epoch(n):
    dev = asaga.asaga_sample_rows(5, n, 0, 2 * n, "permutation")
    for e in range(2):
        c = np.bincount(dev[e * n:(e + 1) * n], minlength=n)
        assert c.min() == 1 and c.max() == 1


def run_pair(p, sampling, seed, epochs=1, draw_ahead=0):
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    with asaga.Context(p, storage="f32", deterministic=1, seed=seed, gamma=gamma, sampling=sampling) as c:
        asaga.asaga_set_draw_ahead(c.ctx, draw_ahead)
        assert asaga.asaga_get_info(c.ctx)["draw_ahead"] == draw_ahead
        asaga.asaga_run(c.ctx, epochs)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
    rows = (R.sampler_indices if sampling == "uniform" else R.permutation_indices)(seed, p.n, 0, epochs * p.n)
    st = R.sparse_saga(p, R.State.zeros(p), rows, gamma)
    return (x, abar, alpha), st


@pytest.mark.parametrize("draw_ahead", [0, 1])
@pytest.mark.parametrize("sampling", ["uniform", "permutation"])
def test_single_warp_run_with_its_own_sampler_matches_the_checker(sampling, draw_ahead):
    """Either draw placement (before an update's reads, or while its gathers
    are in flight) visits the sampler's rows in its order."""
    p = synth.small_logistic()
    p.values = synth.to_storage_grid(p.values, "f32")
    (x, abar, alpha), st = run_pair(p, sampling, seed=31, draw_ahead=draw_ahead)
    assert rel(x, st.x) <= DET_TOL, rel(x, st.x)
    assert rel(alpha, st.alpha) <= DET_TOL
    assert rel(abar, st.abar) <= DET_TOL


def test_single_warp_run_continues_the_stream_across_calls():
    p = synth.small_logistic()
    p.values = synth.to_storage_grid(p.values, "f32")
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    with asaga.Context(p, storage="f32", deterministic=1, seed=8, gamma=gamma, sampling="permutation") as c:
        asaga.asaga_run(c.ctx, 0.5)
        asaga.asaga_run(c.ctx, 1.5)
        x = asaga.asaga_get_state(c.ctx)[0]
    st = R.sparse_saga(p, R.State.zeros(p), R.permutation_indices(8, p.n, 0, 2 * p.n), gamma)
    assert rel(x, st.x) <= DET_TOL


def test_async_permutation_sampling_reaches_1e6():
    p = synth.small_logistic()
    fstar = R.objective(p, R.newton(p))
    with asaga.Context(p, seed=3, sampling="permutation", abar_recompute_every=5) as c:
        asaga.asaga_autotune(c.ctx)
        s, r = asaga.asaga_run(c.ctx, 300, 1e-6, fstar)
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict())


def test_draw_ahead_argument_is_checked():
    p = synth.small_logistic()
    with asaga.Context(p) as c:
        with pytest.raises(asaga.AsagaError) as e:
            asaga.asaga_set_draw_ahead(c.ctx, 2)
        assert e.value.status == asaga.EINVAL
        assert asaga.asaga_get_info(c.ctx)["draw_ahead"] == 0


def test_async_run_with_the_row_drawn_ahead_reaches_1e6():
    p = synth.rcv1_like(seed=24, n=50000, d=5000)
    cert = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, 31, ep), rel_tol=1e-10)
    with asaga.Context(p, seed=5, max_warps=64, abar_recompute_every=5) as c:
        asaga.asaga_set_draw_ahead(c.ctx, 1)
        s, r = asaga.asaga_run(c.ctx, 150, 1e-6, cert["fstar"])
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict())
