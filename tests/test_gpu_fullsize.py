"""Parity at the full workload sizes, in the launch configuration that
bench.py times (the autotuned warps and step), through the C ABI.

At these sizes the oracle cannot follow an asynchronous run update by
update, so the tests check what it can compute at any size:
  * set-up constants (L, gamma0, Delta, longest row) against the oracle;
  * one epoch replayed in order by a single warp against the serial float64
    oracle on the same rows: relative l2 <= 1e-4 and per element
    max_v |x_v - x*_v| <= 1e-3 max_v |x*_v| (as for the small cases);
  * after asynchronous epochs at the tuned schedule: the float64 objective
    and gradient at the GPU iterate against the oracle's (1e-12 / 1e-11),
    and abar recomputed from the memory against the oracle's sum rounded to
    float32 (within one float32 ulp: the float64 column sums add atomics in
    no fixed order);
  * 1e-6 relative suboptimality against the f* stored in tests/golden (the
    oracle's certified value for the same generated problem).
"""
import json
import os

import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS = {  # generator, storage on the device, stored f*
    "rcv1like": (synth.rcv1_like, "f32", "fstar_rcv1like.json"),
    "urllike": (synth.url_like, "bf16", "fstar_urllike.json"),
    "covtypelike": (synth.covtype_like, "f16", "fstar_covtypelike.json"),
}


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


def golden(name, p):
    g = json.load(open(os.path.join(HERE, "golden", name)))
    fp, want = p.fingerprint(), g["fingerprint"]
    assert fp["structure_sha256"] == want["structure_sha256"], "regenerated problem differs from the stored one"
    assert fp["sum_values"] == pytest.approx(want["sum_values"], rel=1e-9)
    return g


@pytest.fixture(scope="module", params=list(WORKLOADS))
def workload(request):
    make, storage, gold = WORKLOADS[request.param]
    p = make()
    return request.param, p, storage, golden(gold, p)


def test_setup_constants_at_full_size(workload):
    _, p, storage, _ = workload
    with asaga.Context(p, storage=storage) as c:
        info = asaga.asaga_get_info(c.ctx)
    assert info["L"] == pytest.approx(R.lipschitz(p), rel=1e-7)
    assert info["delta"] == pytest.approx(R.sparsity_delta(p), rel=1e-15)
    assert info["max_row_len"] == p.row_lengths().max()


def test_one_epoch_in_order_matches_the_oracle_at_full_size(workload):
    _, p, storage, _ = workload
    idx = synth.sample_indices(p.n, p.n, seed=41)
    with asaga.Context(p, storage=storage) as c:
        asaga.asaga_run_indices(c.ctx, idx)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        gamma = asaga.asaga_get_info(c.ctx)["gamma"]
    st = R.sparse_saga(p, R.State.zeros(p), idx, gamma)
    for name, a, b in (("x", x, st.x), ("alpha", alpha, st.alpha), ("abar", abar, st.abar)):
        assert rel(a, b) <= 1e-4, (name, rel(a, b))
        # per element, against the largest coordinate (the tolerance of test_gpu_parity)
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b)), name


def test_tuned_schedule_evaluations_and_target_at_full_size(workload):
    name, p, storage, g = workload
    with asaga.Context(p, storage=storage, seed=5, abar_recompute_every=5) as c:
        tune = asaga.asaga_autotune(c.ctx)
        assert tune["score"] > 0, tune
        # float64 evaluations at an asynchronous iterate of the tuned launch configuration
        asaga.asaga_run(c.ctx, 3)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        f = asaga.asaga_objective(c.ctx)
        gr, n2 = asaga.asaga_full_grad(c.ctx)
        asaga.asaga_recompute_abar(c.ctx)
        abar_new = asaga.asaga_get_state(c.ctx)[1]
        x64 = x.astype(np.float64)
        assert f == pytest.approx(R.objective(p, x64), rel=1e-12)
        g_ref = R.gradient(p, x64)
        assert rel(gr, g_ref) <= 1e-11
        # the float64 column sums add atomics in no fixed order; at millions of
        # columns a few of them round to the neighbouring float32
        np.testing.assert_array_max_ulp(abar_new, R.abar_from_scratch(p, alpha.astype(np.float64)).astype(np.float32),
                                        maxulp=1)
        # the tuned schedule reaches the target from x = 0
        asaga.asaga_set_state(c.ctx, np.zeros(p.d, np.float32), np.zeros(p.d, np.float32),
                              np.zeros(p.n, np.float32), 0)
        s, r = asaga.asaga_run(c.ctx, 300, 1e-6, g["fstar"])
        x = asaga.asaga_get_state(c.ctx)[0]
    assert s == asaga.OK, (name, asaga.STATUS_NAMES[s], r.as_dict(), tune)
    f_ref = R.objective(p, x.astype(np.float64))
    assert (f_ref - g["fstar"]) / abs(g["fstar"]) <= 1e-6 + g["bound"] / abs(g["fstar"])
