"""Malformed problems on a GPU: rejected with EINVAL, and the GPU stays usable.

asaga_create checks the problem's content on host threads while the device
copies it and runs the set-up kernels (column counts, smoothness).  Those
kernels skip columns outside [0, d) and row ranges outside [0, nnz], so a
problem that the check then rejects cannot make them read or write out of
bounds.  Each case below plants one defect in an otherwise valid problem of
a few thousand rows (enough for the set-up kernels to run over it), expects
the check's message, and then solves a valid problem on the same device.
"""
import ctypes

import numpy as np
import pytest

from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


def arrays():
    p = synth.rcv1_like(seed=5, n=4000, d=800)
    return (np.ascontiguousarray(p.row_ptr, dtype=np.int64).copy(), np.ascontiguousarray(p.col_idx, dtype=np.int32).copy(),
            np.ascontiguousarray(p.values, dtype=np.float32).copy(), np.ascontiguousarray(p.labels, dtype=np.float64).copy(),
            p)


def create(rp, ci, v, y, p):
    prob = asaga.Problem(p.n, p.d, rp, ci, v, "f32", y, nnz=len(ci))
    o = asaga.asaga_default_options(loss=p.loss, lam=p.lam, storage_dtype="f32")
    ctx = ctypes.c_void_p()
    s = asaga.load().asaga_create(ctypes.byref(ctx), ctypes.byref(prob.struct), ctypes.byref(o))
    if ctx.value:
        asaga.asaga_destroy(ctx.value)
    return s, asaga.asaga_last_error(None)


def plant(kind, rp, ci, v, y):
    mid = len(rp) // 2
    a, b = rp[mid], rp[mid + 1]
    if kind == "column past d":
        ci[a] = 1 << 30
    elif kind == "negative column":
        ci[a] = -7
    elif kind == "repeated column":
        ci[a + 1] = ci[a]
    elif kind == "row_ptr decreases":
        rp[mid] = rp[mid - 1] - 1  # row mid - 1 ends before it starts
    elif kind == "row_ptr past nnz":
        rp[mid] = len(ci) + 1000
    elif kind == "nan value":
        v[b - 1] = np.nan
    elif kind == "label":
        y[mid] = 0.5


CASES = {"column past d": "out of range", "negative column": "out of range", "repeated column": "repeated column",
         "row_ptr decreases": "row_ptr", "row_ptr past nnz": "row_ptr", "nan value": "non-finite value",
         "label": "not +-1"}


@pytest.mark.parametrize("kind", list(CASES))
def test_a_malformed_problem_is_rejected_and_the_gpu_stays_usable(kind):
    rp, ci, v, y, p = arrays()
    assert rp[len(rp) // 2 + 1] - rp[len(rp) // 2] >= 2  # the planted row has two entries to work with
    plant(kind, rp, ci, v, y)
    s, err = create(rp, ci, v, y, p)
    assert s == asaga.EINVAL and CASES[kind] in err, (s, err)
    # the device is fine: a valid problem solves
    p = arrays()[4]
    with asaga.Context(p, storage="f32", seed=1, max_warps=64) as c:
        s, r = asaga.asaga_run(c.ctx, 2)
        assert s == asaga.OK and np.isfinite(r.f_last)
