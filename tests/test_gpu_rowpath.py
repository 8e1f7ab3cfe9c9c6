"""The multi-warp row path, and one read of the state per entry of a row.

Algorithm 2 reads x^ on S_i once per update; Sec. 4.2's projected l2 term
uses that same x^_v.  The update kernel gathers every entry's {x^_v, abar_v,
D_v} once: entries in the register slots keep the scatter term there, the
entries past them (rows longer than 256 entries per warp of the core) keep
it in a per-core scratch array.  Rows can also be spread over G warps of one
block (the multi-warp row path); then the warps' partial dot products meet in
shared memory and every warp scatters its own entries with the same delta.

Checked here through the C ABI, against the float64 CPU checker:
  * a replay in order on ONE core of G = 2, 4, 8 warps (rows of 300..1224
    entries cross the staged part, the register slots and the scratch part
    for every G) equals the serial float64 Sparse SAGA on the same rows,
    rel-l2 <= 1e-4 and per element (tolerance below);
  * dense rows on multi-warp cores, the same way;
  * asynchronous runs on rows of 300..1224 entries under concurrent cores,
    on single-warp cores, on multi-warp cores for every row and with the
    rows split by a threshold between both paths, reach 1e-6 relative
    suboptimality against the Newton optimum (float64);
  * a batch whose instances take different row paths reaches each
    instance's optimum.

Per-element tolerance of a replay: max_v |x_v - x*_v| <= 1e-3 max_v |x*_v|.
The relative l2 error bounds the average error; float32 rounding of each
coordinate's sum of updates is about eps32 = 6e-8 times the magnitude of the
updates it receives, and the propagated error of the dot products (through
delta) reaches every coordinate of a row in proportion to its value a_iv, so
no coordinate's error exceeds ~1e-4 of the largest coordinate.  A factor ten
over the rel-l2 tolerance leaves room for rounding and still fails a
coordinate that is wrong by a sizeable part of its own value, unless that
coordinate is below 1e-3 of the largest one.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

DET_TOL = 1e-4
ELEM_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def elem(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)


def long_rows(n=3000, d=6000, seed=40, **kw):
    """Rows of 300..1224 entries (the top of the RCV1 support range, App. E.2,
    Table 2), Zipf(1.1) columns."""
    args = dict(k_mean=450, k_min=300, k_max=1224, k_sigma=0.5, zipf_s=1.1, values="abs_normal", storage="f32",
                seed=seed)
    args.update(kw)
    return synth.sparse_logistic(n, d, **args)


def replay(p, idx, threshold, group, storage="f32", draw_ahead=0):
    with asaga.Context(p, storage=storage) as c:
        asaga.asaga_set_row_path(c.ctx, threshold, group)
        asaga.asaga_set_draw_ahead(c.ctx, draw_ahead)
        info = asaga.asaga_get_info(c.ctx)
        assert (info["row_threshold"], info["row_group"]) == ((threshold, group) if group > 1 else (-1, 1))
        asaga.asaga_run_indices(c.ctx, idx)
        x, abar, alpha = asaga.asaga_get_state(c.ctx)
        gamma = info["gamma"]
    st = R.sparse_saga(p, R.State.zeros(p), idx, gamma)
    return (x, abar, alpha), st


def assert_close(got, st):
    x, abar, alpha = got
    for a, b in ((x, st.x), (abar, st.abar), (alpha, st.alpha)):
        assert rel(a, b) <= DET_TOL, rel(a, b)
        assert elem(a, b) <= ELEM_TOL, elem(a, b)


@pytest.mark.parametrize("group", [1, 2, 4, 8])
def test_replay_long_rows_on_one_core_of_group_warps(group):
    p = long_rows()
    lens = p.row_lengths()
    assert lens.min() >= 300 and lens.max() > 1024  # past the register slots of G = 1, 2, 4
    idx = synth.sample_indices(p.n, p.n, seed=41)
    got, st = replay(p, idx, 0 if group > 1 else -1, group)
    assert_close(got, st)


@pytest.mark.parametrize("group", [1, 2, 8])
def test_replay_with_the_row_drawn_ahead(group):
    """The next row drawn while the gathers are in flight: the same rows in
    the same order, on single- and multi-warp cores."""
    p = long_rows(n=2000, seed=49)
    idx = synth.sample_indices(p.n, p.n, seed=42)
    got, st = replay(p, idx, 0 if group > 1 else -1, group, draw_ahead=1)
    assert_close(got, st)


@pytest.mark.parametrize("group", [2, 4])
def test_replay_dense_rows_on_multi_warp_cores(group):
    """Dense rows of 300 entries: 128 G in registers, the rest past the slots."""
    p = synth.dense_ridge(1500, 300, storage="f16", lam=1e-2, seed=43)
    idx = synth.sample_indices(p.n, p.n, seed=44)
    got, st = replay(p, idx, 0, group, storage="f16")
    assert_close(got, st)


def test_replay_bf16_compact_rows_on_a_multi_warp_core():
    """Binary rows scaled to unit norm stored as one value per row and uint16
    columns: the staged column copy and the row value on a 4-warp core."""
    p = long_rows(n=2000, d=5000, seed=45, values="binary", storage="bf16")
    idx = synth.sample_indices(p.n, p.n, seed=46)
    with asaga.Context(p, storage="bf16", compact=1) as c:
        info = asaga.asaga_get_info(c.ctx)
        assert info["col_index_bytes"] == 2 and info["row_values"] == 1
        asaga.asaga_set_row_path(c.ctx, 0, 4)
        asaga.asaga_run_indices(c.ctx, idx)
        got = asaga.asaga_get_state(c.ctx)
    st = R.sparse_saga(p, R.State.zeros(p), idx, info["gamma"])
    assert_close(got, st)


def test_row_path_arguments_are_checked():
    p = long_rows(n=500, d=2000, seed=47)
    with asaga.Context(p) as c:
        for bad in ((0, 3), (0, 16), (-2, 2)):
            with pytest.raises(asaga.AsagaError) as e:
                asaga.asaga_set_row_path(c.ctx, *bad)
            assert e.value.status == asaga.EINVAL
        asaga.asaga_set_row_path(c.ctx, -1, 4)  # no long rows: the group does not apply
        info = asaga.asaga_get_info(c.ctx)
        assert (info["row_threshold"], info["row_group"]) == (-1, 1)
    with asaga.Context(p, deterministic=1) as c:
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_set_row_path(c.ctx, 400, 4)  # two paths cannot run strictly in order
        asaga.asaga_set_row_path(c.ctx, 0, 4)


@pytest.fixture(scope="module")
def long_problem():
    p = long_rows(n=12000, d=3000, seed=48)
    xs = R.newton(p)
    assert np.linalg.norm(R.gradient(p, xs)) <= 1e-12
    return p, R.objective(p, xs)


@pytest.mark.parametrize("path", [(-1, 1, 0), (0, 2, 0), (0, 4, 0), (0, 8, 0), (450, 4, 0), (-1, 1, 1), (450, 4, 1)])
def test_async_long_rows_reach_1e6(long_problem, path):
    """Concurrent cores on rows of 300..1224 entries: every entry's x^ read once
    per update, its lambda term from that read, on either row path and either
    draw placement.  The path regroups the tuned warps into cores (same warps,
    same step)."""
    p, fstar = long_problem
    with asaga.Context(p, seed=6, abar_recompute_every=5) as c:
        tune = asaga.asaga_autotune(c.ctx)
        if path[2] and not tune["draw_ahead"]:  # a longer window: half the step keeps these warps inside the frontier
            wpb = asaga.asaga_get_info(c.ctx)["warps_per_block"]
            asaga.asaga_set_schedule(c.ctx, tune["warps"], tune["gamma"] / 2, wpb)
        asaga.asaga_set_row_path(c.ctx, path[0], path[1])
        asaga.asaga_set_draw_ahead(c.ctx, path[2])
        s, r = asaga.asaga_run(c.ctx, 400, 1e-6, fstar)
        info = asaga.asaga_get_info(c.ctx)
        x = asaga.asaga_get_state(c.ctx)[0]
    assert s == asaga.OK, (asaga.STATUS_NAMES[s], r.as_dict(), info, tune)
    assert info["warps"] == tune["warps"] > 1
    assert R.objective(p, x.astype(np.float64)) - fstar <= 1e-6 * abs(fstar)


def test_autotune_reports_the_row_path_it_keeps(long_problem):
    p, _ = long_problem
    with asaga.Context(p, seed=7) as c:
        tune = asaga.asaga_autotune(c.ctx)
        info = asaga.asaga_get_info(c.ctx)
    assert (tune["row_threshold"], tune["row_group"]) == (info["row_threshold"], info["row_group"])
    assert tune["draw_ahead"] == info["draw_ahead"] in (0, 1)
    assert tune["row_group"] in (1, 2, 4, 8)
    assert (tune["row_group"] == 1) == (tune["row_threshold"] == -1)


def test_batch_with_per_instance_row_paths_reaches_each_optimum():
    ps = [long_rows(n=4000, d=2500, seed=50 + k, lam=lam) for k, lam in enumerate((1e-3, 3e-3, 1e-2))]
    ps.append(synth.sparse_logistic(5000, 2000, k_mean=20, k_min=1, k_max=60, zipf_s=1.1, storage="f32", seed=53,
                                    lam=1e-3))
    fs = []
    for p in ps:
        xs = R.newton(p)
        fs.append(R.objective(p, xs))
    fs = np.array(fs)
    with asaga.Batch(ps, storage="f32", epochs_per_segment=2, abar_recompute_every=5) as b:
        asaga.asaga_batch_autotune(b.b, b.count)
        asaga.asaga_batch_set_row_paths(b.b, [0, 0, 450, -1], [4, 2, 4, 1])
        got = [asaga.asaga_batch_get_info(b.b, i) for i in range(b.count)]
        assert [(g["row_threshold"], g["row_group"]) for g in got] == [(0, 4), (0, 2), (450, 4), (-1, 1)]
        s, res = asaga.asaga_batch_run(b.b, b.count, 600, 1e-6, fs)
        assert s == asaga.OK, (asaga.STATUS_NAMES[s], [r.as_dict() for r in res])
        for i, p in enumerate(ps):
            x = asaga.asaga_batch_get_state(b.b, i, p.d, p.n)[0]
            assert R.objective(p, x.astype(np.float64)) - fs[i] <= 1e-6 * abs(fs[i])
        with pytest.raises(asaga.AsagaError):
            asaga.asaga_batch_set_row_paths(b.b, [0, 0, 0, 0], [8, 1, 1, 1])  # blocks of 4 warps
