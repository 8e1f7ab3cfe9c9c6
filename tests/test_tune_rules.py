"""The autotuners' decision rules on a trial's record (csrc/tune_rules.h),
built with the host compiler through a small C shim, on CPU.

A trial records y_e = log10 |grad f(x_e)|^2 / |grad f(0)|^2 after each epoch
e = 1..m.  Pinned here:
  * the least-squares trend equals scipy's linear regression (slope and its
    standard error) and, on an exact line, the line itself;
  * convergence: any record at or below the convergence level counts; else
    a falling trend with t >= 3.5; a plateau that bounces by one to two
    decades with no trend, a rising record and a diverged trial do not;
  * predicted epochs: the first epoch at or below the prediction level if
    one is; else the crossing of the fitted line (closed form for an exact
    line) when it falls with t >= 3 over the last two thirds; never fewer
    than the trial's own epochs; no prediction for flat, rising, short or
    diverged records.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1606_04809_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("tune") / "libtune_rules.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "tune_rules_shim.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    dp, i = ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.shim_trend.argtypes = [dp, i, i, dp]
    L.shim_trend.restype = None
    L.shim_converging.argtypes = [dp, i, i]
    L.shim_converging.restype = i
    L.shim_predict_epochs.argtypes = [dp, i, i]
    L.shim_predict_epochs.restype = ctypes.c_double
    L.shim_level.argtypes = [i]
    L.shim_level.restype = ctypes.c_double
    return L


def arr(y):
    a = np.ascontiguousarray(y, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def trend(L, y, first):
    a, p = arr(y)
    out = np.zeros(4)
    L.shim_trend(p, len(a), first, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def converging(L, y, diverged=False):
    a, p = arr(y)
    return bool(L.shim_converging(p, len(a), int(diverged)))


def predict(L, y, diverged=False):
    a, p = arr(y)
    return L.shim_predict_epochs(p, len(a), int(diverged))


def test_levels(lib):
    assert lib.shim_level(0) == -10.0 and lib.shim_level(1) == -6.0


def test_trend_equals_a_library_regression(lib):
    stats = pytest.importorskip("scipy.stats")
    g = np.random.default_rng(5)
    for m, first in ((16, 4), (24, 8), (40, 3), (7, 5)):
        y = -0.3 * np.arange(1, m + 1) + g.normal(0, 0.4, m)
        slope, se, e_mean, y_mean = trend(lib, y, first)
        e = np.arange(first, m + 1)
        ref = stats.linregress(e, y[first - 1:])
        assert slope == pytest.approx(ref.slope, rel=1e-12, abs=1e-14)
        assert se == pytest.approx(ref.stderr, rel=1e-10)
        assert e_mean == pytest.approx(e.mean()) and y_mean == pytest.approx(y[first - 1:].mean())


def test_trend_of_an_exact_line_and_of_too_few_points(lib):
    y = 2.0 - 0.5 * np.arange(1, 13)
    slope, se, _, _ = trend(lib, y, 3)
    assert slope == pytest.approx(-0.5, rel=1e-14) and se <= 1e-14
    slope, se, _, _ = trend(lib, y[:4], 3)  # two points: no trend
    assert slope == 0 and se == np.inf


def test_convergence_level_reached_counts(lib):
    assert converging(lib, [-1, -3, -5, -6.0, -5.5, -5.8])
    assert not converging(lib, [-1, -3, -5, -5.9, -5.5, -5.8])  # no trend after the fourth epoch


def test_a_falling_trend_converges_and_a_plateau_does_not(lib):
    g = np.random.default_rng(11)
    e = np.arange(1, 17)
    for seed in range(20):
        falling = -0.25 * e + g.normal(0, 0.15, 16)  # above -6 throughout, t far above 3.5
        assert falling.min() > -6 and converging(lib, falling)
        # bounces by one to two decades around -3 with no trend
        plateau = -3.0 + np.random.default_rng(100 + seed).uniform(-1.0, 1.0, 16)
        assert not converging(lib, plateau), seed
        assert not converging(lib, -3.0 + 0.5 * np.sin(e))  # periodic bounce, no trend
    assert not converging(lib, 0.1 * e - 2)  # rising
    assert not converging(lib, -0.5 * e, diverged=True)


def test_predicted_epochs(lib):
    # the first epoch at or below the prediction level
    assert predict(lib, [-2, -5, -9, -10.0, -12]) == 4
    assert predict(lib, [-2, -5, -9, -11.5]) == 4
    # an exact line that has not reached it: its crossing, e = (y0 - (-10)) / 0.25 for y = y0 - 0.25 e
    y = -1.0 - 0.25 * np.arange(1, 21)
    assert predict(lib, y) == pytest.approx((-1.0 + 10.0) / 0.25, rel=1e-12)
    # never fewer epochs than the trial ran
    y = 5.0 - 0.8 * np.arange(1, 19)  # reaches -9.4 at e = 18, crossing at 18.75
    assert predict(lib, y) == pytest.approx(18.75, rel=1e-12)
    # no prediction: flat, rising, too short, diverged, a slope too small
    assert predict(lib, np.full(20, -3.0)) == np.inf
    assert predict(lib, -3.0 + 0.1 * np.arange(20)) == np.inf
    assert predict(lib, [-1, -2, -3, -4]) == np.inf
    assert predict(lib, -0.5 * np.arange(1, 21), diverged=True) == np.inf
    assert predict(lib, -3.0 - 1e-4 * np.arange(1, 21)) == np.inf
