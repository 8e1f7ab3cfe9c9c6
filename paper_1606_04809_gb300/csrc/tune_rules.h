// Decision rules of the autotuners on a trial's record (host code only, no
// CUDA): the least-squares trend of log10 |grad f|^2 over epochs, the test
// that tells convergence from the plateau above the stability frontier, and
// the predicted epochs to the level the race aims at.  asaga_autotune and
// asaga_batch_autotune apply them; the CPU tests call them through a small
// shim against closed forms and a library regression.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace asaga {
namespace tune {

// log10 of |grad f|^2 / |grad f(x=0)|^2: the level the predictions aim at,
// and the level that proves convergence in a frontier trial
inline constexpr double kTuneDeep = -10.0;
inline constexpr double kTuneConverged = -6.0;

struct TuneTrial {
    bool diverged = false;
    int epochs = 0;
    double t_ms = 0;                 // update-kernel time
    std::vector<double> y;           // log10 |grad f|^2 / g0 after each epoch
    double ms_per_epoch() const { return epochs > 0 ? t_ms / epochs : INFINITY; }
};

// Least-squares line through (e, y[e-1]) for e = first .. y.size().
struct Trend {
    double slope = 0, se = INFINITY, e_mean = 0, y_mean = 0;
};
inline Trend trend(const std::vector<double> &y, int first) {
    Trend t;
    const int m = (int)y.size(), k = m - first + 1;
    if (k < 3) return t;
    double se = 0, sy = 0;
    for (int e = first; e <= m; ++e) {
        se += e;
        sy += y[e - 1];
    }
    t.e_mean = se / k;
    t.y_mean = sy / k;
    double sxx = 0, sxy = 0;
    for (int e = first; e <= m; ++e) {
        sxx += (e - t.e_mean) * (e - t.e_mean);
        sxy += (e - t.e_mean) * (y[e - 1] - t.y_mean);
    }
    t.slope = sxy / sxx;
    double rss = 0;
    for (int e = first; e <= m; ++e) {
        const double r = y[e - 1] - t.y_mean - t.slope * (e - t.e_mean);
        rss += r * r;
    }
    t.se = std::sqrt(rss / std::max(1, k - 2) / sxx);
    return t;
}

// A frontier trial converges when |grad f|^2 reached kTuneConverged, or when
// its trend from the fourth epoch on falls with t-statistic >= 3.5.  On the
// plateau above the frontier |grad f|^2 bounces by one to two decades with
// no trend, which this test rejects.
inline bool converging(const TuneTrial &t) {
    if (t.diverged) return false;
    for (double v : t.y)
        if (v <= kTuneConverged) return true;
    const int m = (int)t.y.size();
    const Trend tr = trend(t.y, std::max(3, m / 4));
    return tr.slope < 0 && -tr.slope >= 3.5 * tr.se;
}

// Predicted epochs for |grad f|^2 to reach kTuneDeep: the first epoch that
// reached it, else the least-squares trend of the trial's last two thirds,
// if it falls with t-statistic >= 3 (INFINITY otherwise).
inline double predict_epochs(const TuneTrial &t) {
    if (t.diverged) return INFINITY;
    const int m = (int)t.y.size();
    for (int e = 1; e <= m; ++e)
        if (t.y[e - 1] <= kTuneDeep) return e;
    if (m < 5) return INFINITY;
    const Trend tr = trend(t.y, std::max(3, m / 3));
    if (!(tr.slope < -1e-3) || -tr.slope < 3.0 * tr.se) return INFINITY;
    return std::max((double)m, tr.e_mean + (kTuneDeep - tr.y_mean) / tr.slope);
}

}  // namespace tune
}  // namespace asaga
