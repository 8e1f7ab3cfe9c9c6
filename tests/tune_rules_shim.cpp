// C entry points over the autotuners' decision rules (tune_rules.h), built
// by tests/test_tune_rules.py with the host compiler for CPU tests.
#include "tune_rules.h"

#include <vector>

using namespace asaga::tune;

namespace {
TuneTrial record(const double *y, int m, int diverged) {
    TuneTrial t;
    t.diverged = diverged != 0;
    t.y.assign(y, y + m);
    t.epochs = m;
    return t;
}
}  // namespace

extern "C" {
// out = {slope, se, e_mean, y_mean} of the least-squares line through
// (e, y[e-1]), e = first .. m
void shim_trend(const double *y, int m, int first, double *out) {
    const Trend t = trend(std::vector<double>(y, y + m), first);
    out[0] = t.slope;
    out[1] = t.se;
    out[2] = t.e_mean;
    out[3] = t.y_mean;
}
int shim_converging(const double *y, int m, int diverged) { return converging(record(y, m, diverged)) ? 1 : 0; }
double shim_predict_epochs(const double *y, int m, int diverged) { return predict_epochs(record(y, m, diverged)); }
double shim_level(int which) { return which == 0 ? kTuneDeep : kTuneConverged; }
}
