"""Writes the float64 optimum f* of the named synthetic workloads to
tests/golden/fstar_<name>.json, using only the CPU checker (oracle/) and the
seeded data generator.

f* is certified by strong convexity: f(x) - f* <= |grad f(x)|^2 / (2 lambda)
(mu >= lambda), run until that bound is <= 1e-10 |f(x)|; the ridge workload
also records the closed-form optimum (normal equations).  The stored
fingerprint lets a consumer check that it regenerated the same problem.

    python tests/golden/make_fstar.py rcv1like covtypelike urllike
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import reference as R  # noqa: E402
from paper_1606_04809_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {
    "rcv1like": lambda: synth.rcv1_like(),
    "urllike": lambda: synth.url_like(),
    "covtypelike": lambda: synth.covtype_like(),
    "smalllogistic": lambda: synth.small_logistic(),
}
SAMPLER_SEED = 30


def main(names):
    for name in names:
        t0 = time.time()
        p = WORKLOADS[name]()
        out = {"name": name, "problem": p.name, "fingerprint": p.fingerprint(), "lambda": p.lam,
               "loss": p.loss, "storage": p.storage}
        if p.loss == "squared":
            xs = R.ridge_closed_form(p)
            out.update(fstar=R.objective(p, xs), bound=R.suboptimality_bound(p, xs), method="closed form")
        else:
            res = R.certified_fstar(p, lambda ep: synth.sample_indices(p.n, p.n, SAMPLER_SEED, ep),
                                    rel_tol=1e-10, max_epochs=300, log=print)
            out.update(fstar=res["fstar"], bound=res["bound"], epochs=res["epochs"],
                       method="serial float64 Sparse SAGA, certified by |grad f|^2/(2 lambda)")
        out["seconds"] = time.time() - t0
        with open(os.path.join(HERE, f"fstar_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, out["fstar"], out["bound"], f"{out['seconds']:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["smalllogistic", "covtypelike", "rcv1like"])
