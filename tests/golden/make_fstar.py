"""Writes the float64 optimum f* of the named synthetic workloads to
tests/golden/fstar_<name>.json, using only the CPU checker (oracle/) and the
seeded data generator.

f* is certified by strong convexity: f(x) - f* <= |grad f(x)|^2 / (2 lambda)
(mu >= lambda), run until that bound is <= 1e-10 |f(x)|; the ridge workload
also records the closed-form optimum (normal equations).  The stored
fingerprint lets a consumer check that it regenerated the same problem.

    python tests/golden/make_fstar.py rcv1like covtypelike urllike
    python tests/golden/make_fstar.py batch256_full      # the full-size batch, all host cores
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

BATCH = dict(count=256, seed=51, n_range=(1_000, 20_000), d_range=(100, 5_000), density_range=(0.005, 0.02),
             lam_range=(1e-6, 1e-2), storage="bf16")

WORKLOADS = {
    "rcv1like": lambda: synth.rcv1_like(),
    "urllike": lambda: synth.url_like(),
    "covtypelike": lambda: synth.covtype_like(),
    "smalllogistic": lambda: synth.small_logistic(),
}
SAMPLER_SEED = 30


def batch_fstar():
    """One certified f* per instance of the 256-instance batch workload."""
    t0 = time.time()
    ps = synth.logistic_batch(**BATCH)
    items = []
    for k, p in enumerate(ps):
        res = R.certified_fstar(p, lambda ep, p=p: synth.sample_indices(p.n, p.n, SAMPLER_SEED, ep),
                                rel_tol=1e-10, max_epochs=20000, check_every=10)
        items.append({"fingerprint": p.fingerprint(), "lambda": p.lam, "fstar": res["fstar"],
                      "bound": res["bound"], "epochs": res["epochs"]})
        print(k, p.n, p.d, p.nnz, p.lam, res["epochs"], res["fstar"], flush=True)
    out = {"name": "batch256", "generator": {k: list(v) if isinstance(v, tuple) else v for k, v in BATCH.items()},
           "method": "serial float64 Sparse SAGA per instance, certified by |grad f|^2/(2 lambda)",
           "instances": items, "seconds": time.time() - t0}
    with open(os.path.join(HERE, "fstar_batch256.json"), "w") as f:
        json.dump(out, f, indent=1)


def _full_batch_one(spec):
    """Certified f* of one full-size batch instance (run in a worker process)."""
    t0 = time.time()
    p = synth.batch_instance(spec, values="f64", threads=2)
    res = R.certified_fstar(p, lambda ep, p=p: synth.sample_indices(p.n, p.n, SAMPLER_SEED, ep),
                            rel_tol=1e-10, max_epochs=5000, check_every=5)
    return {"k": spec["k"], "fingerprint": p.fingerprint(), "lambda": p.lam, "fstar": res["fstar"],
            "bound": res["bound"], "epochs": res["epochs"], "seconds": time.time() - t0}


def full_batch_fstar(workers=None):
    """One certified f* per instance of the full-size batch workload
    (synth.FULL_BATCH, instances from the C generator), on a pool of worker
    processes, largest instances first."""
    import multiprocessing as mp
    t0 = time.time()
    specs = synth.batch_params(**synth.FULL_BATCH)
    order = sorted(specs, key=lambda s: -s["n"] * s["k_mean"])
    workers = workers or max(1, min(6, (os.cpu_count() or 2) - 1))
    items = {}
    with mp.get_context("spawn").Pool(workers) as pool:
        for r in pool.imap_unordered(_full_batch_one, order):
            items[r["k"]] = r
            print(len(items), r["k"], r["fingerprint"]["nnz"], r["lambda"], r["epochs"], f"{r['seconds']:.0f}s",
                  r["fstar"], flush=True)
    out = {"name": "batch256_full", "generator": {k: list(v) if isinstance(v, tuple) else v
                                                  for k, v in synth.FULL_BATCH.items()},
           "method": "serial float64 Sparse SAGA per instance, certified by |grad f|^2/(2 lambda)",
           "instances": [items[k] for k in sorted(items)], "seconds": time.time() - t0}
    with open(os.path.join(HERE, "fstar_batch256_full.json"), "w") as f:
        json.dump(out, f, indent=1)


def main(names):
    for name in names:
        if name == "batch256":
            batch_fstar()
            continue
        if name == "batch256_full":
            full_batch_fstar()
            continue
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
