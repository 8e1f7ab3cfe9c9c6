"""The batch workload at its specified size (256 l2-logistic instances,
n in [10k, 200k], d in [1k, 50k], density 0.5-2%, Zipf(1.1) columns, lambda on
a log grid 1e-6..1e-2, bf16 values), on a deterministic subset of its
instances, through the C ABI.

The instances come from the C generator (the same bits on every host), are
checked against the fingerprints stored with their certified float64 f*
(tests/golden/fstar_batch256_full.json, written by make_fstar.py with the
serial checker alone), solved together in one batch to 1e-6 relative
suboptimality, and each final iterate is evaluated again by the float64
checker: (f(x) - f*) / |f*| <= 1e-6 + bound / |f*|, bound being the
certificate's own slack.
"""
import json
import os

import numpy as np
import pytest

from oracle import reference as R
from paper_1606_04809_gb300 import asaga, build, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# the smallest and largest lambda, two in between, the longest mean row and the most rows
SUBSET = (0, 85, 170, 255)


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return asaga.load()


@pytest.fixture(scope="module")
def subset():
    specs = synth.batch_params(**synth.FULL_BATCH)
    pick = list(SUBSET)
    pick.append(max(range(len(specs)), key=lambda k: specs[k]["k_mean"]))
    pick.append(max(range(len(specs)), key=lambda k: specs[k]["n"]))
    pick = sorted(set(pick))
    gold = {g["k"]: g for g in json.load(open(os.path.join(HERE, "golden", "fstar_batch256_full.json")))["instances"]}
    ps, gs = [], []
    for k in pick:
        p = synth.batch_instance(specs[k], values="f64")
        assert p.fingerprint() == gold[k]["fingerprint"], f"instance {k} differs from the certified one"
        ps.append(p)
        gs.append(gold[k])
    return ps, gs


def test_full_size_instances_reach_1e6_in_one_batch(subset):
    ps, gs = subset
    fs = np.array([g["fstar"] for g in gs])
    with asaga.Batch(ps, storage="bf16", values_dtype="bf16", epochs_per_segment=1, abar_recompute_every=5) as b:
        asaga.asaga_batch_autotune(b.b, b.count)
        s, res = asaga.asaga_batch_run(b.b, b.count, 2000, 1e-6, fs)
        assert s == asaga.OK, (asaga.STATUS_NAMES[s], [r.as_dict() for r in res])
        for i, p in enumerate(ps):
            x = asaga.asaga_batch_get_state(b.b, i, p.d, p.n)[0]
            f = R.objective(p, x.astype(np.float64))
            assert (f - fs[i]) / abs(fs[i]) <= 1e-6 + gs[i]["bound"] / abs(fs[i]), (i, p.name)
            assert res[i].updates == round(res[i].epochs * p.n)
