#!/usr/bin/env python3
"""Throughput and time-to-accuracy of asynchronous Sparse SAGA (ASAGA) on GB300.

One step = one epoch of asynchronous Sparse SAGA updates (n sampled rows,
Algorithm 2) followed by the segment boundary: the float64 objective and the
stopping test (plus the float64 abar recomputation every 5th step).  The
metric is epochs/s on the RCV1-shaped l2-logistic workload (n=700000,
d=47000, ~75 nnz per row with Zipf(1.1) columns, fp32 values, lambda=1/n,
gamma=1/(3L)), with the problem resident in HBM.  The line also reports:
  time_to_target  seconds from x=0 to 1e-6 relative suboptimality against
                  the float64 f* stored in tests/golden;
  e2e             the same epochs/s through the public C ABI from pinned host
                  buffers, every step copying the problem in and the iterate
                  out (asaga_create -> asaga_run(1 epoch) -> asaga_get_state
                  -> asaga_destroy);
  roofline        algorithmic HBM bytes of the update kernel per launch over
                  its CUDA-event time, against the measured HBM peak;
  hotline         the floor that the most frequent column's state line sets
                  (its L2 slice serialises every update's read and reduction
                  of it), measured live, against the kernel's epoch time;
  cpu_baseline    the float64 CPU checker on a bounded sample, one host core;
                  beside it (asaga_all_cores) lock-free ASAGA in C on every
                  host core, the paper's own kind of implementation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1606_04809_gb300 import synth  # noqa: E402

WORKLOADS = {
    "rcv1like": dict(make=synth.rcv1_like, golden="fstar_rcv1like.json",
                     desc="l2-logistic, RCV1-shaped synthetic: n=700000, d=47000, ~75 nnz/row (4..1224, "
                          "lognormal), Zipf(1.1) columns, |N(0,1)| row-normalised, fp32 values, lambda=1/n, "
                          "gamma=1/(3L)"),
    "covtypelike": dict(make=synth.covtype_like, golden="fstar_covtypelike.json",
                        desc="ridge, Covtype-shaped synthetic: n=581000, d=54 dense, N(0,1) standardised, fp16 "
                             "values, lambda=1e-3, gamma=1/(3L)"),
    "urllike": dict(make=synth.url_like, golden="fstar_urllike.json",
                    desc="l2-logistic, URL-shaped synthetic: n=2400000, d=3200000, ~115 nnz/row (16..414), "
                         "Zipf(1.1) columns, binary row-normalised, bf16 values, lambda=1/n, gamma=1/(3L)"),
}
ABAR_EVERY = 5
TARGET = 1e-6
# 256 independent l2-logistic instances (a regularisation path): the batch workload (n ~ U[10k, 200k],
# d ~ U[1k, 50k]) with n and d scaled by 1/10 so that the seeded CPU generator and the float64
# certificates stay within minutes
BATCH = dict(count=256, seed=51, n_range=(1_000, 20_000), d_range=(100, 5_000), density_range=(0.005, 0.02),
             lam_range=(1e-6, 1e-2), storage="bf16")
BATCH_DESC = ("256 l2-logistic instances: n~U[1000,20000], d~U[100,5000], density~U[0.5%,2%], Zipf(1.1) columns, "
              "|N(0,1)| row-normalised, lambda on a log grid 1e-6..1e-2, bf16 values, fp32 state "
              "(n and d scaled 1/10 from the specified batch)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rcv1like", choices=sorted(WORKLOADS) + ["batch"])
    ap.add_argument("--single-sample", type=int, default=256,
                    help="batch workload: instances also solved one at a time in fp32 for comparison")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--experiment", default=None, choices=["warps", "overlap", "cas", "sampling"],
                    help="reproduce one of the paper's qualitative experiments instead of the benchmark")
    ap.add_argument("--warps", type=int, default=0, help="fixed concurrent warps (skips the autotuner)")
    ap.add_argument("--compact", type=int, default=0, choices=[0, 1],
                    help="compact storage of A (uint16 indices / one value per row where exact)")
    ap.add_argument("--gamma-scale", type=float, default=1.0, help="with --warps: step = scale / (3L)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_golden(name, p):
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None, "no stored f*"
    g = json.load(open(path))
    fp, want = p.fingerprint(), g["fingerprint"]
    same = (fp["structure_sha256"] == want["structure_sha256"]
            and abs(fp["sum_values"] - want["sum_values"]) <= 1e-9 * abs(want["sum_values"])
            and abs(fp["sum_labels"] - want["sum_labels"]) <= 1e-9 * max(1.0, abs(want["sum_labels"])))
    if not same:
        return None, "regenerated problem differs from the one f* was computed for"
    return g, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return float(json.load(open(path))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def ncu_summary(workload, profile=None):
    """Per-launch DRAM bytes and the L2 throughput (% of peak) of the update
    kernel from the committed ncu summary (profiles/update_kernel_<workload>.md,
    or profiles/<profile>.md), if it was taken on the current kernel source;
    None otherwise."""
    path = os.path.join(ROOT, "profiles", f"{profile or 'update_kernel_' + workload}.md")
    src = os.path.join(ROOT, "paper_1606_04809_gb300", "csrc", "update.cu")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    kv = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("update.cu sha256") != sha:
        return None
    try:
        out = {"traffic": int(float(kv["traffic_bytes_per_launch"]))}
    except Exception:
        return None
    for key, name in (("l2_throughput_pct_of_peak", "l2_pct"), ("dram_throughput_pct_of_peak", "dram_pct")):
        try:
            out[name] = float(kv[key])
        except Exception:
            pass
    return out


def line_floor(p, kernel_ms):
    """The epoch floor set by the most frequent column's state line.

    Each update whose row holds a column reads that column's 16-byte state and
    then reduces into it; the line's L2 slice serialises the pairs, so an
    epoch needs at least (rows holding the most frequent column) x (service
    time per pair), the latter measured by asaga_probe_line_rate with enough
    warps to saturate the line.
    """
    from paper_1606_04809_gb300 import asaga

    c_max = int(p.n) if p.dense else int(np.bincount(p.col_idx, minlength=p.d).max())
    warps, pairs = 2048, 500
    ns = asaga.asaga_probe_line_rate(warps, pairs)
    floor_ms = c_max * ns * 1e-6
    return {"bound": "l2_line", "ns_per_pair": ns, "pairs_per_epoch": c_max, "floor_ms": floor_ms,
            "kernel_ms": kernel_ms, "frac": floor_ms / kernel_ms,
            "probe": f"asaga_probe_line_rate({warps} warps x {pairs} pairs on one line)"}


def update_hbm_bytes(p, storage, info=None):
    """Algorithmic HBM bytes of one epoch of updates: each sampled row reads
    its CSR slice (index + value per entry; 2-byte indices and one value per
    row in the compact layout) once, row_ptr (2 x 8 B), its label (4 B) and
    swaps alpha_i (4 B read + 4 B write).  The per-column state is
    L2-resident by design and not counted."""
    vsz = {"f32": 4, "bf16": 2, "f16": 2}[storage]
    idx = 0 if p.dense else (info["col_index_bytes"] if info else 4)
    row_values = bool(info and info["row_values"])
    per_nnz = (0 if row_values else vsz) + idx
    per_row = (0 if p.dense else 16) + 4 + 8 + (4 if row_values else 0)
    return p.nnz * per_nnz + p.n * per_row


# ---------------------------------------------------------------- reference arm

REFERENCE_STEPS_PER_EPOCH = 16

def time_checker(p, seconds, steps=None, warmup=0, per_epoch=1):
    """Float64 CPU checker.  One step = n/per_epoch serial Sparse SAGA updates,
    with the float64 objective after every per_epoch-th step (per_epoch = 1:
    a step is one epoch and its objective).  Runs `steps` steps, or as many as
    fit in `seconds`; returns (epochs/s, steps done, seconds)."""
    from oracle import reference as R
    L = R.lipschitz(p)
    gamma, D = 1.0 / (3.0 * L), R.reweighting(p)
    st = R.State.zeros(p)
    count = -(-p.n // per_epoch)

    def step(k):
        R.sparse_saga(p, st, synth.sample_indices(p.n, count, 30, k + 1), gamma, D)
        if (k + 1) % per_epoch == 0:
            R.objective(p, st.x)

    for k in range(warmup):
        step(k)
    t0, done = time.perf_counter(), 0
    while True:
        step(warmup + done)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= seconds):
            break
    return done * count / p.n / el, done, el


def time_cpu_asaga(p, seconds, fstar, target):
    """Multi-threaded lock-free ASAGA on all host cores (Algorithm 2 with the
    compare-and-swap adds of App. G.2, C, float64): epochs/s of the updates and
    the update time to `target` relative suboptimality (the float64 objective
    after each epoch is not timed).  Runs until the target or `seconds`."""
    from oracle import cpu_asaga
    from oracle import reference as R
    gamma = 1.0 / (3.0 * R.lipschitz(p))
    run = cpu_asaga.Runner(p)
    st = R.State.zeros(p)
    upd, epochs, ttt = 0.0, 0, None
    t_all = time.perf_counter()
    while time.perf_counter() - t_all < seconds:
        t0 = time.perf_counter()
        run.run(st, p.n, gamma, seed=4)
        upd += time.perf_counter() - t0
        epochs += 1
        if fstar is not None and (R.objective(p, st.x) - fstar) / abs(fstar) <= target:
            ttt = upd
            break
    return {"value": epochs / upd, "unit": "epochs/s", "cores": run.threads,
            "kind": "lock-free ASAGA on the host cores (Algorithm 2, CAS adds as in App. G.2), float64, C",
            "gamma": gamma, "epochs": epochs, "update_seconds": upd,
            "time_to_target": ({"target_rel_subopt": target, "seconds_updates": ttt, "epochs": epochs}
                               if ttt is not None else None),
            "sample": f"{epochs} epochs from x=0 ({upd:.1f} s of updates)"}


def run_reference(args, p, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    # each step is a bounded sample: 1/16 of an epoch of serial updates, the
    # objective after every 16th step, so K steps stay within minutes
    per_epoch = REFERENCE_STEPS_PER_EPOCH
    eps, done, el = time_checker(p, args.cpu_seconds, steps=args.steps, warmup=args.warmup, per_epoch=per_epoch)
    line = {
        "impl": "reference", "metric": "epochs/s", "value": eps, "unit": "epochs/s", "n_gpus": args.gpus,
        "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"]},
        "cpu_baseline": {"value": eps, "unit": "epochs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{done} steps of n/{per_epoch} serial float64 Sparse SAGA updates, the "
                                   f"float64 objective after every {per_epoch}th, from x=0 ({done / per_epoch:.2f} epochs)"},
        "e2e": {"value": eps, "unit": "epochs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm


def run_batch(args):
    """Batched bf16 solve of many instances vs the same instances solved one at a time in fp32."""
    import torch
    from paper_1606_04809_gb300 import asaga
    from paper_1606_04809_gb300 import build as lib_build
    from paper_1606_04809_gb300 import sharding

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib_build.build()
    asaga.load()
    ps_all = synth.logistic_batch(**BATCH)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "fstar_batch256.json")))
    fs_all = np.array([g["fstar"] for g in gold["instances"]])
    for p, g in zip(ps_all, gold["instances"]):
        if p.fingerprint()["structure_sha256"] != g["fingerprint"]["structure_sha256"]:
            raise SystemExit("regenerated batch differs from the one f* was computed for")
    mine = sharding.rank_instances([sharding.instance_cost(p) for p in ps_all], world, rank)
    ps = [ps_all[i] for i in mine]
    fs = fs_all[mine]
    stream = torch.cuda.current_stream()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    b = asaga.Batch(ps, storage="bf16", values_dtype="bf16", epochs_per_segment=1, abar_recompute_every=ABAR_EVERY,
                    cuda_stream=stream.cuda_stream)
    t0 = time.perf_counter()
    tune = asaga.asaga_batch_autotune(b.b, b.count)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        asaga.asaga_batch_run(b.b, b.count, 1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches, seg_s = 0, 0.0
    for _ in range(args.steps):
        st, res = asaga.asaga_batch_run(b.b, b.count, 1)
        launches += res[0].kernel_launches
        seg_s += res[0].solver_seconds  # the batch epoch's segment (one CUDA graph)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    b.close()
    # HBM roofline of the batch epoch: A's bytes and the per-update row data of
    # every instance over the segment's device time (update launch plus the
    # batched objective, which the segment also holds: a lower bound on the
    # update kernel's own rate)
    hbm_bytes = sum(update_hbm_bytes(p, "bf16") for p in ps)
    peak, peak_kind = measured_peak_hbm()
    seg_ms = 1e3 * seg_s / args.steps
    achieved = hbm_bytes / (seg_ms * 1e-3) / 1e9
    ncu = ncu_summary("batch256", profile="batch_update_kernel_batch256") or {}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu.get("traffic"),
                "kernel": "batch segment: batch_update_kernel + the batched objective (one CUDA graph per batch epoch)",
                "algorithmic_bytes_per_launch": hbm_bytes, "kernel_ms": seg_ms, "peak_source": peak_kind,
                "l2_throughput_pct_of_peak_ncu": ncu.get("l2_pct"), "dram_throughput_pct_of_peak_ncu": ncu.get("dram_pct")}
    # time to 1e-6 for every instance of the batch
    b = asaga.Batch(ps, storage="bf16", values_dtype="bf16", epochs_per_segment=1, abar_recompute_every=ABAR_EVERY,
                    cuda_stream=stream.cuda_stream)
    asaga.asaga_batch_set_schedule(b.b, warps=[t["warps"] for t in tune], gamma=[t["gamma"] for t in tune])
    t0 = time.perf_counter()
    st, res = asaga.asaga_batch_run(b.b, b.count, 5000, TARGET, fs)
    batch_wall = time.perf_counter() - t0
    batch_dev = max(r.solver_seconds for r in res)
    b.close()
    ttt = {"status": asaga.STATUS_NAMES[st], "seconds_device": max_over_ranks(batch_dev), "seconds_wall": batch_wall,
           "max_epochs": max(r.epochs for r in res), "mean_epochs": float(np.mean([r.epochs for r in res])),
           "worst_rel_subopt": float(max(r.rel_subopt for r in res))}
    # the same instances one launch at a time, fp32 (a sample, every k-th instance)
    single = None
    if args.single_sample > 0 and rank == 0:
        step = max(1, len(ps) // args.single_sample)
        sample = list(range(0, len(ps), step))[: args.single_sample]
        tot_dev = tot_wall = tot_tune = 0.0
        statuses, failed = [], []
        for i in sample:
            with asaga.Context(ps[i], storage="f32", seed=i, abar_recompute_every=ABAR_EVERY,
                               cuda_stream=stream.cuda_stream) as c:
                t0 = time.perf_counter()
                tune1 = asaga.asaga_autotune(c.ctx, 20)
                tot_tune += time.perf_counter() - t0
                s1, r1 = asaga.asaga_run(c.ctx, 5000, TARGET, fs[i])
                statuses.append(asaga.STATUS_NAMES[s1])
                tot_dev += r1.solver_seconds + r1.eval_seconds
                tot_wall += r1.seconds
                if s1 != asaga.OK:
                    failed.append({"instance": i, "n": ps[i].n, "d": ps[i].d, "lambda": ps[i].lam,
                                   "status": asaga.STATUS_NAMES[s1], "epochs": r1.epochs,
                                   "rel_subopt": r1.rel_subopt, "warps": tune1["warps"], "gamma": tune1["gamma"],
                                   "tune_score": tune1["score"], "tune_trials": tune1["trials"]})
        batch_sample = float(max(res[i].solver_seconds for i in sample))
        single = {"instances": len(sample), "storage": "f32", "sum_seconds_device": tot_dev,
                  "sum_seconds_wall": tot_wall, "autotune_wall_seconds": tot_tune,
                  "all_ok": all(x == "ASAGA_OK" for x in statuses), "failed": failed,
                  "batch_seconds_for_same_instances": batch_sample,
                  "batch_seconds_all_instances": batch_dev,
                  "speedup_batch_vs_single_same_instances": tot_dev / batch_sample if batch_sample > 0 else None}
    # CPU baseline: the float64 oracle, three epochs (each with its objective)
    # on every 4th instance, scaled to the whole batch by nonzeros
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample = list(range(0, len(ps), 4))
        epochs_each, el = 3, 0.0
        for i in sample:
            el += time_checker(ps[i], 0.0, steps=epochs_each)[2]
        nnz_sample = sum(ps[i].nnz for i in sample)
        per_batch = el / epochs_each * sum(p.nnz for p in ps) / max(1, nnz_sample)
        cpu = {"value": 1.0 / per_batch, "unit": "epochs/s (whole batch)", "cores": 1, "kind": "oracle",
               "sample": f"{epochs_each} epochs of serial float64 Sparse SAGA + objective on {len(sample)} of "
                         f"{len(ps)} instances ({el:.2f} s), scaled to the batch by nonzeros"}
    if rank == 0:
        line = {"metric": "epochs/s", "value": world * args.steps / (ms * 1e-3), "unit": "epochs/s (whole batch)",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 values, f32 state",
                "data": "synthetic", "config": {"workload": BATCH_DESC, "instances_per_rank": len(ps),
                                                "nnz_total": int(sum(p.nnz for p in ps_all))},
                "instance_epochs_per_s": world * args.steps * len(ps) / (ms * 1e-3),
                "time_to_target": ttt, "autotune_wall_seconds": tune_s, "one_at_a_time_fp32": single,
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_experiment(args):
    """The paper's qualitative experiments on the GPU, one JSON line each:
      warps   -- epochs (and device seconds) to 1e-6 against the number of concurrent
                 warps, each at its fastest stable step (App. D.2, "theoretical speedups");
      overlap -- the overlap tau against the number of warps (App. E.2);
      cas     -- atomic against non-thread-safe updates: suboptimality reached and
                 the abar bookkeeping error (App. G.2);
      sampling -- rows drawn with replacement (Algorithm 2) against one permutation
                 per epoch, each autotuned, three seeds: epochs and device seconds
                 to 1e-6."""
    import torch
    from paper_1606_04809_gb300 import asaga
    from paper_1606_04809_gb300 import build as lib_build

    lib_build.build()
    asaga.load()
    wl = WORKLOADS[args.workload]
    p = wl["make"]()
    storage = p.storage if p.storage != "f64" else "f32"
    golden, why = load_golden(wl["golden"], p)
    if golden is None:
        raise SystemExit(why)
    fstar = golden["fstar"]
    out = {"experiment": args.experiment, "workload": wl["desc"], "fstar": fstar}
    rows = []
    if args.experiment == "warps":
        with asaga.Context(p, storage=storage) as c:
            gamma0 = asaga.asaga_get_info(c.ctx)["gamma"]
        for W in (16, 64, 256, 512, 1024, 2048):
            best = {"warps": W, "epochs": None}
            for k in range(0, 9):  # steps gamma0 * 2^(-k/2), largest first: keep the first that converges
                with asaga.Context(p, storage=storage, seed=7, max_warps=W, gamma=gamma0 * 2 ** (-k / 2),
                                   abar_recompute_every=ABAR_EVERY) as c:
                    s, r = asaga.asaga_run(c.ctx, 60, TARGET, fstar)
                if s == asaga.OK:
                    best = {"warps": W, "gamma_scale": 2 ** (-k / 2), "epochs": r.epochs,
                            "seconds_device": r.solver_seconds + r.eval_seconds}
                    break
            rows.append(best)
    elif args.experiment == "overlap":
        for W in (1, 16, 64, 256, 512, 1024, 2048, 4096):
            with asaga.Context(p, storage=storage, seed=7, max_warps=W, gamma=0.01) as c:
                o = asaga.asaga_measure_overlap(c.ctx, 0.05 if W == 1 else 1.0)
            rows.append(o)
    elif args.experiment == "sampling":
        for sampling in ("uniform", "permutation"):
            for seed in (1, 2, 3):
                with asaga.Context(p, storage=storage, seed=seed, sampling=sampling,
                                   abar_recompute_every=ABAR_EVERY) as c:
                    tune = asaga.asaga_autotune(c.ctx)
                    s, r = asaga.asaga_run(c.ctx, 300, TARGET, fstar)
                rows.append({"sampling": sampling, "seed": seed, "status": asaga.STATUS_NAMES[s],
                             "warps": tune["warps"], "gamma": tune["gamma"], "epochs": r.epochs,
                             "seconds_device": r.solver_seconds + r.eval_seconds})
    else:  # cas
        for plain in (0, 1):
            with asaga.Context(p, storage=storage, seed=7, max_warps=1024, gamma=0.05, plain_writes=plain,
                               abar_recompute_every=0) as c:
                s, r = asaga.asaga_run(c.ctx, 30, 0.0, fstar)
                drift = asaga.asaga_recompute_abar(c.ctx)
                f = asaga.asaga_objective(c.ctx)
            rows.append({"plain_writes": plain, "epochs": r.epochs, "rel_subopt": (f - fstar) / abs(fstar),
                         "abar_error": drift})
    out["rows"] = rows
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.experiment:
        return run_experiment(args)
    if args.workload == "batch":
        return run_batch(args)
    world, rank, local = dist_env()
    wl = WORKLOADS[args.workload]
    p = wl["make"]()
    if args.impl == "reference":
        return run_reference(args, p, wl)

    import torch
    from paper_1606_04809_gb300 import asaga
    from paper_1606_04809_gb300 import build as lib_build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib_build.build()
    asaga.load()
    stream = torch.cuda.current_stream()
    storage = p.storage if p.storage != "f64" else "f32"

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    opts = dict(seed=1000 + rank, abar_recompute_every=ABAR_EVERY, cuda_stream=stream.cuda_stream,
                compact=args.compact)
    ctx = asaga.Context(p, storage=storage, values_dtype=storage if storage != "f16" else "f64", **opts)
    # schedule: concurrent warps and step size picked by the native autotuner
    if args.warps > 0:
        L = asaga.asaga_get_info(ctx.ctx)["L"]
        ctx.close()
        opts.update(max_warps=args.warps, gamma=args.gamma_scale / (3.0 * L))
        ctx = asaga.Context(p, storage=storage, values_dtype=storage if storage != "f16" else "f64", **opts)
        tune = {"fixed": True, "warps": args.warps, "gamma_scale": args.gamma_scale}
    else:
        t_tune = time.perf_counter()
        tune = asaga.asaga_autotune(ctx.ctx)
        tune["wall_seconds"] = time.perf_counter() - t_tune
    info = asaga.asaga_get_info(ctx.ctx)
    opts.update(max_warps=info["warps"], gamma=info["gamma"])

    for _ in range(args.warmup):
        asaga.asaga_run(ctx.ctx, 1)
    barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver_s, launches, f_last = 0.0, 0, None
    e0.record(stream)
    for _ in range(args.steps):
        s, r = asaga.asaga_run(ctx.ctx, 1)
        solver_s += r.solver_seconds
        launches += r.kernel_launches
        f_last = r.f_last
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))

    value = world * args.steps / (ms * 1e-3)
    upd_ms = 1e3 * solver_s / args.steps
    hbm_bytes = update_hbm_bytes(p, storage, info)
    peak, peak_kind = measured_peak_hbm()
    achieved = hbm_bytes / (upd_ms * 1e-3) / 1e9
    ncu = ncu_summary(args.workload) or {}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu.get("traffic"), "kernel": "update_kernel (one launch = one epoch)",
                "algorithmic_bytes_per_launch": hbm_bytes, "kernel_ms": upd_ms, "peak_source": peak_kind,
                "l2_throughput_pct_of_peak_ncu": ncu.get("l2_pct"),
                "dram_throughput_pct_of_peak_ncu": ncu.get("dram_pct")}
    hotline = line_floor(p, upd_ms)

    # time to 1e-6 from x = 0
    ttt = None
    golden, why = load_golden(wl["golden"], p)
    if not args.no_ttt:
        if golden is None:
            ttt = {"status": "skipped", "reason": why}
        else:
            # the timed context itself, reset to x = 0 (it keeps the tuned schedule and block shape)
            asaga.asaga_set_state(ctx.ctx, np.zeros(p.d, np.float32), np.zeros(p.d, np.float32),
                                  np.zeros(p.n, np.float32), 0)
            f0 = asaga.asaga_objective(ctx.ctx)  # f(0), outside the timed run
            fstar = golden["fstar"]
            s, r = asaga.asaga_run(ctx.ctx, 200, TARGET, fstar)
            ttt = {"target_rel_subopt": TARGET, "status": asaga.STATUS_NAMES[s], "epochs": r.epochs,
                   "seconds_wall": r.seconds, "seconds_device": r.solver_seconds + r.eval_seconds,
                   "solver_seconds": r.solver_seconds, "eval_seconds": r.eval_seconds,
                   "rel_subopt": r.rel_subopt, "abs_subopt": r.f_last - fstar,
                   "subopt_over_initial": (r.f_last - fstar) / (f0 - fstar) if f0 != fstar else None,
                   "f0": f0, "fstar": fstar, "fstar_bound": golden["bound"]}
    ctx.close()

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        rp = torch.from_numpy(np.ascontiguousarray(p.row_ptr, dtype=np.int64)).pin_memory() if not p.dense else None
        ci = torch.from_numpy(np.ascontiguousarray(p.col_idx, dtype=np.int32)).pin_memory() if not p.dense else None
        npdt = {"f32": np.float32, "f16": np.float16}
        if storage == "bf16":
            v32 = np.ascontiguousarray(p.values, dtype=np.float32).view(np.uint32)
            vals = torch.from_numpy((v32 >> 16).astype(np.uint16).view(np.int16)).pin_memory()
        else:
            vals = torch.from_numpy(np.ascontiguousarray(p.values, dtype=npdt[storage])).pin_memory()
        lab = torch.from_numpy(np.ascontiguousarray(p.labels, dtype=np.float64)).pin_memory()
        prob = asaga.Problem(p.n, p.d, rp, ci, vals, storage, lab, dense=p.dense)
        xh = torch.empty(p.d, dtype=torch.float32).pin_memory()
        o = asaga.asaga_default_options(loss=p.loss, lam=p.lam, storage_dtype=storage, **opts)
        h2d = sum(t.numel() * t.element_size() for t in (rp, ci, vals, lab) if t is not None)
        d2h = p.d * 4 + 8
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            c = asaga.asaga_create(prob, o)
            asaga.asaga_set_schedule(c, info["warps"], info["gamma"], info["warps_per_block"])
            asaga.asaga_run(c, 1)
            asaga.load().asaga_get_state(c, xh.data_ptr(), None, None)
            asaga.asaga_destroy(c)
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * args.e2e_steps / el, "unit": "epochs/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "step": "asaga_create(pinned host CSR) + asaga_run(1 epoch) + asaga_get_state(x) + asaga_destroy"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        eps, done, el = time_checker(p, args.cpu_seconds)
        cpu = {"value": eps, "unit": "epochs/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} epochs of serial float64 Sparse SAGA + objective from x=0 ({el:.1f} s)"}
        cpu["asaga_all_cores"] = time_cpu_asaga(p, args.cpu_seconds * 2,
                                                golden["fstar"] if golden else None, TARGET)

    a_bytes = p.nnz * ({"f32": 4, "bf16": 2, "f16": 2}[storage] + (0 if p.dense else 4))
    if rank == 0:
        line = {
            "metric": "epochs/s", "value": value, "unit": "epochs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": p.n, "d": p.d, "nnz": p.nnz, "storage": storage,
                       "warps": info["warps"], "warps_per_block": info["warps_per_block"], "gamma": info["gamma"],
                       "abar_recompute_every": ABAR_EVERY, "compact": args.compact,
                       "col_index_bytes": info["col_index_bytes"], "row_values": info["row_values"],
                       "l2": f"inputs larger than L2 (A = {a_bytes / 1e6:.0f} MB > 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_target": ttt,
            "autotune": tune,
            "e2e": e2e,
            "roofline": roofline,
            "hotline": hotline,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clk,
            "f_last": f_last,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
