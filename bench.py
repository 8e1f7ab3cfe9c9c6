#!/usr/bin/env python3
"""Throughput and time-to-accuracy of asynchronous Sparse SAGA (ASAGA) on GB300.

One step = one epoch of asynchronous Sparse SAGA updates (n sampled rows,
Algorithm 2) followed by the segment boundary: the float64 objective and the
stopping test (plus the float64 abar recomputation every 5th step).  The
metric is epochs/s, with the problem resident in HBM, on the largest single
configuration, the URL-shaped l2-logistic workload (C2: n=2.4M, d=3.2M,
~115 nnz per row with Zipf(1.1) columns, bf16 values, fp32 state,
lambda=1/n); the RCV1-shaped (C1) and Covtype-shaped (C3) configurations are
measured the same way in the same run, under other_configs.  For each:
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
--workload batch measures the 256-instance batch (C4) instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
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

# L: the smoothness constant of the component the sparse update samples (its
# l2 part projected and reweighted by D_i, Sec. 4.2); gamma = 1/(3L) is the
# autotuner's starting step, which it scales by 2^(-k/2)
L_LOGISTIC = "max_i (0.25 |a_i|^2 + lambda max_{v in S_i} D_v)"
L_SQUARED = "max_i (|a_i|^2 + lambda max_{v in S_i} D_v)"
WORKLOADS = {
    "rcv1like": dict(make=synth.rcv1_like, golden="fstar_rcv1like.json", L=L_LOGISTIC,
                     desc="C1, RCV1-shaped l2-logistic: n=700000, d=47000, ~75 nnz/row (4..1224, lognormal), "
                          "Zipf(1.1) columns, |N(0,1)| row-normalised, fp32 values, lambda=1/n"),
    "covtypelike": dict(make=synth.covtype_like, golden="fstar_covtypelike.json", L=L_SQUARED,
                        desc="C3, Covtype-shaped ridge: n=581000, d=54 dense, N(0,1) standardised, fp16 values, "
                             "lambda=1e-3"),
    "urllike": dict(make=synth.url_like, golden="fstar_urllike.json", L=L_LOGISTIC,
                    desc="C2, URL-shaped l2-logistic: n=2400000, d=3200000, ~115 nnz/row (16..414), Zipf(1.1) "
                         "columns, binary row-normalised, bf16 values, fp32 state, lambda=1/n"),
}
ABAR_EVERY = 5
TARGET = 1e-6
L2_BYTES = 129 * 1024 * 1024  # GB300's L2
# the batch workload (C4): 256 independent l2-logistic instances (a regularisation path)
BATCH_DESC = ("C4, 256 l2-logistic instances: n~U[10000,200000], d~U[1000,50000], density~U[0.5%,2%] "
              "(rows of about density*d entries), Zipf(1.1) columns, |N(0,1)| row-normalised, lambda on a log "
              "grid 1e-6..1e-2, bf16 values, fp32 state")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="urllike", choices=sorted(WORKLOADS) + ["batch"])
    ap.add_argument("--also", default="rcv1like,covtypelike,batch",
                    help="other configurations measured in the same line (comma separated, 'none' for none)")
    ap.add_argument("--also-steps", type=int, default=100, help="timed steps of each --also configuration")
    ap.add_argument("--single-sample", type=int, default=32,
                    help="batch workload: instances also solved one at a time in fp32 for comparison")
    ap.add_argument("--batch-count", type=int, default=0, help="batch workload: the first K instances only")
    ap.add_argument("--batch-max-epochs", type=float, default=3000)
    ap.add_argument("--no-tune", action="store_true", help="batch workload: keep the default schedule and steps")
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
    ap.add_argument("--wpb", type=int, default=0, help="with --warps: warps per block (0: eight)")
    ap.add_argument("--draw-ahead", type=int, default=0, choices=[0, 1],
                    help="with --warps: draw the next row while an update's gathers are in flight")
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


def ncu_summary(profile):
    """Per-launch DRAM bytes and the L2 / DRAM throughput (% of peak) of a
    kernel from profiles/<profile>.json (written beside the ncu summary of the
    same name), if it was taken on the current kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", f"{profile}.json")
    src = os.path.join(ROOT, "paper_1606_04809_gb300", "csrc", "update.cu")
    if not os.path.exists(path):
        return None
    try:
        kv = json.load(open(path))
    except Exception:
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if kv.get("update_cu_sha256") != sha:
        return None
    out = {}
    try:
        out["traffic"] = int(kv["traffic_bytes_per_launch"])
    except Exception:
        return None
    for key, name in (("l2_throughput_pct_of_peak", "l2_pct"), ("dram_throughput_pct_of_peak", "dram_pct"),
                      ("traffic_bytes_per_full_launch", "traffic_full")):
        if key in kv:
            out[name] = float(kv[key])
    return out


def line_floor(p, kernel_ms):
    """The epoch floor set by the most frequent column's state line.

    Each update whose row holds a column reads that column's 8-byte state and
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


def static_config(wl, p, storage, compact, world):
    """The configuration keys that do not depend on the run (the same on both arms)."""
    a_bytes = p.nnz * ({"f32": 4, "bf16": 2, "f16": 2}[storage] + (0 if p.dense else 4))
    side = a_bytes + p.n * (8 + 4 + 8)  # A, row_ptr, labels and the memory
    return {"workload": wl["desc"], "n": p.n, "d": p.d, "nnz": p.nnz, "storage": storage,
            "L": wl["L"], "gamma_default": "1/(3L)", "abar_recompute_every": ABAR_EVERY, "compact": compact,
            "l2": (f"inputs larger than L2 (A = {a_bytes / 1e6:.0f} MB > 129 MB)" if a_bytes > L2_BYTES else
                   f"inputs ({side / 1e6:.0f} MB) fit in L2: each step timed alone, L2 flushed (a 258 MB write) "
                   f"between steps outside the timed events"),
            "parallelism": "replicas" if world > 1 else "single"}


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
        "config": static_config(wl, p, p.storage if p.storage != "f64" else "f32", 0, world),
        "cpu_baseline": {"value": eps, "unit": "epochs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{done} steps of n/{per_epoch} serial float64 Sparse SAGA updates, the "
                                   f"float64 objective after every {per_epoch}th, from x=0 ({done / per_epoch:.2f} epochs)"},
        "e2e": {"value": eps, "unit": "epochs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm


def load_full_batch(specs, indices, gold):
    """Generates instances `indices` of the full-size batch on the host (C
    generator, all cores), checks that each is the problem its f* was
    certified for, moves it to the device and drops the host copy.  Returns
    (metas: shapes and lambda only, structs over the device arrays, the
    device arrays, f*)."""
    import torch
    from paper_1606_04809_gb300 import asaga

    metas, structs, keep, fs = [], [], [], []
    for i in indices:
        p = synth.batch_instance(specs[i], values="bits")
        g = gold.get(specs[i]["k"])
        if g is None or g["fingerprint"] != p.fingerprint():
            raise SystemExit(f"instance {i}: no certified f* for this generated problem")
        fs.append(g["fstar"])
        dev = [torch.from_numpy(p.row_ptr).to("cuda"), torch.from_numpy(p.col_idx).to("cuda"),
               torch.from_numpy(p.values.view(np.int16)).to("cuda"), torch.from_numpy(p.labels).to("cuda")]
        keep.append(dev)
        structs.append(asaga.Problem(p.n, p.d, *dev[:3], "bf16", dev[3], on_device=True, nnz=p.nnz))
        m = synth.Problem(p.name, p.n, p.d, np.array([0, p.nnz]), p.col_idx[:0], p.values[:0], p.labels[:0],
                          p.loss, p.lam, p.storage)
        metas.append(m)  # nnz only (the arrays live on the device)
        del p
    torch.cuda.synchronize()
    return metas, structs, keep, np.array(fs)


def full_batch_gold():
    path = os.path.join(ROOT, "tests", "golden", "fstar_batch256_full.json")
    return {g["k"]: g for g in json.load(open(path))["instances"]} if os.path.exists(path) else {}


def batch_throughput(args, steps, env):
    """The full-size batch (C4) as one more configuration of the default line:
    every instance generated and resident, the default schedule and steps (no
    tuning), `steps` timed batch epochs (one graph segment each, the batched
    abar recomputation every 5th).  Time to 1e-6 needs the batch tuner and
    takes minutes; --workload batch measures it."""
    import torch
    from paper_1606_04809_gb300 import asaga
    from paper_1606_04809_gb300 import sharding

    world, rank, local, stream, barrier, max_over_ranks = env
    t_all = time.perf_counter()
    specs = synth.batch_params(**synth.FULL_BATCH)
    mine = sharding.rank_instances([s["n"] * s["k_mean"] for s in specs], world, rank)
    metas, structs, keep, fs = load_full_batch(specs, mine, full_batch_gold())
    gen_s = time.perf_counter() - t_all
    b = asaga.Batch(metas, storage="bf16", structs=structs, epochs_per_segment=1, abar_recompute_every=ABAR_EVERY,
                    cuda_stream=stream.cuda_stream)
    del structs, keep
    warps = sum(asaga.asaga_batch_get_info(b.b, i)["warps"] for i in range(b.count))
    asaga.asaga_batch_run(b.b, b.count, 1)  # warm-up (captures the segment graph)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seg_s, launches = 0.0, 0
    e0.record(stream)
    for _ in range(steps):
        st, res = asaga.asaga_batch_run(b.b, b.count, 1)
        seg_s += res[0].solver_seconds
        launches += res[0].kernel_launches
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1))
    b.close()
    hbm_bytes = sum(update_hbm_bytes(m, "bf16") for m in metas)
    peak, peak_kind = measured_peak_hbm()
    seg_ms = 1e3 * seg_s / steps
    ncu = ncu_summary("batch_update_kernel_batch256") or {}
    return {"metric": "epochs/s", "value": world * steps / (ms * 1e-3), "unit": "epochs/s (whole batch)",
            "steps": steps, "ms_per_step": ms / steps, "dtype": "bf16 values, f32 state",
            "instance_epochs_per_s": world * steps * len(mine) / (ms * 1e-3),
            "config": {"workload": BATCH_DESC, "instances_per_rank": len(mine),
                       "nnz_per_rank": int(sum(m.nnz for m in metas)), "warps_total": warps,
                       "schedule": "the default (warps in proportion to n_i (1 + k_i/128), steps 1/(3L_i)), untuned",
                       "l2": "inputs larger than L2 (A = 47 GB)"},
            "roofline": {"bound": "hbm", "achieved": hbm_bytes / (seg_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": hbm_bytes / (seg_ms * 1e-3) / 1e9 / peak, "traffic": ncu.get("traffic_full"),
                         "kernel": "batch segment: batch_update_kernel + the batched objective",
                         "algorithmic_bytes_per_launch": hbm_bytes, "kernel_ms": seg_ms, "peak_source": peak_kind},
            "time_to_target": {"status": "not measured here: `bench.py --workload batch` (tuner, then every "
                                         "instance to 1e-6)"},
            "gpu_launches": launches, "setup_seconds": gen_s}


def run_batch(args):
    """The 256-instance batch (C4) at its specified size: batched bf16 solve
    of every instance in one persistent, graph-captured launch per segment,
    against the same instances solved one launch at a time in fp32."""
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
    phases = {}
    t_all = time.perf_counter()
    specs = synth.batch_params(**synth.FULL_BATCH)
    if args.batch_count:
        specs = specs[: args.batch_count]
    gold = full_batch_gold()
    mine = sharding.rank_instances([s["n"] * s["k_mean"] for s in specs], world, rank)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    metas, structs, keep, fs = load_full_batch(specs, mine, gold)
    phases["generate_and_copy_s"] = time.perf_counter() - t0
    nnz_mine = int(sum(m.nnz for m in metas))
    print(f"batch: {len(mine)} instances, {nnz_mine} nonzeros generated in {phases['generate_and_copy_s']:.1f} s",
          file=sys.stderr, flush=True)

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    t0 = time.perf_counter()
    b = asaga.Batch(metas, storage="bf16", structs=structs, epochs_per_segment=1, abar_recompute_every=ABAR_EVERY,
                    cuda_stream=stream.cuda_stream)
    del structs, keep  # the library holds its own copy
    torch.cuda.synchronize()
    phases["create_s"] = time.perf_counter() - t0
    print(f"batch: created in {phases['create_s']:.1f} s", file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    if args.no_tune:  # the default schedule and steps (for profiling the kernels)
        tune = [{"warps": asaga.asaga_batch_get_info(b.b, i)["warps"]} for i in range(b.count)]
    else:
        tune = asaga.asaga_batch_autotune(b.b, b.count)
    phases["autotune_s"] = time.perf_counter() - t0
    print(f"batch: tuned in {phases['autotune_s']:.1f} s", file=sys.stderr, flush=True)
    infos = [asaga.asaga_batch_get_info(b.b, i) for i in range(b.count)]
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
        seg_s += res[0].solver_seconds  # the batch epoch's device time (graph segment and recomputation)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    # HBM roofline of the batch epoch: A's bytes and the per-update row data of
    # every instance over the segment's device time (update launch plus the
    # batched objective, which the segment also holds: a lower bound on the
    # update kernel's own rate)
    hbm_bytes = sum(update_hbm_bytes(m, "bf16") for m in metas)
    peak, peak_kind = measured_peak_hbm()
    seg_ms = 1e3 * seg_s / args.steps
    achieved = hbm_bytes / (seg_ms * 1e-3) / 1e9
    ncu = ncu_summary("batch_update_kernel_batch256") or {}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu.get("traffic_full") if not args.batch_count else None,
                "kernel": "batch segment: batch_update_kernel + the batched objective (one CUDA graph per batch epoch)",
                "algorithmic_bytes_per_launch": hbm_bytes, "kernel_ms": seg_ms, "peak_source": peak_kind,
                "l2_throughput_pct_of_peak_ncu": ncu.get("l2_pct"), "dram_throughput_pct_of_peak_ncu": ncu.get("dram_pct")}
    # time to 1e-6 of every instance, from x = 0 with the tuned schedule
    asaga.asaga_batch_reset(b.b)
    t0 = time.perf_counter()
    st, res = asaga.asaga_batch_run(b.b, b.count, args.batch_max_epochs, TARGET, fs)
    batch_wall = time.perf_counter() - t0
    batch_dev = max(r.solver_seconds for r in res)
    print(f"batch: time to target {batch_dev:.2f} s device, {batch_wall:.1f} s wall, "
          f"{asaga.STATUS_NAMES[st]}", file=sys.stderr, flush=True)
    ttt = {"status": asaga.STATUS_NAMES[st], "seconds_device": max_over_ranks(batch_dev), "seconds_wall": batch_wall,
           "max_epochs": max(r.epochs for r in res), "mean_epochs": float(np.mean([r.epochs for r in res])),
           "worst_rel_subopt": float(max(r.rel_subopt for r in res)),
           "instances_at_target": int(sum(r.rel_subopt <= TARGET for r in res)), "instances": len(res),
           "per_instance_seconds_device": [r.solver_seconds for r in res],
           "per_instance_epochs": [r.epochs for r in res]}
    b.close()
    # the same instances one launch at a time, fp32 (a sample, every k-th instance)
    single = None
    if args.single_sample > 0 and rank == 0:
        step = max(1, len(mine) // args.single_sample)
        sample = list(range(0, len(mine), step))[: args.single_sample]
        tot_dev = tot_wall = tot_tune = 0.0
        nnz_sample = 0
        statuses, failed = [], []
        dev_ok = nnz_ok = 0.0
        drawn_ahead = 0
        for j in sample:
            p = synth.batch_instance(specs[mine[j]], values="bits")
            nnz_sample += p.nnz
            with asaga.Context(p, storage="f32", values_dtype="f32", seed=j, abar_recompute_every=ABAR_EVERY,
                               cuda_stream=stream.cuda_stream) as c:
                t0 = time.perf_counter()
                tune1 = asaga.asaga_autotune(c.ctx, 20)
                tot_tune += time.perf_counter() - t0
                s1, r1 = asaga.asaga_run(c.ctx, args.batch_max_epochs, TARGET, fs[j])
                statuses.append(asaga.STATUS_NAMES[s1])
                tot_dev += r1.solver_seconds + r1.eval_seconds
                tot_wall += r1.seconds
                drawn_ahead += tune1["draw_ahead"]
                if s1 != asaga.OK:
                    failed.append({"instance": mine[j], "n": p.n, "d": p.d, "lambda": p.lam,
                                   "status": asaga.STATUS_NAMES[s1], "epochs": r1.epochs,
                                   "rel_subopt": r1.rel_subopt, "warps": tune1["warps"], "gamma": tune1["gamma"],
                                   "draw_ahead": tune1["draw_ahead"]})
                else:
                    dev_ok += r1.solver_seconds + r1.eval_seconds
                    nnz_ok += p.nnz
            del p
        # one at a time, the instances' times add up; the batch solves all of them in batch_dev
        all_est = tot_dev if len(sample) == len(mine) else tot_dev * nnz_mine / max(1, nnz_sample)
        single = {"instances": len(sample), "storage": "f32", "sum_seconds_device": tot_dev,
                  "sum_seconds_wall": tot_wall, "autotune_wall_seconds": tot_tune,
                  "all_ok": all(x == "ASAGA_OK" for x in statuses), "failed": failed,
                  "sum_seconds_device_all_instances": all_est,
                  "all_instances": "measured" if len(sample) == len(mine) else
                                   f"the sample's sum scaled by nonzeros ({nnz_mine} / {nnz_sample})",
                  "batch_seconds_all_instances": batch_dev,
                  "speedup_batch_vs_one_at_a_time": all_est / batch_dev if batch_dev > 0 and not failed else None,
                  # with a failed instance the sum above holds its whole epoch budget: the
                  # converged instances alone, scaled by nonzeros, bound the comparison instead
                  "speedup_converged_instances_only": (dev_ok * nnz_mine / nnz_ok / batch_dev
                                                       if failed and nnz_ok > 0 and batch_dev > 0 else None),
                  "instances_tuned_to_draw_ahead": drawn_ahead,
                  "note": "time to 1e-6 on both sides counts the updates, the float64 evaluations and the abar "
                          "recomputations (device time); tuning is reported separately"}
    # CPU baseline: the float64 oracle, one epoch (with its objective) on a
    # sample of instances, scaled to the whole batch by nonzeros
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample = list(range(0, len(mine), max(1, len(mine) // 16)))
        el, nnz_sample = 0.0, 0
        for j in sample:
            p = synth.batch_instance(specs[mine[j]], values="f64")
            el += time_checker(p, 0.0, steps=1)[2]
            nnz_sample += p.nnz
            del p
        per_batch = el * nnz_mine / max(1, nnz_sample)
        cpu = {"value": 1.0 / per_batch, "unit": "epochs/s (whole batch)", "cores": 1, "kind": "oracle",
               "sample": f"1 epoch of serial float64 Sparse SAGA + objective on {len(sample)} of "
                         f"{len(mine)} instances ({el:.1f} s), scaled to the batch by nonzeros"}
    phases["total_s"] = time.perf_counter() - t_all
    if rank == 0:
        paths = {}
        for inf in infos:
            key = f"{inf['row_threshold']}/{inf['row_group']}"
            paths[key] = paths.get(key, 0) + 1
        line = {"metric": "epochs/s", "value": world * args.steps / (ms * 1e-3), "unit": "epochs/s (whole batch)",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 values, f32 state",
                "data": "synthetic", "config": {"workload": BATCH_DESC, "instances_per_rank": len(mine),
                                                "nnz_per_rank": nnz_mine,
                                                "row_paths_threshold_over_group": paths,
                                                "warps_total": int(sum(t["warps"] for t in tune))},
                "instance_epochs_per_s": world * args.steps * len(mine) / (ms * 1e-3),
                "time_to_target": ttt, "one_at_a_time_fp32": single, "phases": phases,
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


def measure(args, name, steps, warmup, e2e_steps, cpu_seconds, env):
    """One configuration at N = world GPUs: autotune, `steps` timed steps, time
    to 1e-6 from x = 0, end to end through the C ABI, CPU baselines.  Returns
    the keys of a bench line (without the process-level ones)."""
    import torch
    from paper_1606_04809_gb300 import asaga

    world, rank, local, stream, barrier, max_over_ranks = env
    wl = WORKLOADS[name]
    p = wl["make"]()
    storage = p.storage if p.storage != "f64" else "f32"
    opts = dict(seed=1000 + rank, abar_recompute_every=ABAR_EVERY, cuda_stream=stream.cuda_stream,
                compact=args.compact)
    ctx = asaga.Context(p, storage=storage, values_dtype=storage if storage != "f16" else "f64", **opts)
    # schedule: warps, step size, block shape and row path picked by the native autotuner
    if args.warps > 0:
        L = asaga.asaga_get_info(ctx.ctx)["L"]
        ctx.close()
        opts.update(max_warps=args.warps, gamma=args.gamma_scale / (3.0 * L))
        ctx = asaga.Context(p, storage=storage, values_dtype=storage if storage != "f16" else "f64", **opts)
        if args.wpb:
            asaga.asaga_set_schedule(ctx.ctx, args.warps, args.gamma_scale / (3.0 * L), args.wpb)
        asaga.asaga_set_draw_ahead(ctx.ctx, args.draw_ahead)
        tune = {"fixed": True, "warps": args.warps, "gamma_scale": args.gamma_scale, "warps_per_block": args.wpb,
                "draw_ahead": args.draw_ahead}
    else:
        t_tune = time.perf_counter()
        tune = asaga.asaga_autotune(ctx.ctx)
        tune["wall_seconds"] = time.perf_counter() - t_tune
    info = asaga.asaga_get_info(ctx.ctx)
    opts.update(max_warps=info["warps"], gamma=info["gamma"])

    for _ in range(warmup):
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
    solver_s, launches, f_last = 0.0, 0, None
    a_bytes = p.nnz * ({"f32": 4, "bf16": 2, "f16": 2}[storage] + (0 if p.dense else 4))
    if a_bytes > L2_BYTES:  # inputs larger than L2: one timed region over all steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s, r = asaga.asaga_run(ctx.ctx, 1)
            solver_s += r.solver_seconds
            launches += r.kernel_launches
            f_last = r.f_last
        e1.record(stream)
        torch.cuda.synchronize()
        ms_local = e0.elapsed_time(e1)
    else:  # inputs that fit in L2: every step timed alone, L2 flushed between steps (outside the events)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        ms_local = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, r = asaga.asaga_run(ctx.ctx, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_local += e0.elapsed_time(e1)
            solver_s += r.solver_seconds
            launches += r.kernel_launches
            f_last = r.f_last
        del flush
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms_local)

    value = world * steps / (ms * 1e-3)
    upd_ms = 1e3 * solver_s / steps
    hbm_bytes = update_hbm_bytes(p, storage, info)
    peak, peak_kind = measured_peak_hbm()
    achieved = hbm_bytes / (upd_ms * 1e-3) / 1e9
    ncu = ncu_summary(f"update_kernel_{name}") or {}
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
            # the timed context itself, reset to x = 0 (it keeps the tuned schedule)
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
    if e2e_steps > 0:
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
        for _ in range(e2e_steps):
            c = asaga.asaga_create(prob, o)
            asaga.asaga_set_schedule(c, info["warps"], info["gamma"], info["warps_per_block"])
            asaga.asaga_set_row_path(c, info["row_threshold"], info["row_group"])
            asaga.asaga_set_draw_ahead(c, info["draw_ahead"])
            asaga.asaga_run(c, 1)
            asaga.load().asaga_get_state(c, xh.data_ptr(), None, None)
            asaga.asaga_destroy(c)
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * e2e_steps / el, "unit": "epochs/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "step": "asaga_create(pinned host CSR) + asaga_run(1 epoch) + asaga_get_state(x) + asaga_destroy"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and cpu_seconds > 0:
        eps, done, el = time_checker(p, cpu_seconds)
        cpu = {"value": eps, "unit": "epochs/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} epochs of serial float64 Sparse SAGA + objective from x=0 ({el:.1f} s)"}
        cpu["asaga_all_cores"] = time_cpu_asaga(p, cpu_seconds * 2, golden["fstar"] if golden else None, TARGET)

    return {
        "metric": "epochs/s", "value": value, "unit": "epochs/s", "steps": steps, "warmup": warmup,
        "ms_per_step": ms / steps,
        "dtype": {"f32": "f32 values, f32 state", "bf16": "bf16 values, f32 state",
                  "f16": "f16 values, f32 state"}[storage],
        "config": static_config(wl, p, storage, args.compact, world),
        "schedule": {"warps": info["warps"], "warps_per_block": info["warps_per_block"], "gamma": info["gamma"],
                     "gamma_over_gamma0": info["gamma"] * 3.0 * info["L"], "L_value": info["L"],
                     "row_path": {"threshold": info["row_threshold"], "group": info["row_group"]},
                     "draw_ahead": info["draw_ahead"],
                     "col_index_bytes": info["col_index_bytes"], "row_values": info["row_values"]},
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


def main():
    args = parse()
    if args.experiment:
        return run_experiment(args)
    if args.workload == "batch":
        return run_batch(args)
    world, rank, local = dist_env()
    if args.impl == "reference":
        wl = WORKLOADS[args.workload]
        return run_reference(args, wl["make"](), wl)

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

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    env = (world, rank, local, stream, barrier, max_over_ranks)
    head = measure(args, args.workload, args.steps, args.warmup, args.e2e_steps, args.cpu_seconds, env)
    # the other single-instance configurations, each with its own line of keys
    others = {}
    for name in [w for w in args.also.split(",") if w and w not in (args.workload, "none")]:
        if name == "batch":
            others[name] = batch_throughput(args, min(args.steps, 10), env)
            continue
        others[name] = measure(args, name, min(args.steps, args.also_steps), args.warmup, min(1, args.e2e_steps),
                               args.cpu_seconds / 2, env)
    if rank == 0:
        line = {"metric": head.pop("metric"), "value": head.pop("value"), "unit": head.pop("unit"),
                "n_gpus": world, "steps": head.pop("steps"), "warmup": head.pop("warmup"),
                "ms_per_step": head.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": head.pop("dtype"), "data": "synthetic"}
        line.update(head)
        line["other_configs"] = others
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
