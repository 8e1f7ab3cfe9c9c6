"""The measurement helpers of bench.py, on CPU: the algorithmic byte count
behind roofline.achieved, the committed ncu summaries behind roofline.traffic,
and the bounded-sample arithmetic of the CPU reference arm."""
import hashlib
import json
import os

import numpy as np

import bench
from paper_1606_04809_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_count_each_entry_and_row_once():
    p = synth.small_logistic()
    # per entry: a 4-byte column index and the value; per row: two row_ptr
    # entries, the label and alpha read + write
    assert bench.update_hbm_bytes(p, "f32") == p.nnz * (4 + 4) + p.n * (16 + 4 + 8)
    assert bench.update_hbm_bytes(p, "bf16") == p.nnz * (4 + 2) + p.n * (16 + 4 + 8)
    # compact layout: 2-byte indices and one float32 value per row
    info = {"col_index_bytes": 2, "row_values": 1}
    assert bench.update_hbm_bytes(p, "bf16", info) == p.nnz * 2 + p.n * (16 + 4 + 8 + 4)


def test_dense_rows_have_no_indices_and_no_row_ptr():
    p = synth.covtype_like(n=1000)
    assert bench.update_hbm_bytes(p, "f16") == p.nnz * 2 + p.n * (4 + 8)


def test_a_profile_counts_only_for_the_kernel_source_it_was_captured_on(tmp_path, monkeypatch):
    """roofline.traffic comes from the machine-readable file beside a committed
    ncu summary only while update.cu is the source it records; after any
    change the bench reports null."""
    csrc = tmp_path / "paper_1606_04809_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "update.cu"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "update_kernel_toy.json").write_text(json.dumps(
        {"update_cu_sha256": sha, "traffic_bytes_per_launch": 123456, "l2_throughput_pct_of_peak": 11.5,
         "dram_throughput_pct_of_peak": 1.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    s = bench.ncu_summary("update_kernel_toy")
    assert s == {"traffic": 123456, "l2_pct": 11.5, "dram_pct": 1.5}
    src.write_text("// kernel v2\n")
    assert bench.ncu_summary("update_kernel_toy") is None
    assert bench.ncu_summary("missing") is None


def test_committed_profiles_have_a_readable_figure_file():
    """Every ncu summary the bench reads has its figures in a JSON file beside
    it; the Markdown stays prose and gives the command."""
    for name in ("update_kernel_rcv1like", "update_kernel_urllike", "batch_update_kernel_batch256"):
        text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
        assert "ncu " in text
        kv = json.load(open(os.path.join(ROOT, "profiles", name + ".json")))
        assert len(kv["update_cu_sha256"]) == 64 and int(kv["traffic_bytes_per_launch"]) > 0


def test_reference_steps_are_bounded_samples_reported_in_epochs():
    p = synth.small_logistic()
    per = bench.REFERENCE_STEPS_PER_EPOCH
    eps, done, el = bench.time_checker(p, 0.0, steps=2 * per, warmup=3, per_epoch=per)
    assert done == 2 * per and el > 0
    # 2 * per steps of ceil(n / per) updates each = about two epochs
    count = -(-p.n // per)
    assert np.isclose(eps, done * count / p.n / el)
    assert 1.9 < done * count / p.n < 2.2
