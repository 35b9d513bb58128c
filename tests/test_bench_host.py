"""Host logic of bench.py that needs no GPU: the algorithmic bytes model
behind roofline.achieved, and the DRAM-traffic record, which is reported
only while the solver source it was measured on is unchanged."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_bytes_model_counts_vectors_faces_and_replacements():
    # per iteration: 52 B of FP32 vectors per cell plus 12 B per face (index
    # pair + FP32 coefficient); per FP64 residual replacement (the first one,
    # which builds r from x0, included): 24 B per cell plus 16 B per face
    n, F = 1000, 2000
    assert bench._bytes_model(n, F, 0, 0) == 0.0
    assert bench._bytes_model(n, F, 1, 0) == 52 * n + 12 * F
    assert bench._bytes_model(n, F, 0, 1) == 24 * n + 16 * F
    assert bench._bytes_model(n, F, 10, 3) == 10 * (52 * n + 12 * F) + 3 * (24 * n + 16 * F)


def _fake_tree(tmp_path, source: bytes, records: dict):
    csrc = tmp_path / "paper_1804_01130_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gfm_solve.cu").write_bytes(source)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(records))


def test_traffic_record_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    source = b"// solver source as measured\n"
    sha = hashlib.sha256(source).hexdigest()[:16]
    _fake_tree(tmp_path, source, {
        "tank2d": {"source_sha": sha, "kernel": "void k_solve_fused<4, 0>(SolveArgs)", "dram_bytes_per_launch": 1.0e8},
        "box3d": {"source_sha": "0" * 16, "kernel": "void k_solve_mixed<6, 1, 0>(SolveArgs)",
                  "dram_bytes_per_launch": 4.0e11},
    })
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec, got = bench._traffic_record("tank2d", "k_solve_fused")
    assert got == sha and rec["dram_bytes_per_launch"] == 1.0e8
    # a capture of another kernel (the other iteration form): not reported
    rec, _ = bench._traffic_record("tank2d", "k_solve_mixed")
    assert rec is None
    # measured on another source: not reported
    rec, _ = bench._traffic_record("box3d", "k_solve_mixed")
    assert rec is None
    # no record at all
    rec, _ = bench._traffic_record("batch64", "k_solve_batched")
    assert rec is None
    # the source changes after the capture: the record stops counting
    (tmp_path / "paper_1804_01130_gb300" / "csrc" / "gfm_solve.cu").write_bytes(source + b"// edited\n")
    rec, _ = bench._traffic_record("tank2d", "k_solve_fused")
    assert rec is None


def test_committed_traffic_records_name_their_kernels():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        recs = json.load(fh)
    for workload, kernels in (("tank2d", ("k_solve_mixed", "k_solve_fused")), ("box3d", ("k_solve_mixed", "k_solve_fused")),
                              ("batch64", ("k_solve_batched",))):
        r = recs[workload]
        assert any(k in r["kernel"] for k in kernels) and r["dram_bytes_per_launch"] > 0 and len(r["source_sha"]) == 16
