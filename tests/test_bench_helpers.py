"""Host logic of bench.py that needs no GPU: a counter recorded in a committed
ncu summary is used only while the kernel source still has the hash recorded
with it, and the rate and time reductions over ranks."""
import hashlib

import bench


def _setup(tmp_path, text):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "summary.md").write_text(text.format(sha=sha))
    return src


def test_counter_read_while_the_source_is_unchanged(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _setup(tmp_path, "k.cu sha256 (first 16 hex): {sha}\ndram_bytes_per_launch: 123\n"
                     "l1tex_wavefronts_per_launch: 456\n")
    assert bench.captured_counter("kernel.cu", "summary.md") == 123
    assert bench.captured_counter("kernel.cu", "summary.md", "l1tex_wavefronts_per_launch") == 456
    assert bench.captured_counter("kernel.cu", "summary.md", "absent_key") is None


def test_counter_dropped_once_the_source_changes(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = _setup(tmp_path, "k.cu sha256 (first 16 hex): {sha}\ndram_bytes_per_launch: 123\n")
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.captured_counter("kernel.cu", "summary.md") is None


def test_counter_without_summary_or_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _setup(tmp_path, "dram_bytes_per_launch: 123\n")  # no hash line
    assert bench.captured_counter("kernel.cu", "summary.md") is None
    assert bench.captured_counter("kernel.cu", "missing.md") is None


def test_single_rank_reductions():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.sum_over_ranks(7, 1) == 7
    assert bench.whole_job_rate(100, 2.0, 1) == 50.0
