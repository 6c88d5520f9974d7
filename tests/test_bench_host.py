"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports is
read from a committed ncu summary only while the kernel source still has the
hash the summary names."""
import hashlib

import bench


def _tree(tmp_path, kernel_src, sha):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2307_03307_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2307_03307_gb300" / "csrc" / "mwu_kernels.cu").write_text(kernel_src)
    (tmp_path / "profiles" / "traffic_w.md").write_text(
        f"kernels_sha256_16: {sha}\n\n| class | kernel | dram_bytes_per_launch |\n|---|---|---|\n"
        "| cand | k_cand_newton | 12345 |\n| dir | k_dir_pairs | 678 |\n")


def test_traffic_read_while_the_kernels_match(tmp_path, monkeypatch):
    src = "// kernels\n"
    _tree(tmp_path, src, hashlib.sha256(src.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("w", "cand") == 12345
    assert bench.profiled_traffic("w", "dir") == 678
    assert bench.profiled_traffic("w", "update") is None
    assert bench.profiled_traffic("other", "cand") is None


def test_traffic_null_once_the_kernels_change(tmp_path, monkeypatch):
    _tree(tmp_path, "// changed kernels\n", hashlib.sha256(b"// kernels\n").hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("w", "cand") is None
