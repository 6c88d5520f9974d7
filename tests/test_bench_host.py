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


def test_byte_models_and_roofline_arithmetic(monkeypatch):
    """Per-launch algorithmic bytes of the vertex-cover split form (20N + 8E
    direction, 12E + 4N SpMV, 8E per candidate pass, 12E + 16N update) and the
    roofline fields computed from per-class event times."""
    N, E = 1000, 16000
    ab = bench.algorithmic_bytes("vcover", N, E)
    assert ab == {"dir": 20 * N + 8 * E, "spmv": 12 * E + 4 * N, "cand": 8 * E, "update": 12 * E + 16 * N}
    monkeypatch.setattr(bench, "measured_peaks", lambda: (1000.0, "measured"))
    tim = {"dir_ms": 1.0, "spmv_ms": 1.0, "cand_ms": 4.0, "update_ms": 1.0, "iters": 10, "cand_passes": 40}
    r = bench.roofline(ab, tim, "none")
    assert r["class"] == "cand"
    assert abs(r["avg_launch_ms"] - 0.1) < 1e-12
    assert abs(r["achieved"] - 8 * E / 1e-4 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["traffic"] is None


def test_oracle_slices_are_disjoint_blocks_of_the_same_graph():
    from graphgen import workloads as W
    wl = W.vcover(12, seed=5)
    jobs, how = bench.oracle_jobs("vcover-rmat24", wl, 3, 0.1, "newton")
    assert len(jobs) == 3 and "whole workload" in how     # small graph: every process runs all of it
    lp, n, u, v, extra, seconds, step, warmup, iters = jobs[0]
    assert lp == "vcover" and u.size == wl.graph.m and n == wl.graph.n
    e, it, dt = bench.oracle_worker((lp, n, u, v, extra, 0.0, "newton", 1, 2))
    assert e == wl.graph.m and it == 2 and dt >= 0.0
