"""Host logic of bench.py that needs no GPU: the kernel-source hash that
decides whether the committed ncu traffic still describes the kernels
(comments and whitespace do not change it, code does), and the lookup
that returns no traffic when the hash differs."""
import json
import os

import bench


def _write(root, name, text):
    d = os.path.join(root, "paper_2010_11847_gb300", "csrc")
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, name), "w") as f:
        f.write(text)


def test_source_hash_ignores_comments_and_whitespace_but_not_code(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path, "k.cu", "int f(int a) {\n  return a + 1;  // one\n}\n")
    h0 = bench.kernel_source_hash(["k.cu"])
    _write(tmp_path, "k.cu", "/* header */\nint f(int a) {\n\n    return a + 1;   // plus one\n}\n")
    assert bench.kernel_source_hash(["k.cu"]) == h0
    _write(tmp_path, "k.cu", "int f(int a) {\n  return a + 2;\n}\n")
    assert bench.kernel_source_hash(["k.cu"]) != h0


def test_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path, "k.cu", "int f(int a) { return a; }\n")
    os.makedirs(tmp_path / "profiles")
    entry = {"files": ["k.cu"], "source_hash": bench.kernel_source_hash(["k.cu"]),
             "dram_bytes_per_launch_full_size": 123.0}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"kernels": {"cls": entry}}))
    assert bench.ncu_traffic("cls") == 123.0
    assert bench.ncu_traffic("other") is None
    _write(tmp_path, "k.cu", "int f(int a) { return -a; }\n")
    assert bench.ncu_traffic("cls") is None


def test_committed_traffic_matches_the_current_readout_sources():
    """The committed capture was taken on the readout's current code."""
    assert bench.ncu_traffic("kdk_readout_kick_drift") is not None


def test_roofline_bytes_follow_the_method_minimum():
    """The readout's roofline numerator is the method's 48 B/particle + 12
    B/cell (keys and the float4 padding are build overhead, reported apart);
    the PM step is 60 B/particle + 44 B/cell, the adjoint run 3x that."""
    N = M = 512 ** 3
    assert bench._alg_bytes("kdk_readout_kick_drift", N, M, 512) == 60.0 * N
    assert bench._build_bytes("kdk_readout_kick_drift", N, M, 512) == 68.0 * N
    assert bench.step_algorithmic_bytes(N, M) == 104.0 * N
    assert bench.adjoint_algorithmic_bytes(N, M, 40) == 3 * 104.0 * N * 40
    N2, M2 = 128 ** 3, 256 ** 3
    assert bench._alg_bytes("kdk_readout_kick_drift", N2, M2, 256) == 48.0 * N2 + 12.0 * M2
