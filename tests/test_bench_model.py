"""bench.py's roofline arithmetic and the keying of the committed DRAM-traffic figures (CPU)."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_join_roofline_arithmetic():
    import bench
    w = types.SimpleNamespace(N=1000, d=128, k=64, M=32, R=32, h=4)
    stats = {"join_cands": 2000, "join_pairs": 10_000}
    out = bench.roofline_for("k_join", 10.0, 2, w, [], None, {"hbm_gbs": 1000.0, "bf16_tflops_sustained": 100.0},
                             stats, 1)
    per_launch = 1000 * (1 * 128 + 4 * 64)          # candidates per launch x (byte row + list)
    assert out["algorithmic_bytes"] == per_launch
    out4 = bench.roofline_for("k_join", 10.0, 2, w, [], None, {"hbm_gbs": 1000.0}, stats, 4)
    assert out4["algorithmic_bytes"] == 1000 * (4 * 128 + 4 * 64)   # FP32 rows
    assert out["achieved"] == pytest.approx(per_launch / 0.01 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 1000.0)
    assert out["algorithmic_flops"] == 5000 * 2 * 128
    assert out["traffic"] is None                    # not the captured workload size


def test_traffic_figures_follow_the_kernel_sources(monkeypatch):
    import bench
    live = bench.measured_traffic()
    assert set(live) <= set(bench.TRAFFIC_SOURCES)
    # a family whose sources changed since the capture loses its figure, the others keep theirs
    real = bench.kernel_sources_sha256
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda k: "changed" if k == "k_join" else real(k))
    stale = bench.measured_traffic()
    assert "k_join" not in stale
    assert {k: v for k, v in live.items() if k != "k_join"} == stale


def test_row_bytes():
    """One byte per coordinate exactly when byte rows apply: integers in [0, 255], d <= 128,
    d % 16 == 0."""
    import bench
    row = np.arange(16, dtype=np.float32) * 17            # 0 .. 255
    assert bench.row_bytes(types.SimpleNamespace(X=row[None], d=16)) == 1
    assert bench.row_bytes(types.SimpleNamespace(X=(row + 0.5)[None], d=16)) == 4   # not integers
    assert bench.row_bytes(types.SimpleNamespace(X=(row + 1)[None], d=16)) == 4     # 256 out of range
    assert bench.row_bytes(types.SimpleNamespace(X=row[None, :12], d=12)) == 4      # d % 16 != 0


def test_update_launches_fold_into_one_family():
    """The Update's tile and warp-per-vertex launches are one roofline family: times and launch
    counts add, the other kernels pass through."""
    import bench
    k = {"k_join": {"launches": 4, "ms": 40.0}, "k_join_sparse": {"launches": 2, "ms": 10.0},
         "k_prune": {"launches": 1, "ms": 5.0}}
    f = bench.roofline_kernels(k)
    assert f == {"k_join": {"launches": 6, "ms": 50.0}, "k_prune": {"launches": 1, "ms": 5.0}}
    assert bench.roofline_kernels({"k_join_sparse": {"launches": 2, "ms": 3.0}}) == {
        "k_join": {"launches": 2, "ms": 3.0}}


def test_source_hash_ignores_comments_only():
    """The traffic figures are keyed by the kernels' code: comments and blank lines do not change
    the hash, any code change does, and literals containing comment markers are kept."""
    import bench
    a = 'int f(int x) { return x + 1; }  // one\n/* two\n lines */\nconst char* s = "a//b/*c*/";\n'
    b = '// header\nint f(int x) { return x + 1; }\n\nconst char* s = "a//b/*c*/";  /* tail */\n'
    c = 'int f(int x) { return x + 2; }\nconst char* s = "a//b/*c*/";\n'
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)
    assert '"a//b/*c*/"' in bench.strip_comments(a)
