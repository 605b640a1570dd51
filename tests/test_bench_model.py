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
    per_launch = 1000 * (2 * 128 + 4 * 64)          # candidates per launch x (BF16 row + list)
    assert out["algorithmic_bytes"] == per_launch
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
