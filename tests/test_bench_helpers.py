"""Host-side arithmetic of bench.py: captured DRAM traffic is reported only for
the kernel source and the workload (xi, M) it was captured at; the per-kernel
roofline divides algorithmic bytes by the live per-launch time."""
import hashlib
import os

import pytest

import bench


def test_captured_traffic_needs_the_same_source_and_workload(monkeypatch):
    src = os.path.join(os.path.dirname(bench.__file__), "paper_1611_09322_gb300", "csrc", "kernels_real.cu")
    with open(src, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    monkeypatch.setattr(bench, "TRAFFIC", {"k": (123, ("csrc/kernels_real.cu",), digest, (0.5, 256))})
    assert bench.captured_traffic("k", 0.5, 256) == 123
    assert bench.captured_traffic("k", 0.51, 256) is None      # another splitting
    assert bench.captured_traffic("k", 0.5, 250) is None       # another grid
    assert bench.captured_traffic("other", 0.5, 256) is None   # never captured
    monkeypatch.setattr(bench, "TRAFFIC", {"k": (123, ("csrc/kernels_real.cu",), "0" * 64, (0.5, 256))})
    assert bench.captured_traffic("k", 0.5, 256) is None       # source changed since the capture


def test_kernel_roofline_arithmetic():
    N, M, n_pairs, peak = 1000, 16, 5000, 1000.0
    stages = {"matvec": (0.004, 4), "neighbours": (0.002, 1), "lanczos_update": (0.0, 4),
              "interp": (0.001, 1), "grid_copy": (0.0005, 1), "wave_noise": (0.001, 0)}
    r = bench.kernel_roofline(stages, N, M, n_pairs, peak)
    mv = 16 * N + 12 * N + 12 * N + 4 * n_pairs  # positions, input, output, list (the minimum the method moves)
    assert r["k_lz_matvec"]["algorithmic_bytes"] == mv
    assert r["k_lz_matvec"]["achieved_gbs"] == pytest.approx(mv / 1e-6 / 1e9, rel=1e-3)
    assert r["k_interp4"]["algorithmic_bytes"] == 32 * N + 16 * M ** 3
    assert r["k_grid_aos"]["frac"] == pytest.approx(28 * M ** 3 / 5e-7 / 1e9 / peak, rel=1e-3)
    assert "k_lz_update" not in r and "k_wave_noise" not in r  # no time or no launch: no entry
    assert bench.kernel_roofline(stages, N, M, n_pairs, peak, "k_interp")["k_interp"]["algorithmic_bytes"] == \
        32 * N + 12 * M ** 3
