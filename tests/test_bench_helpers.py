"""Host-side helpers of bench.py: the roofline arithmetic and the lookup of
recorded DRAM traffic (no GPU)."""
import hashlib
import importlib.util
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_root(tmp_path, rows):
    src = tmp_path / "paper_2603_04035_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "epoch.cu").write_text("// epoch source\n")
    (src / "knn_tc.cu").write_text("// knn source\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    lines = ["| kernel | workload | dram bytes per launch | source sha256[:12] | note |", "|---|---|---|---|---|"]
    lines += [f"| {k} | {w} | {b} | {s} | x |" for k, w, b, s in rows]
    (prof / "ncu_traffic.md").write_text("\n".join(lines) + "\n")
    return tmp_path


def test_traffic_needs_same_kernel_workload_and_source(bench, tmp_path, monkeypatch):
    sha = hashlib.sha256(b"// epoch source\n").hexdigest()[:12]
    root = _fake_root(tmp_path, [("epoch_force_kernel", "70k", "1000", sha),
                                 ("epoch_force_kernel", "10m", "5000", "0" * 12)])
    monkeypatch.setattr(bench, "ROOT", str(root))
    rel = "paper_2603_04035_gb300/csrc/epoch.cu"
    assert bench.kernel_traffic("epoch_force_kernel", rel, "70k") == 1000.0
    assert bench.kernel_traffic("epoch_force_kernel", rel, "10m") is None      # stale source
    assert bench.kernel_traffic("epoch_force_kernel", rel, "batched") is None  # no capture of it
    assert bench.kernel_traffic("knn_tc_kernel", rel, "70k") is None           # other kernel
    (root / rel).write_text("// changed\n")
    assert bench.kernel_traffic("epoch_force_kernel", rel, "70k") is None      # source changed


def test_roofline_epoch_arithmetic(bench, monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda *a: None)
    args = types.SimpleNamespace(workload="70k")
    n, nnz, T = 1000, 30000, 100
    updates = 1_000_000.0                          # 10,000 active entries per epoch
    stage = {"epochs": 2.0, "knn": 0.5}            # ms over 2 steps: 10 us per epoch
    r = bench.roofline(args, n, 50, nnz, updates, stage, 2, {"hbm_gbs": 1000.0}, "measured", T)
    bytes_ep = 4 * (n + 1) + 16 * n + 8 * nnz + 8 * 10_000 * (1 + bench.NEG)
    assert r["kernel"] == "epoch_force_kernel" and r["bound"] == "hbm"
    assert r["bytes_per_launch"] == pytest.approx(bytes_ep)
    assert r["launch_ms"] == pytest.approx(0.01)
    assert r["achieved"] == pytest.approx(bytes_ep / 10e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)


def test_roofline_knn_gemm_arithmetic(bench, monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda *a: None)
    args = types.SimpleNamespace(workload="10m")
    stage = {"epochs": 1.0, "knn": 4.0, "knn_gemm": 3.0}   # ms over one step
    peaks = {"hbm_gbs": 1.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1500.0}
    r = bench.roofline(args, 10_000, 50, 0, 0.0, stage, 1, peaks, "measured", 200, tiles_done=1000)
    flops = 2.0 * 1000 * 128 * 256 * 50
    assert r["kernel"] == "knn_tc_kernel" and r["bound"] == "tensor"
    assert r["peak"] == 1500.0                       # the sustained figure inside a long step
    assert r["achieved"] == pytest.approx(flops / 3e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1500.0)
