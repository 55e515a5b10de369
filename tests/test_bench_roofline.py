"""Host logic of bench.py's roofline record: the binding-roof fraction, the per-kernel and
per-product tables built from kernel times, and the DRAM traffic that is reported only while the
ncu summary matches the kernel sources it was taken on."""
import hashlib

import pytest

import bench


def test_binding_roof_takes_the_slower_roof():
    # 1 GB at 1000 GB/s = 1 ms, 2 TFLOP at 1 TFLOP/s = 2 s -> ALU bound
    bound, frac, hbm, alu = bench.binding_roof(1e9, 2e12, 4.0, 1000.0, 1.0)
    assert bound == "alu"
    assert frac == pytest.approx(0.5) and alu == pytest.approx(0.5)
    assert hbm == pytest.approx(0.25e-3)
    bound, frac, hbm, alu = bench.binding_roof(8e9, 1e9, 0.01, 1000.0, 1.0)
    assert bound == "hbm" and frac == pytest.approx(0.8) and alu == pytest.approx(0.1)


def _info():
    return {"kernel_bytes_fp64": [100e6, 200e6], "kernel_bytes_fp32": [50e6, 40e6],
            "kernel_flops": [1e9, 2e9], "kernel_flops_built": [0.5e9, 0.25e9],
            "kernel_flops_built_fp32": [0.6e9, 0.4e9]}


def test_roofline_figures_per_kernel_and_product(monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda name: 123.0 if name == "struct_kernel_fp64" else None)
    # (precision, kernel, direction) -> (total ms, launches)
    kt = {("fp64", "struct", "vmult"): (4.0, 8), ("fp64", "cut", "vmult"): (2.4, 8),
          ("fp32", "struct", "vmult"): (0.32, 8), ("fp32", "cut", "vmult"): (0.56, 8)}
    table, products, roof = bench.roofline_figures(_info(), kt, 5000.0, 5e6)
    s = table["struct_kernel_fp64"]
    assert s["avg_ms"] == pytest.approx(0.5)
    assert s["pipe_frac"] == pytest.approx(0.5e9 / 0.5e-3 / 1e12 / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert s["hbm_frac"] == pytest.approx(100e6 / 0.5e-3 / 5000e9, rel=1e-3)
    assert s["roof_frac"] == pytest.approx(max(s["pipe_frac"], s["hbm_frac"]), rel=1e-3)
    # a product sums its kernels' times, bytes and operations
    p = products["fp64_vmult"]
    assert p["ms"] == pytest.approx(0.8)
    assert p["gdofs"] == pytest.approx(5e6 / 0.8e-3 / 1e9, rel=1e-3)
    t_alu = 0.75e9 / (bench.FP64_PEAK_TFLOPS * 1e12)
    assert p["pipe_frac"] == pytest.approx(t_alu / 0.8e-3, rel=1e-3)
    # the roofline object describes the kernel with the largest total time
    assert roof["kernel"] == "struct_kernel_fp64" and roof["bound"] == "alu"
    assert roof["traffic"] == 123.0 and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(s["roof_frac"], rel=1e-3)


def test_traffic_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cuh"
    src.write_text("// kernel source\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    rec = tmp_path / "traffic.txt"
    rec.write_text(f"# comment line\nsource_sha256_16 {digest}\ncut_kernel_fp64 314930176\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [str(src)])
    monkeypatch.setattr(bench, "TRAFFIC", str(rec))
    assert bench.kernel_traffic("cut_kernel_fp64") == 314930176.0
    assert bench.kernel_traffic("struct_kernel_fp64") is None
    src.write_text("// kernel source, changed\n")
    assert bench.kernel_traffic("cut_kernel_fp64") is None
