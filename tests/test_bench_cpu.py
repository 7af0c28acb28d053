"""bench.py's roofline choice (host logic, no GPU): a kernel class is reported against
the resource that caps it at its own arithmetic intensity."""
import importlib.util
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


PEAKS = {"bf16_tflops": 1920.0, "hbm_gbs": 6800.0}


def _rec(tflops, gbs, ms=1000.0, launches=10):
    return {"launches": launches, "ms": ms, "flops": tflops * 1e12 * ms * 1e-3, "bytes": gbs * 1e9 * ms * 1e-3}


def test_low_intensity_tensor_class_is_hbm_bound():
    b = _bench()
    r = b.roofline_of("sandwich", _rec(24.0, 830.0), "tf32x3", PEAKS)      # ~29 flop/byte < ridge ~46
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 830.0) < 1e-6 and abs(r["frac"] - 830.0 / 6800.0) < 1e-12
    assert r["traffic"] is not None


def test_high_intensity_gemm_is_tensor_bound():
    b = _bench()
    r = b.roofline_of("gemm_tc_tf32x3", _rec(200.0, 900.0), "tf32x3", PEAKS)   # ~222 flop/byte
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["peak"] - 1920.0 * 1.1 / 2.25) < 1e-9


def test_fp32_sandwich_and_streaming_classes():
    b = _bench()
    assert b.roofline_of("sandwich", _rec(4.0, 140.0), "f32", PEAKS)["bound"] == "alu"
    r = b.roofline_of("sketch", _rec(0.0, 34.0), "tf32x3", PEAKS)
    assert r["bound"] == "hbm" and r["peak"] == 6800.0
