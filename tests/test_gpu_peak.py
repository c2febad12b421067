"""FP32 roofline denominator: the derived peak (152 SMs x 128 FP32 lanes x 2
flops x 2.07 GHz = 80.5 TFLOP/s) against a measured FFMA loop (a burst and
1000 launches back to back), and the packed FFMA2 form, which halves the
instruction count but not the flop rate (so the denominator is the same for
the packed rollout kernel).  The XU (special-function unit) rate on
reciprocal square roots is measured and printed (the secondary bound)."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DERIVED_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def test_fp32_peak_probe():
    exe = os.path.join(HERE, "cuda", "_build", "fp32_peak_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "cuda", "fp32_peak_probe.cu")])
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    r = json.loads(out.strip().splitlines()[-1])
    print("FP32 probe:", r, "derived peak %.1f TFLOP/s" % DERIVED_TFLOPS)
    assert r["status"] == "no error"
    # a measured FFMA loop reaches most of the derived peak and never exceeds it by much
    assert 0.7 * DERIVED_TFLOPS <= r["ffma_tflops"] <= 1.05 * DERIVED_TFLOPS
    # packing two FMAs per instruction does not double the FP32 rate
    assert r["ffma2_tflops"] <= 1.1 * r["ffma_tflops"]
    # sustained over 1000 launches (a quarter second): the clock may settle lower
    assert 0.5 * DERIVED_TFLOPS <= r["ffma_sustained_tflops"] <= 1.05 * DERIVED_TFLOPS
    # XU: far below the FP32 lane rate (a few operations per SM per clock)
    assert 0.0 < r["xu_rsqrt_per_s"] < 0.5 * DERIVED_TFLOPS * 1e12 / 2
