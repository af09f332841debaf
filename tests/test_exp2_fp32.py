"""The FP32 2^(x + j) of the stage kernels (exp2_fp32, the integer j carried in its rounding constant):
its coefficients are the committed fit, and the algorithm, emulated step by step in FP32 on the CPU
(each fused multiply-add as an exact FP64 product and sum rounded once to FP32), has a relative error
below 8e-8 whose mean over unit intervals is below 2e-9. A biased 2^x drifts the moments by dt/tau
times its mean error at every relaxation."""
import os
import re

import numpy as np

from paper_2308_06196_gb300 import exp2_fit

f32 = np.float32
SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2308_06196_gb300", "csrc", "stage_common.cuh")


def kernel_coefficients():
    s = open(SRC).read()
    body = s[s.index("float exp2_fp32(float x, float kmagic)"):]
    body = body[:body.index("return")]
    first = float(re.search(r"float p = ([0-9.e+-]+)f;", body).group(1))
    rest = [float(v) for v in re.findall(r"p = fmaf\(p, r, ([0-9.e+-]+)f\);", body)]
    return np.array(([first] + rest)[::-1], dtype=np.float32)  # c0 .. c6


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def exp2_emulated(x, c, j=0):
    magic = f32(12582912.0 + j)
    x = np.maximum(x.astype(f32), f32(-100.0))
    t = (x + magic).astype(f32)
    r = (x - (t - magic).astype(f32)).astype(f32)
    p = np.full_like(r, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = fma32(p, r, np.full_like(r, c[k]))
    bits = p.view(np.int32).astype(np.int64) + (t.view(np.int32).astype(np.int64) << 23)
    return (bits & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def pair_coefficients():
    """The coefficients of the packed-pair version (exp2_fp32x2), in the same order (c0 .. c6)."""
    s = open(SRC).read()
    body = s[s.index("void exp2_fp32x2("):]
    body = body[:body.index("unpack2(pp")]
    vals = re.findall(r"pack2\(([0-9.e+-]+)f, ([0-9.e+-]+)f\)", body)
    assert all(a == b for a, b in vals)
    return np.array([float(a) for a, _ in vals][::-1], dtype=np.float32)


def test_coefficients_are_the_fit():
    assert np.array_equal(kernel_coefficients(), exp2_fit.coefficients())
    assert np.array_equal(pair_coefficients(), exp2_fit.coefficients())


def test_error_and_mean_error():
    c = kernel_coefficients()
    for lo, j in ((-20.0, 0), (-9.0, 3), (-4.0, -7), (-1.0, 20), (0.0, -20), (3.0, 0)):
        x = (lo + (np.arange(1 << 20) + 0.5) / (1 << 20)).astype(f32)
        y = exp2_emulated(x, c, j).astype(np.float64)
        e = y / np.exp2(x.astype(np.float64) + j) - 1.0
        assert np.abs(e).max() < 8e-8, lo
        assert abs(e.mean()) < 2e-9, lo


def test_integer_and_clamped_inputs():
    c = kernel_coefficients()
    n = np.arange(-100, 100).astype(f32)
    for j in (-20, 0, 20):
        assert np.array_equal(exp2_emulated(n, c, j), np.exp2(n.astype(np.float64) + j).astype(f32))
    assert exp2_emulated(np.array([-400.0], dtype=f32), c, -20)[0] == f32(2.0**-120)
