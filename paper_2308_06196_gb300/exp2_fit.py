"""Coefficients of the FP32 2^r polynomial on [-1/2, 1/2] used by the stage kernels (exp2_fp32 in
csrc/stage_common.cuh): a degree-6 fit of 2^r by least squares with relative-error weighting on 4000
Chebyshev nodes, in FP64, then rounded to FP32. Run as a script to print them."""
import numpy as np

DEGREE = 6


def coefficients(degree: int = DEGREE) -> np.ndarray:
    t = 0.5 * np.cos(np.pi * (np.arange(4000) + 0.5) / 4000)
    A = np.vander(t, degree + 1, increasing=True)
    wgt = 1.0 / np.exp2(t)
    c, *_ = np.linalg.lstsq(A * wgt[:, None], np.exp2(t) * wgt, rcond=None)
    return c.astype(np.float32)


if __name__ == "__main__":
    for k, c in enumerate(coefficients()):
        print(f"c{k} = {c:.9e}f")
