"""Host checks of the formulas the FP32 kernels use for transcendentals (no GPU).

* erfc: the Chebyshev-exponent form t exp(-y^2 + P(t)), t = 1/(1 + y/2), with the coefficients
  read from the kernel header, against scipy's erfc in FP64: relative error <= 5.5e-8 on [0, 12],
  the bound the header states.
* log1p below 1/2: the atanh series 2 s (1 + s^2/3 + ... + s^8/9), s = y/(2 + y), evaluated step by
  step in float32 as the kernel does (one rounding per operation; the kernel's reciprocal is the
  hardware approximation, emulated here by a correctly rounded one), against log1p in FP64.
  Above 1/2 the kernels take the hardware log2 of 1 + y, which has no host counterpart; the GPU
  vol tests bound the result.
"""
import os
import re

import numpy as np
from scipy.special import erfc

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2408_01470_b300", "csrc", "device_math.cuh")


def _erfc_coefficients():
    src = open(HEADER).read()
    body = src[src.index("constexpr float erfc_fit(int j)"):]
    body = body[: body.index("}")]
    vals = {}
    for m in re.finditer(r"j == (\d) \? ([+-][0-9.]+e[+-]\d+)f", body):
        vals[int(m.group(1))] = float(m.group(2))
    last = re.findall(r":\s+([+-][0-9.]+e[+-]\d+)f;", body)
    vals[9] = float(last[-1])
    assert sorted(vals) == list(range(10))
    return [vals[j] for j in range(10)]


def test_erfc_fit_within_stated_bound():
    c = _erfc_coefficients()
    y = np.linspace(0.0, 12.0, 200001)
    t = 1.0 / (1.0 + 0.5 * y)
    p = np.zeros_like(t)
    for j in range(9, -1, -1):
        p = p * t + c[j]
    approx = t * np.exp(-y * y + p)
    rel = np.abs(approx / erfc(y) - 1.0)
    assert rel.max() <= 5.5e-8, rel.max()
    # the fit is tight: a perturbed leading coefficient breaks the bound
    p2 = p + 1e-6
    assert np.abs(t * np.exp(-y * y + p2) / erfc(y) - 1.0).max() > 5.5e-8


def _log1p_series_f32(y):
    f = np.float32
    y = f(y)
    s = f(y * f(f(1.0) / f(f(2.0) + y)))
    s2 = f(s * s)
    p = f(f(s2 * f(1.0 / 9.0)) + f(1.0 / 7.0))
    p = f(f(s2 * p) + f(1.0 / 5.0))
    p = f(f(s2 * p) + f(1.0 / 3.0))
    p = f(f(s2 * p) + f(1.0))
    return f(f(f(2.0) * s) * p)


def test_log1p_series_branch_float32():
    ys = np.concatenate([np.geomspace(1e-8, 0.5, 20000, endpoint=False), [0.4999999]])
    got = np.array([_log1p_series_f32(v) for v in ys], dtype=np.float64)
    ref = np.log1p(ys.astype(np.float32).astype(np.float64))
    rel = np.abs(got / ref - 1.0)
    assert rel.max() <= 4e-7, rel.max()
    # the truncation of the series alone (in FP64) stays below 1e-8 relative up to y = 1/2 (the first
    # omitted term is s^10 / 11 <= 0.2^10 / 11 = 9.3e-9)
    s = ys / (2.0 + ys)
    s2 = s * s
    ser = 2.0 * s * (1.0 + s2 / 3.0 + s2 ** 2 / 5.0 + s2 ** 3 / 7.0 + s2 ** 4 / 9.0)
    assert np.abs(ser / np.log1p(ys) - 1.0).max() <= 1e-8
