"""Host checks of the formulas the FP32 kernels use for transcendentals (no GPU).

* erfc: the Chebyshev-exponent form t exp(-y^2 + P(t)), t = 1/(1 + y/2), with the coefficients
  read from the kernel header, against scipy's erfc in FP64: relative error <= 5.5e-8 on [0, 12],
  the bound the header states.
* the packed normal CDF: the same fit rearranged (u = 1/(2 + y), coefficients 2^j c_j log2 e, the
  exponent in base 2), evaluated step by step in float32 as the kernel does, against 0.5 erfc in
  FP64: the rearrangement adds no error over the fit beyond the float32 roundings of the exponent.
  For x <= 0 these are also the steps of the select-free form the caplet pricer takes for the
  far-side Black argument (the same operations on -x, bit for bit).
* log1p below 1/2: the atanh series 2 s (1 + s^2/3 + ... + s^8/9), s = y/(2 + y), with the factor 2
  on the coefficients, evaluated step by step in float32 as the kernel does (one rounding per
  operation), against log1p in FP64.
In both the kernel's hardware approximations (reciprocal, 2^x) are emulated by correctly rounded
ones.
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


def _fma32(a, b, c):
    # float32 fused multiply-add: the product of two float32 values is exact in FP64
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _ncdf_pair_form_f32(x):
    f = np.float32
    c = _erfc_coefficients()
    d = [f(float(f(c[j])) * (1 << j) * 1.44269504088896341) for j in range(10)]
    ax = f(abs(f(x)))
    u = f(1.0 / np.float64(_fma32(ax, f(0.70710678), f(2.0))))
    p = d[9]
    for j in range(8, -1, -1):
        p = _fma32(p, u, d[j])
    m = f(ax * f(-0.721347520444481703))
    h = f(u * f(2.0 ** np.float64(_fma32(m, ax, p))))
    return h if x < 0 else f(f(1.0) - h)


def test_ncdf_pair_form_float32():
    xs = np.linspace(-12.0, 0.0, 24001)
    got = np.array([_ncdf_pair_form_f32(v) for v in xs], dtype=np.float64)
    ref = 0.5 * erfc(-xs.astype(np.float32).astype(np.float64) / np.sqrt(2.0))
    rel = np.abs(got / ref - 1.0)
    # near the centre the fit and a few float32 roundings; far out the two roundings of the base-2
    # exponent a = -x^2 log2(e) / 2 dominate (m, then the fma), each <= 2^-24 |a| absolute, i.e.
    # 2^-24 |a| ln 2 = 2^-24 x^2 / 2 relative in 2^a
    assert rel[xs > -1.0].max() <= 4e-7, rel[xs > -1.0].max()
    bound = 4e-7 + xs ** 2 * 2.0 ** -24
    assert np.all(rel <= bound), (rel / bound).max()
    # the upper half is 1 - Phi(-x) to float32 rounding
    for v in (0.1, 0.7, 1.5, 3.0):
        assert abs(float(_ncdf_pair_form_f32(v)) - (1.0 - 0.5 * erfc(v / np.sqrt(2.0)))) <= 1.2e-7


def _log1p_series_f32(y):
    f = np.float32
    y = f(y)
    s = f(y * f(f(1.0) / f(f(2.0) + y)))
    s2 = f(s * s)
    p = f(f(s2 * f(2.0 / 9.0)) + f(2.0 / 7.0))
    p = f(f(s2 * p) + f(2.0 / 5.0))
    p = f(f(s2 * p) + f(2.0 / 3.0))
    p = f(f(s2 * p) + f(2.0))
    return f(s * p)


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
