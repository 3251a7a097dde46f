"""Coefficients of the FP32 complementary error function used by the FP32 pricer.

Form (the Chebyshev-exponent form of Press, Teukolsky, Vetterling, Flannery, "Numerical
Recipes", 2nd ed., Section 6.2):

    erfc(x) ~= t * exp(-x^2 + P(t)),   t = 1 / (1 + x/2),   x >= 0,   deg P = 9,

with erfc(x) = 2 - erfc(-x) for x < 0.  The coefficients of P are fitted here, by iteratively
reweighted least squares towards a minimax fit of log(erfc(x) / t) + x^2 on t in (0, 1] (x in
[0, inf)), against 40-digit mpmath values.  Run to regenerate the table printed in
device_math.cuh:

    python paper_2408_01470_b300/csrc/gen_erfc_fit.py
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 40
DEG = 9


def target(t):
    # x from t = 1 / (1 + x/2):  x = 2 (1/t - 1)
    x = 2 * (1 / mp.mpf(t) - 1)
    return mp.log(mp.erfc(x) / t) + x * x


def fit():
    # Chebyshev-distributed samples in t over (t_min, 1]; t_min corresponds to x = 12
    t_min = 1.0 / (1.0 + 6.0)
    k = np.arange(4000)
    ts = 0.5 * (1 + t_min) + 0.5 * (1 - t_min) * np.cos(np.pi * (k + 0.5) / len(k))
    ys = np.array([float(target(t)) for t in ts])
    V = np.vander(ts, DEG + 1, increasing=True)
    w = np.ones_like(ts)
    for _ in range(30):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], ys * sw, rcond=None)
        err = V @ c - ys
        w *= (np.abs(err) / np.abs(err).max()) ** 0.5 + 1e-3
        w /= w.mean()
    return c, np.abs(V @ c - ys).max()


if __name__ == "__main__":
    c, e = fit()
    print(f"// max |error| of P on the fit range: {e:.3e} (relative error of erfc)")
    for i, v in enumerate(c):
        print(f"  {v:+.9e}f,  // t^{i}")
