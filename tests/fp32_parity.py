"""Shared rules of the reduced-precision parity tests (imported by the GPU test modules).

Feasibility.  A point is infeasible when some model vol is not a finite positive number (the
objective is then +inf).  The FP32 path must classify every instrument of every point exactly as
the FP64 oracle does, with one stated exception: an instrument whose oracle vol lies within
NEAR_ZERO_REL of zero, relative to the largest |vol| of the same point, sits on the feasibility
boundary (the Hagan correction factor crosses zero there), and FP32 rounding may decide its sign
either way.  `feasibility_mismatches` returns the disagreements; `assert_feasibility_rule` fails on
any that is not on that boundary.

Per-price error.  The library's residuals are r_k = sqrt(w_k) (P_k - P_k^mkt) with the default
weights w_k = 1 / vega_k^2 at the quoted vol, so r_k is a price error in vol units and
|r_k^FP32 - r_k^oracle| is |dP_k| / vega_k, the per-price error in vol units (x 100: vol points).
Two sources bound it: the model vol's error (vega_model / vega_mkt x dsigma) and the relative
rounding of the FP32 Black price (eps_B P_k sqrt(w_k)).  Near the market vol (the generating point,
the end of a search) vega_model ~ vega_mkt and P_k sqrt(w_k) is of order sigma sqrt(T), so the error
is the vol error: GEN_BAR_VOLPT, the FP32 vol bar's order (FP32 vols of FP64 points carry ~1e-6 of
themselves: the rounding of the parameters to FP32, 6e-8, amplified by exponents c u of up to ~20 in
the vol functions; measured per price at the generating points of nine markets: 2.5e-5 to 4.6e-5
vol-pt).  At a point far from the market both terms grow with the model price, and so does |r_k|
(P_k sqrt(w_k) = r_k + P_k^mkt sqrt(w_k)): the bar there is FAR_ABS_VOLPT + FAR_REL |r_k|, FAR_REL
the vol's relative error (~1e-6) times the price's elasticity to the vol, sigma vega / P, which is
large out of the money (measured |dr| / |r| up to 4.2e-6).
"""
import numpy as np

NEAR_ZERO_REL = 1e-5
GEN_BAR_VOLPT = 1e-4      # per price at the generating point (vol points)
FAR_ABS_VOLPT = 2e-4      # per price anywhere: FAR_ABS_VOLPT + FAR_REL |r| (vol points)
FAR_REL = 1e-5


def feasible(v):
    v = np.asarray(v, dtype=np.float64)
    return np.isfinite(v) & (v > 0)


def feasibility_mismatches(ok_lo, v_oracle):
    """Instruments whose reduced-precision feasibility (ok_lo, bool) differs from the oracle's."""
    return np.nonzero(np.asarray(ok_lo, bool) != feasible(v_oracle))[0]


def on_boundary(v_oracle, k):
    v = np.asarray(v_oracle, dtype=np.float64)
    scale = np.max(np.abs(v[np.isfinite(v)])) if np.any(np.isfinite(v)) else 0.0
    return bool(np.isfinite(v[k]) and abs(v[k]) <= NEAR_ZERO_REL * scale)


def assert_feasibility_rule(ok_lo, v_oracle, where=""):
    """Every disagreement must be an instrument on the boundary; returns their count."""
    bad = feasibility_mismatches(ok_lo, v_oracle)
    for k in bad:
        assert on_boundary(v_oracle, k), (
            f"{where}: instrument {k} feasible={bool(ok_lo[k])} in reduced precision, "
            f"oracle vol {v_oracle[k]!r} is not within {NEAR_ZERO_REL} of zero")
    return len(bad)


def assert_point_feasibility_rule(f_lo, f_oracle, om, X, where=""):
    """Point level: finite objective in reduced precision iff finite in the oracle, except at points
    with an instrument on the boundary.  Returns the number of disagreeing points."""
    fin_lo, fin_or = np.isfinite(f_lo), np.isfinite(f_oracle)
    bad = np.nonzero(fin_lo != fin_or)[0]
    for i in bad:
        v = om.model_vols(X[i])
        assert any(on_boundary(v, k) for k in range(len(v))), (
            f"{where}: point {i} objective finite={bool(fin_lo[i])} in reduced precision but "
            f"{bool(fin_or[i])} in the oracle, with no instrument on the feasibility boundary")
    return len(bad)


def residual_errors(gm, om, X, prec, market=0):
    """|r_lo - r_oracle| per (point, instrument) in vol points over the points both sides find
    feasible, after checking the feasibility rule per instrument.  Returns (errors, |r_oracle|),
    each [points x instruments] (rows of infeasible points are NaN)."""
    _, r_lo = gm.residuals(X, prec, market=market)
    r_lo = r_lo.cpu().numpy()
    err = np.full(r_lo.shape, np.nan)
    mag = np.full(r_lo.shape, np.nan)
    for i in range(X.shape[0]):
        v_or = om.model_vols(X[i])
        assert_feasibility_rule(np.isfinite(r_lo[i]), v_or, where=f"point {i}")
        r_or, _ = om.residuals_jac(X[i])
        if r_or is None or not np.all(np.isfinite(r_lo[i])):
            continue
        err[i] = np.abs(r_lo[i] - r_or) * 100.0
        mag[i] = np.abs(r_or) * 100.0
    return err, mag


def check_per_price(err, mag, gen_row, where=""):
    """The per-price bars on residual_errors' output, gen_row the generating point's row; returns a
    one-line summary."""
    ok = np.isfinite(err)
    assert ok.any(), f"{where}: no feasible point"
    ratio = err[ok] / (FAR_ABS_VOLPT + FAR_REL * mag[ok])
    gen = err[gen_row][np.isfinite(err[gen_row])]
    line = (f"{where}: per-price error max {err[ok].max():.3e} median {np.median(err[ok]):.3e} vol-pt, "
            f"worst / far bar {ratio.max():.3f}, generating point max {gen.max() if gen.size else float('nan'):.3e}")
    print(line)
    assert ratio.max() <= 1.0, line
    assert gen.size > 0 and gen.max() <= GEN_BAR_VOLPT, line
    return line


def objective_bound_at_noise_floor(f_oracle, n_instr):
    """|f_lo - f_oracle| allowed where every price meets GEN_BAR_VOLPT (a in vol units):
    |sum (r + dr)^2 - sum r^2| <= 2 ||r|| ||dr|| + ||dr||^2 <= 2 sqrt(f n) a + n a^2."""
    a = GEN_BAR_VOLPT / 100.0
    return 2.0 * np.sqrt(f_oracle * n_instr) * a + n_instr * a * a


def objective_bound(f_oracle, n_instr):
    """|f_lo - f_oracle| allowed at any feasible point where every price meets the far bar
    |dr_k| <= a + b |r_k| (a = FAR_ABS_VOLPT, b = FAR_REL, in vol units): ||dr|| <= a sqrt(n) + b sqrt(f),
    so |sum (r + dr)^2 - sum r^2| <= 2 sqrt(f) d + d^2 with d = a sqrt(n) + b sqrt(f)."""
    d = FAR_ABS_VOLPT / 100.0 * np.sqrt(n_instr) + FAR_REL * np.sqrt(f_oracle)
    return 2.0 * np.sqrt(f_oracle) * d + d * d
