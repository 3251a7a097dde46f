"""Seeded synthetic market inputs, shared by the oracle tests, the library tests and the bench.

This module holds none of the calibration method's arithmetic.  It lays out

* a tenor grid and discount factors built from a prescribed simply-compounded forward curve
  (the recipe's forward levels, P(0,T_{k+1}) = P(0,T_k) / (1 + tau_k F_k)),
* strike grids around the recipe's forward levels (never around a model quantity),
* parameter boxes, generating ("true") parameters drawn uniformly inside them,
* Gaussian noise draws, in vol units, one per instrument.

Model vols at the generating parameters, and the quotes built from them, are computed by whoever
consumes a skeleton: the oracle in the tests, the library itself in the bench.

The shapes follow the paper's EURIBOR workload (Section 4, Tables tab:curvaFD, tab:smilesFws and
tab:smilesTS): semi-annual forwards, caplet smiles on a log-moneyness grid, and an expiry x tenor x
moneyness swaption grid.  The values are synthetic.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

MODEL_SABR_SMILE = 0
MODEL_REBONATO_LMM = 1
MODEL_MERCURIO_MORINI = 2

FORMULA_HAGAN2002 = 0
FORMULA_PAPER = 1

# Parameter slots of the Rebonato SABR/LIBOR model (Section 2.3 and the parameter classes of
# Section 3): g(u) = (a + b u) e^{-c u} + d, h(u) = (alpha_h + beta_h u) e^{-gamma_h u} + delta_h,
# phi = phi_ii, and the correlation decays lambda1 (rho_ij), lambda2 (theta_ij), lambda3 (phi_ij).
REBONATO_SLOTS = ("a", "b", "c", "d", "alpha_h", "beta_h", "gamma_h", "delta_h",
                  "phi", "lambda1", "lambda2", "lambda3")
SMILE_SLOTS = ("alpha", "rho", "nu")


def mm_slots(n_fwd: int):
    """Parameter slots of the Mercurio & Morini model on n_fwd forwards (Section 2.2 and the
    parameter classes of Section 3): phi_0..phi_{M-1}, the common sigma, alpha_0..alpha_{M-1}."""
    return tuple([f"phi_{i}" for i in range(n_fwd)] + ["sigma"] + [f"alpha_{i}" for i in range(n_fwd)])

BASE_SEED = 240801470


@dataclasses.dataclass
class Skeleton:
    """Everything a market needs except its quotes."""
    name: str
    model: int
    formula: int
    beta: float
    T: np.ndarray          # float64 [n_fwd+1]: fixing times T_0..T_{n-1}, then the last payment time
    P: np.ndarray          # float64 [n_fwd+1]: discount factors P(0, T_k)
    cap_fwd: np.ndarray    # int32 [n_cap]: forward index of each caplet
    cap_K: np.ndarray      # float64 [n_cap]
    swp_start: np.ndarray  # int32 [n_swp]: first forward of the underlying swap
    swp_end: np.ndarray    # int32 [n_swp]: one past the last forward
    swp_K: np.ndarray      # float64 [n_swp]
    lo: np.ndarray         # float64 [n_param]: search box
    hi: np.ndarray
    free: np.ndarray       # uint8 [n_param]: 1 = the annealer moves this slot
    theta_true: np.ndarray  # float64 [n_param]: generating parameters
    noise: np.ndarray      # float64 [n_cap + n_swp]: N(0, sigma_n) draws in vol units
    panel: float = 0.5     # quadrature panel width (years)
    quad_nodes: int = 8    # Gauss-Legendre nodes per panel
    # annealing schedule of the workload
    n_chains: int = 64
    n_levels: int = 100
    steps: int = 50
    cooling: float = 0.9

    @property
    def n_fwd(self) -> int:
        return len(self.T) - 1

    @property
    def n_cap(self) -> int:
        return len(self.cap_K)

    @property
    def n_swp(self) -> int:
        return len(self.swp_K)

    @property
    def n_instr(self) -> int:
        return self.n_cap + self.n_swp

    @property
    def n_param(self) -> int:
        return len(self.lo)

    def box_centre(self) -> np.ndarray:
        return 0.5 * (self.lo + self.hi)

    def replace(self, **kw) -> "Skeleton":
        return dataclasses.replace(self, **kw)


def _curve_from_forwards(fix_times: np.ndarray, fwd: np.ndarray, p_first: float):
    """Tenor grid and discount factors for a prescribed forward curve (the input recipe)."""
    n = len(fwd)
    T = np.empty(n + 1)
    T[:n] = fix_times
    T[n] = fix_times[-1] + (fix_times[-1] - fix_times[-2] if n > 1 else 0.5)
    P = np.empty(n + 1)
    P[0] = p_first
    for k in range(n):
        P[k + 1] = P[k] / (1.0 + (T[k + 1] - T[k]) * fwd[k])
    return T, P


def smile_2y(seed: int = BASE_SEED, noise_volpt: float = 0.2, formula: int = FORMULA_HAGAN2002,
             noise_free: bool = False) -> Skeleton:
    """Single SABR smile: F = 3%, expiry 2y, 11 strikes F-200bp..F+200bp in 40bp steps.

    Generating point (alpha, beta, rho, nu) = (0.03, 0.5, -0.3, 0.4); beta is fixed.
    Annealing schedule: 64 chains x 100 temperatures x 50 steps, cooling 0.9.
    """
    rng = np.random.default_rng(seed)
    f = 0.03
    # flat simply-compounded 3% curve, semi-annual: P(0,2) = 1.015^-4, P(0,2.5) = P(0,2)/1.015
    T, P = _curve_from_forwards(np.array([2.0]), np.array([f]), 1.015 ** -4)
    T[1] = 2.5
    strikes = f + 1e-4 * np.arange(-200, 201, 40)
    n = len(strikes)
    noise = np.zeros(n) if noise_free else rng.normal(0.0, noise_volpt / 100.0, size=n)
    return Skeleton(
        name="smile_2y", model=MODEL_SABR_SMILE, formula=formula, beta=0.5, T=T, P=P,
        cap_fwd=np.zeros(n, np.int32), cap_K=strikes.astype(np.float64),
        swp_start=np.zeros(0, np.int32), swp_end=np.zeros(0, np.int32), swp_K=np.zeros(0),
        lo=np.array([0.005, -0.99, 0.01]), hi=np.array([0.1, 0.99, 1.5]),
        free=np.ones(3, np.uint8), theta_true=np.array([0.03, -0.3, 0.4]), noise=noise,
        n_chains=64, n_levels=100, steps=50, cooling=0.9)


# Boxes the generating Rebonato parameters are drawn from (uniform), slot by slot.
_REB_TRUE_BOX = np.array([
    [0.0, 0.02],   # a
    [0.0, 0.05],   # b
    [0.3, 2.0],    # c
    [0.02, 0.05],  # d
    [0.0, 0.3],    # alpha_h
    [0.0, 0.5],    # beta_h
    [0.3, 2.0],    # gamma_h
    [0.1, 0.4],    # delta_h
    [-0.6, 0.2],   # phi
    [0.05, 0.3],   # lambda1
    [0.05, 0.5],   # lambda2
    [0.0, 0.3],    # lambda3
])


def _rebonato_search_box():
    lo = _REB_TRUE_BOX[:, 0].copy()
    hi = _REB_TRUE_BOX[:, 1].copy()
    w = hi - lo
    lo, hi = lo - 0.5 * w, hi + 0.5 * w
    lo[2] = max(lo[2], 0.05)   # c
    lo[6] = max(lo[6], 0.05)   # gamma_h
    lo[8] = max(lo[8], -0.99)  # phi
    hi[8] = min(hi[8], 0.99)
    lo[9:12] = np.maximum(lo[9:12], 0.0)  # correlation decays stay non-negative
    return lo, hi


def _semiannual_curve(n_fwd: int):
    fix = 0.5 * (np.arange(n_fwd) + 1.0)
    fwd = 0.01 + 0.03 * np.arange(n_fwd) / max(n_fwd - 1, 1)
    T, P = _curve_from_forwards(fix, fwd, 1.0 / (1.0 + 0.5 * 0.01))
    return T, P, fwd


def caplet_term_structure(seed: int = BASE_SEED + 1, noise_volpt: float = 0.02,
                          n_fwd: int = 20, n_strikes: int = 15, noise_free: bool = False,
                          formula: int = FORMULA_HAGAN2002) -> Skeleton:
    """Rebonato SABR/LIBOR caplet term structure.

    n_fwd semi-annual forwards (fixings 0.5, 1.0, ...), forward levels rising linearly from 1% to
    4%, and n_strikes caplets per forward at K = F e^m, m in linspace(-0.7, 0.7).  Nine free
    parameters (the abcd forms of g and h, and phi); the correlation decays do not reach caplets
    and stay fixed.  Schedule: 4096 chains x 200 temperatures x 100 steps, cooling 0.95.
    """
    rng = np.random.default_rng(seed)
    T, P, fwd = _semiannual_curve(n_fwd)
    m = np.linspace(-0.7, 0.7, n_strikes)
    cap_fwd = np.repeat(np.arange(n_fwd, dtype=np.int32), n_strikes)
    cap_K = (fwd[:, None] * np.exp(m)[None, :]).reshape(-1)
    lo, hi = _rebonato_search_box()
    theta = rng.uniform(_REB_TRUE_BOX[:, 0], _REB_TRUE_BOX[:, 1])
    free = np.array([1] * 9 + [0] * 3, np.uint8)
    n = len(cap_K)
    noise = np.zeros(n) if noise_free else rng.normal(0.0, noise_volpt / 100.0, size=n)
    return Skeleton(
        name=f"caplets_{n_fwd}x{n_strikes}", model=MODEL_REBONATO_LMM, formula=formula, beta=0.5,
        T=T, P=P, cap_fwd=cap_fwd, cap_K=cap_K, swp_start=np.zeros(0, np.int32),
        swp_end=np.zeros(0, np.int32), swp_K=np.zeros(0), lo=lo, hi=hi, free=free,
        theta_true=theta, noise=noise, n_chains=4096, n_levels=200, steps=100, cooling=0.95)


def joint_caplet_swaption(seed: int = BASE_SEED + 2, noise_volpt: float = 0.02, n_fwd: int = 40,
                          cap_fwds: int = 20, n_strikes: int = 15, expiries=range(1, 11),
                          tenors=range(1, 11), swp_m=(-0.6, -0.4, -0.2, 0.0, 0.2, 0.4, 0.6),
                          noise_free: bool = False) -> Skeleton:
    """Joint caplet + swaption market on n_fwd semi-annual forwards (1% -> 4%).

    Caplets: forwards 0..cap_fwds-1 x n_strikes log-moneyness points in [-0.7, 0.7].
    Swaptions: expiry E years x tenor L years x moneyness m; the underlying swap runs over the
    forwards fixing at E, E+0.5, ..., E+L-0.5, and the strike is the plain average of those
    forward levels times e^m.  All twelve parameters free.  Schedule: 16384 chains x 200 x 100.
    """
    rng = np.random.default_rng(seed)
    T, P, fwd = _semiannual_curve(n_fwd)
    m = np.linspace(-0.7, 0.7, n_strikes)
    cap_fwd = np.repeat(np.arange(cap_fwds, dtype=np.int32), n_strikes)
    cap_K = (fwd[:cap_fwds, None] * np.exp(m)[None, :]).reshape(-1)
    s0, s1, sk = [], [], []
    for e in expiries:
        for ln in tenors:
            a = int(round(2 * e)) - 1
            b = a + int(round(2 * ln))
            if b > n_fwd:
                continue
            level = fwd[a:b].mean()
            for mm in swp_m:
                s0.append(a)
                s1.append(b)
                sk.append(level * np.exp(mm))
    lo, hi = _rebonato_search_box()
    theta = rng.uniform(_REB_TRUE_BOX[:, 0], _REB_TRUE_BOX[:, 1])
    n = len(cap_K) + len(sk)
    noise = np.zeros(n) if noise_free else rng.normal(0.0, noise_volpt / 100.0, size=n)
    return Skeleton(
        name=f"joint_{n_fwd}f_{len(cap_K)}c_{len(sk)}s", model=MODEL_REBONATO_LMM,
        formula=FORMULA_HAGAN2002, beta=0.5, T=T, P=P, cap_fwd=cap_fwd, cap_K=cap_K,
        swp_start=np.array(s0, np.int32), swp_end=np.array(s1, np.int32),
        swp_K=np.array(sk, np.float64), lo=lo, hi=hi, free=np.ones(12, np.uint8),
        theta_true=theta, noise=noise, n_chains=16384, n_levels=200, steps=100, cooling=0.95)


def batch_market(j: int, noise_volpt: float = 0.02) -> Skeleton:
    """Member j of the uneven batch: M ~ U{10..60} forwards, U{50..1000} instruments.

    The swaption fraction is U(0,1); caplets sample (forward, m) pairs and swaptions sample
    (expiry, tenor, m) triples inside the M/2-year horizon.  Each member has its own seed.
    """
    rng = np.random.default_rng(BASE_SEED + 1000 + j)
    n_fwd = int(rng.integers(10, 61))
    n_instr = int(rng.integers(50, 1001))
    frac_swp = float(rng.uniform(0.0, 1.0))
    n_swp = int(round(frac_swp * n_instr))
    n_cap = n_instr - n_swp
    T, P, fwd = _semiannual_curve(n_fwd)
    cf = rng.integers(0, n_fwd, size=n_cap).astype(np.int32)
    cm = rng.uniform(-0.7, 0.7, size=n_cap)
    order = np.lexsort((cm, cf))
    cf, cm = cf[order], cm[order]
    cap_K = fwd[cf] * np.exp(cm)
    s0 = np.empty(n_swp, np.int32)
    s1 = np.empty(n_swp, np.int32)
    sk = np.empty(n_swp)
    for s in range(n_swp):
        a = int(rng.integers(1, n_fwd))       # first forward index >= 1: expiry >= 1y... 0.5y grid
        b = int(rng.integers(a + 1, min(a + 20, n_fwd) + 1))
        s0[s], s1[s] = a, b
        sk[s] = fwd[a:b].mean() * np.exp(rng.uniform(-0.6, 0.6))
    order = np.lexsort((sk, s1, s0))
    s0, s1, sk = s0[order], s1[order], sk[order]
    lo, hi = _rebonato_search_box()
    theta = rng.uniform(_REB_TRUE_BOX[:, 0], _REB_TRUE_BOX[:, 1])
    noise = rng.normal(0.0, noise_volpt / 100.0, size=n_instr)
    return Skeleton(
        name=f"batch_{j}", model=MODEL_REBONATO_LMM, formula=FORMULA_HAGAN2002, beta=0.5,
        T=T, P=P, cap_fwd=cf, cap_K=cap_K, swp_start=s0, swp_end=s1, swp_K=sk, lo=lo, hi=hi,
        free=np.ones(12, np.uint8), theta_true=theta, noise=noise,
        n_chains=4096, n_levels=100, steps=50, cooling=0.9)


def mercurio_morini_caplets(seed: int = BASE_SEED + 3, noise_volpt: float = 0.02, n_fwd: int = 13,
                            n_strikes: int = 9, formula: int = FORMULA_PAPER,
                            noise_free: bool = False) -> Skeleton:
    """Mercurio & Morini caplet smiles: n_fwd semi-annual forwards (fixings 0.5, 1.0, ..., levels
    1% -> 4% as in the caplet term structure) with n_strikes caplets each at K = F e^m,
    m in linspace(-0.8, 0.8) (the moneyness span of the paper's smiles).  Generating point:
    phi_i ~ U(-0.8, 0.2), sigma ~ U(0.3, 0.8), alpha_i ~ U(0.05, 0.1) (the ranges of the paper's
    calibrated Table tab:paramsMercurioVolas); search box phi in [-0.99, 0.99], sigma in
    [0.01, 1.5], alpha in [0.001, 0.5].  Schedule: 4096 chains x 100 temperatures x 20 steps,
    cooling 0.95.  2 n_fwd + 1 slots, all free."""
    rng = np.random.default_rng(seed)
    T, P, fwd = _semiannual_curve(n_fwd)
    m = np.linspace(-0.8, 0.8, n_strikes)
    cap_fwd = np.repeat(np.arange(n_fwd, dtype=np.int32), n_strikes)
    cap_K = (fwd[:, None] * np.exp(m)[None, :]).reshape(-1)
    theta = np.concatenate([rng.uniform(-0.8, 0.2, n_fwd), rng.uniform(0.3, 0.8, 1),
                            rng.uniform(0.05, 0.1, n_fwd)])
    lo = np.concatenate([np.full(n_fwd, -0.99), [0.01], np.full(n_fwd, 0.001)])
    hi = np.concatenate([np.full(n_fwd, 0.99), [1.5], np.full(n_fwd, 0.5)])
    n = len(cap_K)
    noise = np.zeros(n) if noise_free else rng.normal(0.0, noise_volpt / 100.0, size=n)
    return Skeleton(
        name=f"mm_caplets_{n_fwd}x{n_strikes}", model=MODEL_MERCURIO_MORINI, formula=formula, beta=0.5,
        T=T, P=P, cap_fwd=cap_fwd, cap_K=cap_K, swp_start=np.zeros(0, np.int32),
        swp_end=np.zeros(0, np.int32), swp_K=np.zeros(0), lo=lo, hi=hi,
        free=np.ones(2 * n_fwd + 1, np.uint8), theta_true=theta, noise=noise,
        n_chains=4096, n_levels=100, steps=20, cooling=0.95)


def uniform_in_box(skel: Skeleton, n: int, seed: int) -> np.ndarray:
    """n parameter sets drawn uniformly in the search box (fixed slots keep theta_true)."""
    rng = np.random.default_rng(seed)
    X = np.repeat(skel.theta_true[None, :], n, axis=0)
    free = skel.free.astype(bool)
    X[:, free] = rng.uniform(skel.lo[free], skel.hi[free], size=(n, int(free.sum())))
    return X


def market_vols(skel: Skeleton, model_vols_at_truth: np.ndarray,
                noise: Optional[np.ndarray] = None) -> np.ndarray:
    """Quotes in vol units: the model vols at the generating point plus the noise draws."""
    nz = skel.noise if noise is None else noise
    return np.asarray(model_vols_at_truth, np.float64) + nz


# ---------------------------------------------------------------- the paper's real-data caplet smiles
def read_paper_market(path: str) -> dict:
    """The sections of a real-data market file (discount curve, moneyness, smiles, the paper's
    calibrated parameters and published figures), as plain lists; no arithmetic of the method."""
    sec, out = None, {"curve": [], "moneyness": [], "smiles": [], "params": [], "published": {}}
    # (other sections, e.g. [sigma] and [model_vols] of a model's calibration, as lists of rows)
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            sec = line.strip("[]")
            out.setdefault(sec, [])
            continue
        parts = line.split()
        if sec == "published":
            out["published"][parts[0]] = " ".join(parts[1:])
        else:
            out[sec].append(parts)
    return out


def paper_euribor_caplet_smiles(path: str):
    """The 13 caplet smiles of the paper's real-data test (Section 4) as 13 single-smile markets of
    the Hagan model with Eq. (sigmaHagan), beta = 0.5, one per forward.

    Readings (the paper does not state them): expiries in ACT/365 years from the valuation date
    21/11/2011; a forward accrues over its fixing date to the next one in ACT/360 (the EURIBOR
    convention); discount factors between the curve's dates by linear interpolation of log P in
    ACT/365 time; the smiles' moneyness is ln(K / F); search box alpha in [0.001, 0.5], rho in
    [-0.99, 0.99], nu in [0.01, 1] (the paper's calibrated sigma_1 sits at 1.0000); the paper's
    schedule: w = 256 x 64 = 16384 chains, N = 10 steps per level, cooling 0.99 from T0 = 10 to
    T_min = 0.01 (688 levels; T0 is passed to the search, it is no field of a skeleton).
    Returns (skeletons, quotes, paper_params [13 x (alpha, rho, nu)], published figures).
    """
    import datetime as _dt
    d = read_paper_market(path)
    d0 = _dt.date(2011, 11, 21)

    def days(s, sep, century):
        a, b, c = (int(x) for x in s.split(sep))
        return (_dt.date(c + century, b, a) - d0).days

    ct = np.array([days(r[0], "/", 0) / 365.0 for r in d["curve"]])
    lp = np.log(np.array([float(r[1]) for r in d["curve"]]))

    def disc(t):
        return float(np.exp(np.interp(t, ct, lp)))

    m = np.array([float(x) / 100.0 for x in d["moneyness"][0]])
    fix = [days(r[0], "-", 2000) for r in d["smiles"]]
    # the payment date of the last forward: six months after its fixing
    last = _dt.date(2011, 11, 21) + _dt.timedelta(days=fix[-1])
    fix.append((_dt.date(last.year + (last.month + 6 - 1) // 12, (last.month + 6 - 1) % 12 + 1, last.day) - d0).days)
    sks, quotes = [], []
    for i, row in enumerate(d["smiles"]):
        t0, tau = fix[i] / 365.0, (fix[i + 1] - fix[i]) / 360.0
        p0, p1 = disc(t0), disc(fix[i + 1] / 365.0)
        F = (p0 / p1 - 1.0) / tau
        sks.append(Skeleton(
            name=f"paper_F{i + 1}", model=MODEL_SABR_SMILE, formula=FORMULA_PAPER, beta=0.5,
            T=np.array([t0, t0 + tau]), P=np.array([p0, p1]), cap_fwd=np.zeros(len(m), np.int32),
            cap_K=F * np.exp(m), swp_start=np.zeros(0, np.int32), swp_end=np.zeros(0, np.int32),
            swp_K=np.zeros(0), lo=np.array([0.001, -0.99, 0.01]), hi=np.array([0.5, 0.99, 1.0]),
            free=np.ones(3, np.uint8), theta_true=np.array([0.05, 0.0, 0.5]), noise=np.zeros(len(m)),
            n_chains=16384, n_levels=688, steps=10, cooling=0.99))
        quotes.append(np.array([float(v) / 100.0 for v in row[1:]]))
    params = np.array([[float(r[3]), float(r[1]), float(r[2])] for r in d["params"]])
    return sks, quotes, params, d["published"]


def paper_euribor_mm_market(path: str, mm_path: str):
    """The 13 caplet smiles of the paper's real-data test (Section 4) as ONE market of the
    Mercurio & Morini model (Section 2.2) with Eq. (sigmaHagan), beta = 0.5: 27 parameters
    [phi_1..phi_13, sigma, alpha_1..alpha_13], coupled through sigma and the drift of
    Eq. (haganForMercurio), so the smiles cannot be searched one by one.

    Readings (the paper does not state them), beside those of paper_euribor_caplet_smiles: the 13
    forwards are consecutive six-month periods, so they form the tenor structure whose fixing
    dates the drift integral steps through; the tenor grid runs on the accrual clock, T_0 = the
    first fixing (ACT/365 from 21/11/2011) and T_{i+1} = T_i + tau_i (ACT/360), so that
    T_{i+1} - T_i is the accrual of forward i (with the fixings in ACT/365 instead, the descent
    from the paper's parameters ends at the same MRE and parameters to 1e-6); discount factors
    at the actual dates; box phi in [-0.99, 0.99], sigma in [0.01, 1.5], alpha in [0.001, 0.5].
    Schedule: the paper's (16384 chains, N = 10, cooling 0.99 from T0 = 10 to T_min = 0.01:
    688 levels).
    Returns (skeleton, quotes [117], paper_params [27], paper model vols [12 x 5] (percent),
    published figures)."""
    import datetime as _dt
    d = read_paper_market(path)
    mm = read_paper_market(mm_path)
    d0 = _dt.date(2011, 11, 21)

    def days(s, sep, century):
        a, b, c = (int(x) for x in s.split(sep))
        return (_dt.date(c + century, b, a) - d0).days

    ct = np.array([days(r[0], "/", 0) / 365.0 for r in d["curve"]])
    lp = np.log(np.array([float(r[1]) for r in d["curve"]]))

    def disc_days(n):
        return float(np.exp(np.interp(n / 365.0, ct, lp)))

    m = np.array([float(x) / 100.0 for x in d["moneyness"][0]])
    fix = [days(r[0], "-", 2000) for r in d["smiles"]]
    last = d0 + _dt.timedelta(days=fix[-1])
    fix.append((_dt.date(last.year + (last.month + 6 - 1) // 12, (last.month + 6 - 1) % 12 + 1, last.day) - d0).days)
    n_fwd = len(d["smiles"])
    T = np.empty(n_fwd + 1)
    T[0] = fix[0] / 365.0
    for i in range(n_fwd):
        T[i + 1] = T[i] + (fix[i + 1] - fix[i]) / 360.0
    P = np.array([disc_days(n) for n in fix])
    F = np.array([(P[i] / P[i + 1] - 1.0) / (T[i + 1] - T[i]) for i in range(n_fwd)])
    cap_fwd = np.repeat(np.arange(n_fwd, dtype=np.int32), len(m))
    cap_K = (F[:, None] * np.exp(m)[None, :]).reshape(-1)
    quotes = np.array([[float(v) / 100.0 for v in row[1:]] for row in d["smiles"]]).reshape(-1)
    phi = np.array([float(r[1]) for r in mm["params"]])
    alpha = np.array([float(r[2]) for r in mm["params"]])
    sigma = float(mm["sigma"][0][0])
    params = np.concatenate([phi, [sigma], alpha])
    vols = np.array([[float(v) for v in r[1:]] for r in mm["model_vols"]])
    lo = np.concatenate([np.full(n_fwd, -0.99), [0.01], np.full(n_fwd, 0.001)])
    hi = np.concatenate([np.full(n_fwd, 0.99), [1.5], np.full(n_fwd, 0.5)])
    sk = Skeleton(
        name="paper_mm", model=MODEL_MERCURIO_MORINI, formula=FORMULA_PAPER, beta=0.5, T=T, P=P,
        cap_fwd=cap_fwd, cap_K=cap_K, swp_start=np.zeros(0, np.int32), swp_end=np.zeros(0, np.int32),
        swp_K=np.zeros(0), lo=lo, hi=hi, free=np.ones(2 * n_fwd + 1, np.uint8),
        theta_true=0.5 * (lo + hi), noise=np.zeros(len(cap_K)),
        n_chains=16384, n_levels=688, steps=10, cooling=0.99)
    return sk, quotes, params, vols, mm["published"]


def paper_hagan_mc_model(path: str, mm_path: str, mc_path: str):
    """The paper's calibrated Hagan SABR/LIBOR model (Section 4.1) as the input of the Monte Carlo
    pricer: the 13-forward EURIBOR tenor structure of paper_euribor_mm_market (its skeleton carries
    T and P), the per-forward (phi_ii, sigma_i, alpha_i) of Table tab:paramsHaganVolas, beta = 0.5,
    the correlation parameters of Section 4.1.2, and the 117 caplets of Table tab:smilesFws (9
    strikes on each forward).  Returns (skeleton, model dict, caplet forwards, caplet strikes,
    Table tab:haganMCpricer rows [paths, dt, CPU s, GPU s, speedup])."""
    sk, _, _, _, _ = paper_euribor_mm_market(path, mm_path)
    _, _, hp, _ = paper_euribor_caplet_smiles(path)
    mc = read_paper_market(mc_path)
    corr = {r[0]: float(r[1]) for r in mc["correlation"]}
    model = dict(M=sk.n_fwd, beta=0.5, eta1=corr["eta1"], lambda1=corr["lambda1"], eta2=corr["eta2"],
                 lambda2=corr["lambda2"], lambda3=corr["lambda3"], alpha=hp[:, 0].copy(), sigma=hp[:, 2].copy(),
                 phi=hp[:, 1].copy())
    rows = np.array([[float(x) for x in r] for r in mc["mc_timings"]])
    return sk, model, sk.cap_fwd.copy(), sk.cap_K.copy(), rows


def paper_swaption_smiles(path: str, mm_path: str, swp_path: str):
    """The 180 swaptions of the paper's real-data test (Table tab:smilesTS: maturities 21/05/2012 ..
    21/11/2013, the fixings of the first four forwards, swaps of 1 .. 5 years, nine moneyness
    levels) on the 13-forward tenor structure of paper_euribor_mm_market: payer swaption on the
    forwards [a, a + 2 x years) with strike K = S e^m, S = (P(0, T_a) - P(0, T_b)) / sum tau_k
    P(0, T_{k+1}) the forward swap rate (input preparation: the swap rate's definition).
    Returns (skeleton, swp_start, swp_end, swp_K, quote vols [180], published figures)."""
    import datetime as _dt
    sk, _, _, _, _ = paper_euribor_mm_market(path, mm_path)
    d = read_paper_market(swp_path)
    fix_dates = [r[0] for r in read_paper_market(path)["smiles"]]
    m = np.array([float(x) / 100.0 for x in d["moneyness"][0]])
    T, P = sk.T, sk.P
    sa, sb, sK, vol = [], [], [], []
    for row in d["smiles"]:
        years = int(row[0])
        dd, mo, yy = (int(x) for x in row[1].split("/"))
        key = _dt.date(yy, mo, dd).strftime("%d-%m-%y")
        a = fix_dates.index(key)
        b = a + 2 * years
        A = sum((T[k + 1] - T[k]) * P[k + 1] for k in range(a, b))
        S = (P[a] - P[b]) / A
        for mk, v in zip(m, row[2:]):
            sa.append(a); sb.append(b); sK.append(S * np.exp(mk)); vol.append(float(v) / 100.0)
    return (sk, np.array(sa, np.int32), np.array(sb, np.int32), np.array(sK), np.array(vol), d["published"])


def paper_mm_mc_model(path: str, mm_path: str):
    """The paper's calibrated Mercurio & Morini model (Section 4.2) as the input of the Monte Carlo
    pricer: the 13-forward tenor structure of paper_euribor_mm_market, alpha_i and phi_i of Table
    tab:paramsMercurioVolas, the common sigma (sigma[i] = sigma for every forward), beta = 0.5, and
    eta1, lambda1 of Section 4.2.2 (the other correlation fields are unused by the model).  Returns
    (skeleton, model dict with model = 2)."""
    sk, _, params, _, _ = paper_euribor_mm_market(path, mm_path)
    mm = read_paper_market(mm_path)
    corr = {r[0]: float(r[1]) for r in mm["correlation"]}
    M = sk.n_fwd
    model = dict(M=M, model=MODEL_MERCURIO_MORINI, beta=0.5, eta1=corr["eta1"], lambda1=corr["lambda1"], eta2=0.0,
                 lambda2=0.0, lambda3=0.0, alpha=params[M + 1:].copy(), sigma=np.full(M, params[M]),
                 phi=params[:M].copy())
    return sk, model
