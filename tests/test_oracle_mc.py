"""Pins of the oracle's Monte Carlo pricer (the Hagan SABR/LIBOR dynamics of Section 2.1 under the
spot measure; Table tab:haganMCpricer) against what no-arbitrage and closed forms fix: a zero-strike
caplet is the floating coupon P(0,T_i) - P(0,T_{i+1}) and a zero-strike payer swaption the floating
leg P(0,T_a) - P(0,T_b) under any arbitrage-free dynamics (a dropped or mis-signed drift term, a
wrong numeraire roll or a wrong fixing breaks them); with no vol of vol, beta = 1 and no
forward-vol correlation the model is the lognormal LIBOR market model, where every caplet is
Black's at vol alpha_i.  The Philox4x32-10 generator against Random123's known-answer vectors, the
normals by their moments.  Statistical pins run seeded: a fixed outcome, with bars of 4.5 standard
errors.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
THREADS = max(1, min(16, os.cpu_count() or 1))


def _paper_model():
    return synth.paper_hagan_mc_model(os.path.join(GOLDEN, "paper_euribor_20111121.txt"),
                                      os.path.join(GOLDEN, "paper_mm_20111121.txt"),
                                      os.path.join(GOLDEN, "paper_hagan_mc_20111121.txt"))


def test_philox4x32_known_answers():
    # Random123's kat_vectors for philox4x32 with 10 rounds
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
        ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
        ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
         [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
    ]
    for ctr, key, out in kat:
        assert oracle.philox4x32_10(ctr, key).tolist() == out


def test_mc_normals_moments():
    # 200,000 normals of the pricer's stream: mean 0, variance 1, skew 0, kurtosis 3 within sampling
    # error, and the two halves of a Box-Muller pair uncorrelated
    z = np.array([oracle.mc_normals4(7, p, s, b) for p in range(1000) for s in range(10) for b in range(5)])
    x = z.reshape(-1)
    n = x.size
    assert abs(x.mean()) < 4.5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 4.5 * np.sqrt(2.0 / n)
    assert abs(np.mean(x ** 3)) < 4.5 * np.sqrt(15.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 4.5 * np.sqrt(96.0 / n)
    assert abs(np.mean(z[:, 0] * z[:, 1])) < 4.5 / np.sqrt(z.shape[0])


def test_mc_zero_strike_caplets_and_swaptions_are_the_floating_legs():
    # the paper's calibrated Hagan model (its correlation matrix is indefinite and gets the spectral
    # repair); 20,000 paths, dt = 0.01
    sk, model, cf, ck, _ = _paper_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    P = sk.P
    M = sk.n_fwd
    swp_a, swp_b = [0, 2, 4, 0], [13, 10, 13, 1]
    r = oracle.mc_price(om, model, cap_fwd=np.arange(M), cap_K=np.zeros(M), swp_a=swp_a, swp_b=swp_b,
                        swp_K=np.zeros(4), n_paths=20000, dt=0.01, seed=3, n_threads=THREADS)
    price, se, n_bad = r
    assert n_bad == 0
    exact = np.concatenate([P[:M] - P[1:M + 1], [P[a] - P[b] for a, b in zip(swp_a, swp_b)]])
    z = (price - exact) / se
    assert np.max(np.abs(z)) < 4.5, z
    # the one-period swaption is the first caplet, path by path
    assert price[-1] == pytest.approx(price[0], rel=1e-13)


def test_mc_lognormal_limit_is_black():
    # sigma_i = 0, beta = 1, phi_ii = 0: dF_i = F_i (drift dt + alpha_i dW_i), the lognormal LIBOR
    # market model under the spot measure: caplet on F_i at strike K = Black(F_i, K, T_i, alpha_i)
    sk, model, _, _, _ = _paper_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    al = np.linspace(0.2, 0.4, M)
    m2 = dict(model, beta=1.0, sigma=np.zeros(M), alpha=al, phi=np.zeros(M))
    for mny in (0.9, 1.1):
        K = F * mny
        price, se, n_bad = oracle.mc_price(om, m2, cap_fwd=np.arange(M), cap_K=K, n_paths=20000, dt=0.01, seed=4,
                                           n_threads=THREADS)
        bl = np.array([oracle.black_call(F[i], K[i], sk.T[i], al[i], tau[i] * sk.P[i + 1]) for i in range(M)])
        z = (price - bl) / se
        assert n_bad == 0 and np.max(np.abs(z)) < 4.5, z


def test_mc_is_deterministic_and_thread_count_independent():
    sk, model, cf, ck, _ = _paper_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    a = oracle.mc_price(om, model, cap_fwd=cf[:20], cap_K=ck[:20], n_paths=300, dt=0.05, seed=5, n_threads=1)
    b = oracle.mc_price(om, model, cap_fwd=cf[:20], cap_K=ck[:20], n_paths=300, dt=0.05, seed=5, n_threads=THREADS)
    assert np.allclose(a[0], b[0], rtol=1e-13, atol=0)


# ---------------------------------------------------------------- SA over the Monte Carlo objective
def _self_quoted_swaptions(M=6, n_paths=2000, dt=0.05, seed=5):
    """Payer swaptions on the paper's first M forwards quoted at the Black vols that reproduce the
    oracle's own Monte Carlo prices at the paper's correlation parameters (root-finding on Black)."""
    from scipy.optimize import brentq
    sk, model, _, _, _ = _paper_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    P, T = sk.P, sk.T
    tau = np.diff(T)
    m6 = dict(model, M=M)
    sa, sb, sK = [], [], []
    for a in (0, 1, 2):
        for b in (a + 2, a + 4):
            A = sum(tau[j] * P[j + 1] for j in range(a, b))
            S = (P[a] - P[b]) / A
            for mny in (0.8, 1.0, 1.25):
                sa.append(a); sb.append(b); sK.append(S * mny)
    pr, _, _ = oracle.mc_price(om, m6, swp_a=sa, swp_b=sb, swp_K=sK, n_paths=n_paths, dt=dt, seed=seed, n_threads=1)
    qv = []
    for k in range(len(sa)):
        a, b = sa[k], sb[k]
        A = sum(tau[j] * P[j + 1] for j in range(a, b))
        S = (P[a] - P[b]) / A
        qv.append(brentq(lambda v: oracle.black_call(S, sK[k], T[a], v, A) - pr[k], 1e-4, 5.0, xtol=1e-15))
    y = np.array([model[k] for k in ("eta1", "lambda1", "eta2", "lambda2", "lambda3")])
    return om, m6, np.array(sa), np.array(sb), np.array(sK), np.array(qv), y


def test_mc_objective_vanishes_at_the_generating_correlations():
    # quotes made by the pricer itself at y: f_s(y) = 0 up to the root-finding, so the market prices
    # of the objective (Black's formula, annuity, swap rate, expiry) and the Monte Carlo payoffs agree
    # on every convention; away from y, f_s > 0
    om, m6, sa, sb, sK, qv, y = _self_quoted_swaptions()
    kw = dict(swp_a=sa, swp_b=sb, swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5)
    f_true = oracle.mc_objective(om, m6, y, qv, **kw)
    f_off = oracle.mc_objective(om, m6, y * np.array([0.9, 1.2, 0.9, 1.2, 2.0]), qv, **kw)
    assert f_true <= 1e-12 * f_off and f_off > 0


def test_mc_anneal_descends_from_the_box_centre():
    # the annealing loop over f_s (common random numbers: f_s is deterministic in y) ends well below
    # f_s at its start, at a point whose f_s re-evaluates to the reported value
    om, m6, sa, sb, sK, qv, y = _self_quoted_swaptions()
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    kw = dict(swp_a=sa, swp_b=sb, swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5)
    r = oracle.mc_anneal(om, m6, qv, lo, hi, np.ones(5), 8, 8, 8, 0.7, 9, n_threads=THREADS, **kw)
    f_c = oracle.mc_objective(om, m6, 0.5 * (lo + hi), qv, **kw)
    assert r["f_best"] <= 0.05 * f_c
    assert r["f_best"] == pytest.approx(oracle.mc_objective(om, m6, r["y_best"], qv, **kw), rel=1e-14)
    assert np.all(r["y_best"] >= lo) and np.all(r["y_best"] <= hi)


# ---------------------------------------------------------------- Mercurio & Morini dynamics
def _mm_model():
    return synth.paper_mm_mc_model(os.path.join(GOLDEN, "paper_euribor_20111121.txt"),
                                   os.path.join(GOLDEN, "paper_mm_20111121.txt"))


def test_mc_mm_zero_strike_instruments_are_the_floating_legs():
    # the paper's calibrated Mercurio & Morini model (Section 4.2), one vol process for all forwards
    sk, model = _mm_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    P = sk.P
    M = sk.n_fwd
    swp_a, swp_b = [0, 2, 4, 0], [13, 10, 13, 1]
    price, se, n_bad = oracle.mc_price(om, model, cap_fwd=np.arange(M), cap_K=np.zeros(M), swp_a=swp_a, swp_b=swp_b,
                                       swp_K=np.zeros(4), n_paths=20000, dt=0.01, seed=6, n_threads=THREADS)
    assert n_bad == 0
    exact = np.concatenate([P[:M] - P[1:M + 1], [P[a] - P[b] for a, b in zip(swp_a, swp_b)]])
    z = (price - exact) / se
    assert np.max(np.abs(z)) < 4.5, z
    assert price[-1] == pytest.approx(price[0], rel=1e-13)


def test_mc_mm_lognormal_limit_is_black():
    # sigma = 0 (V stays 1), beta = 1, phi_i = 0: dF_i = F_i (drift dt + alpha_i dW_i), Black at alpha_i
    sk, model = _mm_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    al = np.linspace(0.2, 0.4, M)
    m2 = dict(model, beta=1.0, sigma=np.zeros(M), alpha=al, phi=np.zeros(M))
    K = F * 1.1
    price, se, n_bad = oracle.mc_price(om, m2, cap_fwd=np.arange(M), cap_K=K, n_paths=20000, dt=0.01, seed=7,
                                       n_threads=THREADS)
    bl = np.array([oracle.black_call(F[i], K[i], sk.T[i], al[i], tau[i] * sk.P[i + 1]) for i in range(M)])
    z = (price - bl) / se
    assert n_bad == 0 and np.max(np.abs(z)) < 4.5, z


def test_mc_mm_vol_of_vol_fattens_the_tails():
    # with beta = 1 and every phi_i = 0 the common vol process only mixes the lognormal variance:
    # sigma > 0 raises the price of far out-of-the-money caplets above Black's at alpha_i (the
    # same paths give Black within sampling error at sigma = 0, test above)
    sk, model = _mm_model()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    m2 = dict(model, beta=1.0, sigma=np.full(M, 0.8), alpha=np.full(M, 0.3), phi=np.zeros(M))
    K = F * 2.5
    price, se, _ = oracle.mc_price(om, m2, cap_fwd=np.arange(M), cap_K=K, n_paths=20000, dt=0.01, seed=8,
                                   n_threads=THREADS)
    bl = np.array([oracle.black_call(F[i], K[i], sk.T[i], 0.3, tau[i] * sk.P[i + 1]) for i in range(M)])
    z = (price[1:] - bl[1:]) / se[1:]
    assert np.all(z > 2.0) and np.mean(z) > 4.5, z
