"""The Monte Carlo pricer and the annealer over it for the Mercurio & Morini dynamics (Section 2.2:
one volatility process shared by every forward, dV = sigma V dZ, V(0) = 1, dF_i = mu_i dt + alpha_i V
F_i^beta dW_i, corr(W_i, Z) = phi_i) on the GPU, through the C-ABI.

FP64: the oracle's paths (the same Philox4x32-10 counters, Box-Muller normals, time grid and
correlation factor with Z first), so prices and standard errors agree to rounding order.  FP32: bar
derived as for the Hagan dynamics.  At production path counts the no-arbitrage pins hold for the
device's own paths.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mm():
    return synth.paper_mm_mc_model(os.path.join(GOLDEN, "paper_euribor_20111121.txt"),
                                   os.path.join(GOLDEN, "paper_mm_20111121.txt"))


def _instruments(sk):
    # caplets on every forward at 0.7, 1.0 and 1.5 times its forward rate, and payer swaptions
    # (expiries on forwards 0..8, ends up to the last forward, strikes around the forward swap rate)
    P, T = sk.P, sk.T
    M = sk.n_fwd
    F = (P[:M] / P[1:M + 1] - 1.0) / np.diff(T)
    cf = np.repeat(np.arange(M), 3)
    ck = np.concatenate([F[i] * np.array([0.7, 1.0, 1.5]) for i in range(M)])
    sa, sb, sK = [], [], []
    for a in (0, 2, 4, 8):
        for b in (a + 1, a + 4, 13):
            if a < b <= M:
                A = sum((T[j + 1] - T[j]) * P[j + 1] for j in range(a, b))
                S = (P[a] - P[b]) / A
                for m in (0.8, 1.0, 1.25):
                    sa.append(a); sb.append(b); sK.append(S * m)
    return cf, ck, np.array(sa), np.array(sb), np.array(sK)


def test_mc_mm_fp64_paths_match_the_oracle(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    cf, ck, sa, sb, sK = _instruments(sk)
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    for n_paths, dt, seed in ((1000, 0.05, 31), (777, 0.02, 32)):   # 777: a ragged last warp
        po, so, bo = oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, swp_a=sa, swp_b=sb, swp_K=sK,
                                     n_paths=n_paths, dt=dt, seed=seed, n_threads=16)
        pg, sg, bg = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=n_paths, dt=dt, seed=seed,
                                  prec="fp64")
        assert bg == bo
        nz = po > 0
        assert np.array_equal(nz, pg > 0)
        rel = np.abs(pg[nz] - po[nz]) / po[nz]
        print(f"MM MC FP64 against the oracle ({n_paths} paths, dt {dt}): max relative {rel.max():.3e}")
        assert rel.max() <= 1e-11
        assert np.max(np.abs(sg[nz] - so[nz]) / so[nz]) <= 1e-9


def test_mc_mm_fp32_against_the_oracle(gpu_lib):
    # the FP32 bar of the Hagan dynamics: 1e-5 relative above 1e-3 of the largest price, 1e-7 below
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    cf, ck, sa, sb, sK = _instruments(sk)
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    po, so, bo = oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, swp_a=sa, swp_b=sb, swp_K=sK,
                                 n_paths=4096, dt=0.01, seed=33, n_threads=16)
    pg, sg, bg = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=4096, dt=0.01, seed=33, prec="fp32")
    assert bg == bo == 0
    big = po > 1e-3 * po.max()
    rel = np.abs(pg[big] - po[big]) / po[big]
    print(f"MM MC FP32 against the oracle: max relative {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= 1e-5
    assert np.max(np.abs(pg[~big] - po[~big]), initial=0.0) <= 1e-7


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_mc_mm_zero_strike_instruments_are_the_floating_legs(gpu_lib, prec):
    # the floating legs P(0, T_a) - P(0, T_b) within 4.5 standard errors plus 1e-3 of the price (the
    # Euler bias at dt = 0.01); a dropped V in the drift moves them by several percent
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    P = sk.P
    M = sk.n_fwd
    sa, sb = np.array([0, 2, 4, 0]), np.array([13, 10, 13, 1])
    n = 1_000_000 if prec == "fp32" else 100_000
    pg, sg, bg = lib.mc_price(sk.T, P, model, np.arange(M), np.zeros(M), sa, sb, np.zeros(4), n_paths=n, dt=0.01,
                              seed=34, prec=prec)
    exact = np.concatenate([P[:M] - P[1:M + 1], [P[a] - P[b] for a, b in zip(sa, sb)]])
    z = (pg - exact) / sg
    print(f"MM MC {prec} zero-strike z-scores: {np.round(z, 2)}")
    assert bg == 0 and np.all(np.abs(pg - exact) <= 4.5 * sg + 1e-3 * exact)


def test_mc_mm_lognormal_limit_is_black(gpu_lib):
    # sigma = 0 (V stays 1), beta = 1, phi = 0: Black at alpha_i for every caplet
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    al = np.linspace(0.2, 0.4, M)
    m2 = dict(model, beta=1.0, sigma=np.zeros(M), alpha=al, phi=np.zeros(M))
    K = np.concatenate([F * 0.9, F * 1.1])
    cf = np.concatenate([np.arange(M), np.arange(M)])
    pg, sg, _ = lib.mc_price(sk.T, sk.P, m2, cf, K, n_paths=1_000_000, dt=0.01, seed=35, prec="fp32")
    bl = np.array([oracle.black_call(F[i], k, sk.T[i], al[i], tau[i] * sk.P[i + 1]) for i, k in zip(cf, K)])
    z = (pg - bl) / sg
    assert np.max(np.abs(z)) < 4.5, z


def test_mc_mm_vol_of_vol_fattens_the_tails(gpu_lib):
    # beta = 1, phi = 0, sigma = 0.8: far out-of-the-money caplets above Black at alpha_i
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    m2 = dict(model, beta=1.0, sigma=np.full(M, 0.8), alpha=np.full(M, 0.3), phi=np.zeros(M))
    K = F * 2.5
    pg, sg, _ = lib.mc_price(sk.T, sk.P, m2, np.arange(M), K, n_paths=1_000_000, dt=0.01, seed=36, prec="fp32")
    bl = np.array([oracle.black_call(F[i], K[i], sk.T[i], 0.3, tau[i] * sk.P[i + 1]) for i in range(M)])
    z = (pg[1:] - bl[1:]) / sg[1:]
    assert np.all(z > 4.5), z


def test_mc_mm_rejects_an_unknown_model(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk, model = _mm()
    with pytest.raises(lib.SabrLmmError, match="model"):
        lib.mc_price(sk.T, sk.P, dict(model, model=1), [0], [0.01], n_paths=128, dt=0.1, prec="fp64")


# ---------------------------------------------------------------- SA over the Monte Carlo objective
def _self_quoted(M=6, n_paths=2000, dt=0.05, seed=5):
    """Payer swaptions on the paper's first M forwards, quoted at the Black vols that reproduce the
    oracle's Mercurio & Morini Monte Carlo prices at the paper's eta1, lambda1."""
    from scipy.optimize import brentq
    sk, model = _mm()
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
    pr, _, _ = oracle.mc_price(om, m6, swp_a=sa, swp_b=sb, swp_K=sK, n_paths=n_paths, dt=dt, seed=seed, n_threads=16)
    qv = []
    for k in range(len(sa)):
        a, b = sa[k], sb[k]
        A = sum(tau[j] * P[j + 1] for j in range(a, b))
        S = (P[a] - P[b]) / A
        qv.append(brentq(lambda v: oracle.black_call(S, sK[k], T[a], v, A) - pr[k], 1e-4, 5.0, xtol=1e-15))
    return sk, om, m6, np.array(sa), np.array(sb), np.array(sK), np.array(qv)


def test_mc_mm_anneal_fp64_matches_the_oracle(gpu_lib):
    # the MM model's correlation has two parameters: eta1, lambda1 free, the other three slots fixed
    import paper_2408_01470_b300 as lib
    sk, om, m6, sa, sb, sK, qv = _self_quoted()
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    free = np.array([1, 1, 0, 0, 0])
    kw = dict(n_paths=2000, dt=0.05, mc_seed=5)
    ro = oracle.mc_anneal(om, m6, qv, lo, hi, free, 8, 3, 4, 0.7, 9, swp_a=sa, swp_b=sb, swp_K=sK,
                          n_threads=16, **kw)
    rg = lib.mc_anneal(sk.T[:7], sk.P[:7], m6, qv, lo, hi, free, 8, 3, 4, 0.7, 9, swp_start=sa, swp_end=sb,
                       swp_K=sK, prec="fp64", **kw)
    assert rg["T0"] == pytest.approx(ro["T0"], rel=1e-10)
    assert np.allclose(rg["trace_f"], ro["trace_f"], rtol=1e-9, atol=0)
    assert np.allclose(rg["trace_y"], ro["trace_x"], rtol=1e-12, atol=1e-15)
    assert np.allclose(rg["y_best"], ro["y_best"], rtol=1e-12, atol=1e-15)
    assert np.all(rg["y_best"][2:] == 0.5 * (lo + hi)[2:])
    assert rg["f_best"] == pytest.approx(ro["f_best"], rel=1e-9)


def test_mc_mm_anneal_fp32_recovers_the_quoting_point(gpu_lib):
    # FP32 paths: the search over (eta1, lambda1) ends far below its start, at a point whose oracle
    # f_s confirms it
    import paper_2408_01470_b300 as lib
    sk, om, m6, sa, sb, sK, qv = _self_quoted()
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    free = np.array([1, 1, 0, 0, 0])
    rg = lib.mc_anneal(sk.T[:7], sk.P[:7], m6, qv, lo, hi, free, 64, 12, 8, 0.7, 3, swp_start=sa, swp_end=sb,
                       swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5, prec="fp32")
    kw = dict(swp_a=sa, swp_b=sb, swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5)
    f_c = oracle.mc_objective(om, m6, 0.5 * (lo + hi), qv, **kw)
    f_o = oracle.mc_objective(om, m6, rg["y_best"], qv, **kw)
    print(f"MM MC anneal FP32: f_s {rg['f_best']:.3e} (oracle at the point {f_o:.3e}, box centre {f_c:.3e}), "
          f"y {rg['y_best'][:2]} (quoted at {m6['eta1']:.6f}, {m6['lambda1']:.6f})")
    assert rg["f_best"] <= 0.02 * f_c
    assert f_o <= 0.02 * f_c
