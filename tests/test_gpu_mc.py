"""The Monte Carlo pricer (Hagan SABR/LIBOR model under the spot measure; Section 3, Table
tab:haganMCpricer) on the GPU, through the C-ABI.

FP64: the same paths as the oracle (the same Philox4x32-10 counters, Box-Muller normals, time grid
and correlation factor), so every price and standard error agrees to rounding order (1e-12
relative).  FP32: the same normals up to the 24-bit uniforms, the path arithmetic, the payoffs and
their sums over a warp's 32 paths in FP32, the warp sums accumulated in FP64; bar derived below.  At production path counts the no-arbitrage pins of the oracle
(zero-strike floating legs, the lognormal LMM's Black prices) hold for the device's own paths.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    return synth.paper_hagan_mc_model(os.path.join(GOLDEN, "paper_euribor_20111121.txt"),
                                      os.path.join(GOLDEN, "paper_mm_20111121.txt"),
                                      os.path.join(GOLDEN, "paper_hagan_mc_20111121.txt"))


def _instruments(sk):
    # the 117 caplets of the paper's smiles and payer swaptions on the same tenor structure (expiries
    # on forwards 0..8, ends up to the last forward, strikes around the forward swap rate)
    _, model, cf, ck, _ = _paper()
    P, T = sk.P, sk.T
    sa, sb, sK = [], [], []
    for a in (0, 2, 4, 8):
        for b in (a + 1, a + 4, 13):
            if b <= 13 and b > a:
                A = sum((T[j + 1] - T[j]) * P[j + 1] for j in range(a, b))
                S = (P[a] - P[b]) / A
                for m in (0.8, 1.0, 1.25):
                    sa.append(a); sb.append(b); sK.append(S * m)
    return model, cf, ck, np.array(sa), np.array(sb), np.array(sK)


def test_mc_fp64_paths_match_the_oracle(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = _paper()[0]
    model, cf, ck, sa, sb, sK = _instruments(sk)
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    for n_paths, dt, seed in ((1000, 0.05, 11), (777, 0.02, 12)):   # 777: a ragged last warp
        po, so, bo = oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, swp_a=sa, swp_b=sb, swp_K=sK,
                                     n_paths=n_paths, dt=dt, seed=seed, n_threads=16)
        pg, sg, bg = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=n_paths, dt=dt, seed=seed,
                                  prec="fp64")
        assert bg == bo
        nz = po > 0
        assert np.array_equal(nz, pg > 0)
        # a mean of non-negative deflated payoffs: rounding order only (per path ~1e-15 relative,
        # amplified through ~700 steps of the path recursion)
        assert np.max(np.abs(pg[nz] - po[nz]) / po[nz]) <= 1e-11, np.max(np.abs(pg[nz] - po[nz]) / po[nz])
        assert np.max(np.abs(sg[nz] - so[nz]) / so[nz]) <= 1e-9


def test_mc_fp32_against_the_oracle(gpu_lib):
    # FP32 paths: the uniforms keep 24 of their 32 bits (normals differ by ~1e-7), every state
    # update rounds to 6e-8 of the state, ~700 steps: the forwards at their fixings carry ~1e-6 of
    # themselves, a price ~1e-6 / (moneyness distance) of itself, and the means over paths average
    # these errors; a warp's FP32 payoff sum adds ~1e-7 of itself (measured 2.7e-6 relative at most
    # in all); bar 1e-5 relative on every price above 1e-3 of the largest, 1e-7 absolute below
    import paper_2408_01470_b300 as lib
    sk = _paper()[0]
    model, cf, ck, sa, sb, sK = _instruments(sk)
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    po, so, bo = oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, swp_a=sa, swp_b=sb, swp_K=sK,
                                 n_paths=4096, dt=0.01, seed=13, n_threads=16)
    pg, sg, bg = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=4096, dt=0.01, seed=13, prec="fp32")
    assert bg == bo == 0
    big = po > 1e-3 * po.max()
    rel = np.abs(pg[big] - po[big]) / po[big]
    print(f"MC FP32 against the oracle: max relative {rel.max():.3e}, median {np.median(rel):.3e}, "
          f"max absolute below {np.max(np.abs(pg[~big] - po[~big]), initial=0.0):.3e}")
    assert rel.max() <= 1e-5
    assert np.max(np.abs(pg[~big] - po[~big]), initial=0.0) <= 1e-7


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_mc_zero_strike_instruments_are_the_floating_legs(gpu_lib, prec):
    # no-arbitrage, at the device's own production path counts: within 4.5 standard errors plus the
    # Euler scheme's discretisation bias at dt = 0.01, allowed up to 1e-3 of the price (a dropped or
    # mis-signed drift term moves the floating legs by several percent)
    import paper_2408_01470_b300 as lib
    sk, model, _, _, _ = _paper()
    P = sk.P
    M = sk.n_fwd
    sa, sb = np.array([0, 2, 4, 0]), np.array([13, 10, 13, 1])
    n = 1_000_000 if prec == "fp32" else 100_000
    pg, sg, bg = lib.mc_price(sk.T, P, model, np.arange(M), np.zeros(M), sa, sb, np.zeros(4), n_paths=n, dt=0.01,
                              seed=21, prec=prec)
    exact = np.concatenate([P[:M] - P[1:M + 1], [P[a] - P[b] for a, b in zip(sa, sb)]])
    z = (pg - exact) / sg
    print(f"MC {prec} zero-strike z-scores: {np.round(z, 2)}, relative {np.round((pg - exact) / exact, 5)}")
    assert bg == 0 and np.all(np.abs(pg - exact) <= 4.5 * sg + 1e-3 * exact)


def test_mc_lognormal_limit_is_black(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk, model, _, _, _ = _paper()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    M = sk.n_fwd
    tau = np.diff(sk.T)
    al = np.linspace(0.2, 0.4, M)
    m2 = dict(model, beta=1.0, sigma=np.zeros(M), alpha=al, phi=np.zeros(M))
    K = np.concatenate([F * 0.9, F * 1.1])
    cf = np.concatenate([np.arange(M), np.arange(M)])
    pg, sg, _ = lib.mc_price(sk.T, sk.P, m2, cf, K, n_paths=1_000_000, dt=0.01, seed=22, prec="fp32")
    bl = np.array([oracle.black_call(F[i], k, sk.T[i], al[i], tau[i] * sk.P[i + 1]) for i, k in zip(cf, K)])
    z = (pg - bl) / sg
    assert np.max(np.abs(z)) < 4.5, z


def test_mc_grid_and_plan_replay(gpu_lib):
    # a persistent grid of 3 CTAs gives the paths of the default grid (FP64 sums in another order),
    # and a plan launched twice gives the same prices
    import torch
    import paper_2408_01470_b300 as lib
    sk = _paper()[0]
    model, cf, ck, sa, sb, sK = _instruments(sk)
    p1, s1, _ = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=5000, dt=0.05, seed=5, prec="fp64")
    p2, s2, _ = lib.mc_price(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=5000, dt=0.05, seed=5, prec="fp64",
                             grid=3)
    nz = p1 > 0
    assert np.allclose(p2[nz], p1[nz], rtol=1e-13, atol=0)
    plan = lib.McPlan(sk.T, sk.P, model, cf, ck, sa, sb, sK, n_paths=5000, dt=0.05, seed=5, prec="fp64")
    out = []
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        out.append(plan.price.cpu().numpy().copy())
    assert np.array_equal(out[0], out[1])
    assert np.allclose(out[0][nz], p1[nz], rtol=1e-13, atol=0)


def test_mc_rejects_bad_input(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk, model, cf, ck, _ = _paper()
    with pytest.raises(lib.SabrLmmError) as e:
        lib.mc_price(sk.T, sk.P, model, cf, ck, n_paths=0)
    assert e.value.status == 1 and "n_paths" in str(e.value)
    with pytest.raises(lib.SabrLmmError) as e:
        lib.mc_price(sk.T, sk.P, dict(model, eta1=1.5), cf, ck, n_paths=10)
    assert e.value.status == 1 and "eta1" in str(e.value)
    sk20 = synth.caplet_term_structure(n_fwd=20)
    m20 = dict(model, alpha=np.full(20, 0.2), sigma=np.full(20, 0.3), phi=np.full(20, -0.3))
    with pytest.raises(lib.SabrLmmError) as e:
        lib.mc_price(sk20.T, sk20.P, m20, [17], [0.03], n_paths=10)
    assert e.value.status == 5 and "16 forwards" in str(e.value)


def test_mc_sixteen_forwards_match_the_oracle(gpu_lib):
    # the largest tenor structure the pricer takes: every interval's step code, down to 16 alive
    # forwards, against the oracle's paths (FP64) and within the FP32 bar
    import paper_2408_01470_b300 as lib
    sk = synth.caplet_term_structure(n_fwd=16)
    M = 16
    m16 = dict(M=M, beta=0.5, eta1=0.8, lambda1=0.5, eta2=0.9, lambda2=0.3, lambda3=0.1,
               alpha=np.linspace(0.05, 0.08, M), sigma=np.linspace(0.4, 0.25, M), phi=np.linspace(-0.4, 0.2, M))
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    cf = np.repeat(np.arange(M), 2)
    ck = np.concatenate([F[i] * np.array([0.9, 1.2]) for i in range(M)])
    sa, sb = np.array([0, 3, 7, 12]), np.array([16, 10, 16, 16])
    P, T = sk.P, sk.T
    sK = np.array([(P[a] - P[b]) / sum((T[j + 1] - T[j]) * P[j + 1] for j in range(a, b)) for a, b in zip(sa, sb)])
    po, so, bo = oracle.mc_price(om, m16, cap_fwd=cf, cap_K=ck, swp_a=sa, swp_b=sb, swp_K=sK, n_paths=1000, dt=0.1,
                                 seed=41, n_threads=16)
    pg, sg, bg = lib.mc_price(T, P, m16, cf, ck, sa, sb, sK, n_paths=1000, dt=0.1, seed=41, prec="fp64")
    assert bg == bo
    nz = po > 0
    assert np.array_equal(nz, pg > 0)
    assert np.max(np.abs(pg[nz] - po[nz]) / po[nz]) <= 1e-11
    p32, _, b32 = lib.mc_price(T, P, m16, cf, ck, sa, sb, sK, n_paths=1000, dt=0.1, seed=41, prec="fp32")
    big = po > 1e-3 * po.max()
    rel = np.abs(p32[big] - po[big]) / po[big]
    print(f"MC 16 forwards: FP64 max relative {np.max(np.abs(pg[nz] - po[nz]) / po[nz]):.2e}, FP32 {rel.max():.2e}")
    assert b32 == bo and rel.max() <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mc_many_instruments_shrink_the_cta(gpu_lib, prec):
    # 4096 caplets (the limit): the per-warp sums of a 512- or 128-path CTA would not fit in shared
    # memory, so the plan takes 64-path CTAs; the prices are still the oracle's
    import paper_2408_01470_b300 as lib
    sk, model, _, _, _ = _paper()
    om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
    F = om.info()["F"]
    rng = np.random.default_rng(7)
    cf = rng.integers(0, sk.n_fwd, 4096)
    ck = F[cf] * rng.uniform(0.6, 1.6, 4096)
    po, _, bo = oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, n_paths=1024, dt=0.1, seed=43, n_threads=16)
    pg, _, bg = lib.mc_price(sk.T, sk.P, model, cf, ck, n_paths=1024, dt=0.1, seed=43, prec=prec)
    assert bg == bo == 0
    big = po > 1e-3 * po.max()
    rel = np.abs(pg[big] - po[big]) / po[big]
    assert rel.max() <= (1e-11 if prec == "fp64" else 1e-5), rel.max()
    assert np.max(np.abs(pg[~big] - po[~big]), initial=0.0) <= (1e-15 if prec == "fp64" else 1e-7)


# ---------------------------------------------------------------- SA over the Monte Carlo objective
def _self_quoted(M=6, n_paths=2000, dt=0.05, seed=5):
    """Payer swaptions on the paper's first M forwards, quoted at the Black vols that reproduce the
    oracle's Monte Carlo prices at the paper's correlation parameters (root-finding on Black)."""
    from scipy.optimize import brentq
    sk, model, _, _, _ = _paper()
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


def test_mc_anneal_fp64_matches_the_oracle(gpu_lib):
    # the same search on both sides: FP64 paths equal to the oracle's (f_s to rounding order), the
    # same proposals and Metropolis decisions, so the same trace and result
    import paper_2408_01470_b300 as lib
    sk, om, m6, sa, sb, sK, qv = _self_quoted()
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    kw = dict(n_paths=2000, dt=0.05, mc_seed=5)
    ro = oracle.mc_anneal(om, m6, qv, lo, hi, np.ones(5), 8, 3, 4, 0.7, 9, swp_a=sa, swp_b=sb, swp_K=sK,
                          n_threads=16, **kw)
    T6, P6 = sk.T[:7], sk.P[:7]
    rg = lib.mc_anneal(T6, P6, m6, qv, lo, hi, np.ones(5), 8, 3, 4, 0.7, 9, swp_start=sa, swp_end=sb, swp_K=sK,
                       prec="fp64", **kw)
    assert rg["T0"] == pytest.approx(ro["T0"], rel=1e-10)
    assert np.allclose(rg["trace_f"], ro["trace_f"], rtol=1e-9, atol=0)
    assert np.allclose(rg["trace_y"], ro["trace_x"], rtol=1e-12, atol=1e-15)
    assert np.allclose(rg["y_best"], ro["y_best"], rtol=1e-12, atol=1e-15)
    assert rg["f_best"] == pytest.approx(ro["f_best"], rel=1e-9)
    assert rg["n_evals"] == 8 * 3 * 4 + 1


def test_mc_anneal_fp32_descends(gpu_lib):
    # FP32 paths, more chains and levels: the search ends far below its start and at a point the
    # oracle's f_s (FP64, the same paths up to FP32 rounding) confirms
    import paper_2408_01470_b300 as lib
    sk, om, m6, sa, sb, sK, qv = _self_quoted()
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    rg = lib.mc_anneal(sk.T[:7], sk.P[:7], m6, qv, lo, hi, np.ones(5), 64, 12, 8, 0.7, 3, swp_start=sa, swp_end=sb,
                       swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5, prec="fp32")
    kw = dict(swp_a=sa, swp_b=sb, swp_K=sK, n_paths=2000, dt=0.05, mc_seed=5)
    f_c = oracle.mc_objective(om, m6, 0.5 * (lo + hi), qv, **kw)
    f_o = oracle.mc_objective(om, m6, rg["y_best"], qv, **kw)
    print(f"MC anneal FP32: f_s {rg['f_best']:.3e} (oracle at the point {f_o:.3e}, box centre {f_c:.3e}), "
          f"{rg['n_evals']} evaluations in {rg['seconds']:.2f} s")
    assert rg["f_best"] <= 0.02 * f_c
    assert f_o <= 0.02 * f_c
