"""GPU-vs-oracle parity through the C-ABI (run on a B300: pytest -m gpu).

FP64: objective <= 1e-12 relative at points away from the optimum, model vols <= 1e-13 relative,
and the annealer's accept/reject trajectories identical on the same Philox stream.
FP32: feasibility per instrument equal to the oracle's (boundary rule in fp32_parity.py), the
search's own pricer compared per price (|dP| / vega in vol points, from sabr_lmm_residuals), model
vols per instrument, and the objective within 1e-4 relative at random points, at the generating
point and at the end points of FP32 searches.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth
from fp32_parity import (assert_feasibility_rule, assert_point_feasibility_rule, check_per_price, feasible,
                         objective_bound_at_noise_floor, residual_errors)

pytestmark = pytest.mark.gpu


def _markets(skel):
    """The same quotes for both sides: oracle model vols at the generating point plus noise."""
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(skel)
    gm = lib.Market(skel, vols)
    return om, gm, vols


def _ragged_caplets():
    sk = synth.caplet_term_structure(n_fwd=7, n_strikes=5)   # 35 caplets: one full warp + a tail of 3
    return sk


def _single_caplet():
    sk = synth.caplet_term_structure(n_fwd=3, n_strikes=1)
    keep = np.array([2])
    return sk.replace(cap_fwd=sk.cap_fwd[keep], cap_K=sk.cap_K[keep], noise=sk.noise[keep])


CASES = {
    "smile_2y": lambda: synth.smile_2y(),
    "smile_2y_paper": lambda: synth.smile_2y(formula=synth.FORMULA_PAPER),
    "caplets_20x15": lambda: synth.caplet_term_structure(),
    "caplets_20x15_paper": lambda: synth.caplet_term_structure(formula=synth.FORMULA_PAPER),
    "caplets_7x5_ragged": _ragged_caplets,
    "one_caplet": _single_caplet,
}


@pytest.mark.parametrize("name", list(CASES))
def test_objective_fp64_matches_oracle(gpu_lib, name):
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = synth.uniform_in_box(sk, 200, seed=7)
    X = np.vstack([X, sk.theta_true[None, :], sk.box_centre()[None, :]])
    f_gpu = gm.objective(X, "fp64").cpu().numpy()
    f_orc = om.objective_batch(X)
    fin = np.isfinite(f_orc)
    assert np.array_equal(fin, np.isfinite(f_gpu)), "feasibility must agree"
    # points far from the optimum: 1e-12 relative.  The generating point (row -2, residuals at
    # the noise level, where rounding of the prices is amplified by P / (P - P_mkt)) is judged by
    # its RMS error in vol units: 1e-9 vol points.
    far = fin.copy()
    far[-2] = False
    rel = np.abs(f_gpu[far] - f_orc[far]) / np.abs(f_orc[far])
    assert np.max(rel) <= 1e-12, np.max(rel)
    if fin[-2]:
        n = sk.n_instr
        assert abs(math.sqrt(f_gpu[-2] / n) - math.sqrt(f_orc[-2] / n)) * 100 <= 1e-9


@pytest.mark.parametrize("name", list(CASES))
def test_model_vols_fp64_match_oracle(gpu_lib, name):
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = synth.uniform_in_box(sk, 50, seed=8)
    v_gpu = gm.model_vols(X, "fp64").cpu().numpy()
    for i in range(X.shape[0]):
        v_orc = om.model_vols(X[i])
        ok = np.isfinite(v_orc) & (v_orc > 0)
        assert np.array_equal(ok, np.isfinite(v_gpu[i]))
        assert np.max(np.abs(v_gpu[i][ok] - v_orc[ok]) / v_orc[ok]) <= 1e-13


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15", "caplets_7x5_ragged"])
def test_model_vols_fp32_error_bound(gpu_lib, name):
    # FP32 pricing: per-quote vol error bounded by 2e-4 vol points (2e-6 in vol units); feasibility
    # per instrument equal to the oracle's (fp32_parity's boundary rule)
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 50, seed=9), sk.theta_true[None, :]])
    v32 = gm.model_vols(X, "fp32").cpu().numpy()
    worst = 0.0
    for i in range(X.shape[0]):
        v_orc = om.model_vols(X[i])
        assert_feasibility_rule(np.isfinite(v32[i]), v_orc, where=f"{name} point {i}")
        ok = feasible(v_orc) & np.isfinite(v32[i])
        worst = max(worst, float(np.max(np.abs(v32[i][ok] - v_orc[ok]), initial=0.0)) * 100.0)
    print(f"{name}: FP32 vol error max {worst:.3e} vol-pt")
    assert worst <= 2e-4


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15", "caplets_7x5_ragged", "caplets_20x15_paper"])
def test_residuals_fp32_per_price(gpu_lib, name):
    # the search's own FP32 pricer (packed pairs for the Hagan form), per price: |dP| / vega in vol
    # points against the FP64 oracle, at random points and at the generating point (the bars and
    # their derivation: fp32_parity.py)
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 40, seed=19), sk.theta_true[None, :]])
    err, mag = residual_errors(gm, om, X, "fp32")
    check_per_price(err, mag, -1, where=name)


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15", "caplets_7x5_ragged"])
def test_residuals_fp64_per_price(gpu_lib, name):
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 20, seed=20), sk.theta_true[None, :]])
    f, r = gm.residuals(X, "fp64")
    f, r = f.cpu().numpy(), r.cpu().numpy()
    for i in range(X.shape[0]):
        r_or, _ = om.residuals_jac(X[i])
        if r_or is None:
            assert not np.all(np.isfinite(r[i])) and not np.isfinite(f[i])
            continue
        # |dP| / vega from rounding order only: the price's rounding (~1e-16 P) over vega, with P /
        # vega of order one at most on these markets: 1e-13 in vol units (measured 8e-16)
        assert np.max(np.abs(r[i] - r_or)) <= 1e-13
        if i < X.shape[0] - 1:   # away from the noise floor
            assert f[i] == pytest.approx(np.sum(r_or * r_or), rel=1e-12)


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15", "caplets_7x5_ragged"])
def test_objective_fp32_relative(gpu_lib, name):
    # FP32 objective within 1e-4 relative of the oracle's at random points and at the generating
    # point (residuals at the noise floor); feasibility per point as the oracle's
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 100, seed=10), sk.theta_true[None, :]])
    f32 = gm.objective(X, "fp32").cpu().numpy()
    f64 = om.objective_batch(X)
    assert_point_feasibility_rule(f32, f64, om, X, where=name)
    fin = np.isfinite(f64) & np.isfinite(f32)
    fin[-1] = False
    rel = np.abs(f32[fin] - f64[fin]) / f64[fin]
    rel_gen = abs(f32[-1] - f64[-1]) / f64[-1]
    print(f"{name}: FP32 objective relative error max {rel.max():.3e} at random points, "
          f"{rel_gen:.3e} at the generating point")
    assert np.max(rel) <= 1e-4
    # at the generating point the residuals are the noise (0.02 vol-pt): the error bound that
    # follows from the per-price bar, and 1e-4 relative on the benchmark's 300-caplet market
    assert abs(f32[-1] - f64[-1]) <= objective_bound_at_noise_floor(f64[-1], sk.n_instr)
    if sk.n_instr >= 300:
        assert rel_gen <= 1e-4


@pytest.mark.parametrize("name,C,L,N,cool", [("smile_2y", 64, 100, 50, 0.9), ("caplets_20x15", 512, 20, 50, 0.95)])
def test_objective_fp32_at_annealed_end_points(gpu_lib, name, C, L, N, cool):
    # the final objective of an FP32 search (the value it reports at its best point) against the
    # oracle's objective at that point: 1e-4 relative
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    r = gm.anneal(C, L, N, cool, seed=29, prec="fp32")
    fo = om.objective(r["x_best"][0])
    rel = abs(r["f_best"][0] - fo) / fo
    print(f"{name}: final FP32 objective {r['f_best'][0]:.6e}, oracle {fo:.6e}, relative {rel:.2e}")
    assert rel <= 1e-4


def _anneal_both(sk, C, L, N, cool, seed, prec="fp64"):
    om, gm, _ = _markets(sk)
    r_o = om.anneal(C, L, N, cool, seed=seed, want_bits=True, want_chains=True, n_threads=8)
    r_g = gm.anneal(C, L, N, cool, seed=seed, prec=prec, record_accepts=True)
    return om, gm, r_o, r_g


def test_anneal_fp64_trajectory_identical_smile_full_schedule(gpu_lib):
    # the single-smile workload at its full schedule: 64 chains x 100 temperatures x 50 steps
    sk = synth.smile_2y()
    om, gm, r_o, r_g = _anneal_both(sk, 64, 100, 50, 0.9, seed=240801470)
    assert r_g["n_evals"] == r_o["n_evals"] == 64 * (100 * 50 + 1)
    assert r_g["T0"] == pytest.approx(r_o["T0"], rel=1e-12)
    diff = np.argwhere(r_g["bits"] != r_o["bits"])
    assert diff.size == 0, f"first differing (chain, level, step): {diff[:1]}"
    assert np.allclose(r_g["trace_f"][0], r_o["trace_f"], rtol=1e-11, atol=0)
    assert np.allclose(r_g["x_best"][0], r_o["x_best"], rtol=1e-12, atol=1e-15)
    assert r_g["f_best"][0] == pytest.approx(r_o["f_best"], rel=1e-11)


def test_anneal_fp64_trajectory_identical_caplets(gpu_lib):
    sk = synth.caplet_term_structure()
    om, gm, r_o, r_g = _anneal_both(sk, 48, 4, 8, 0.95, seed=3)
    diff = np.argwhere(r_g["bits"] != r_o["bits"])
    assert diff.size == 0, f"first differing (chain, level, step): {diff[:1]}"
    assert np.allclose(r_g["trace_f"][0], r_o["trace_f"], rtol=1e-11, atol=0)
    assert np.allclose(r_g["x_best"][0], r_o["x_best"], rtol=1e-12, atol=1e-15)


def test_anneal_ragged_chain_count_and_graph_replay(gpu_lib):
    # 37 chains (not a multiple of the CTA's warps), graph capture on, same trajectories
    sk = synth.smile_2y()
    om, gm, _ = _markets(sk)
    r_o = om.anneal(37, 6, 7, 0.8, seed=5, want_bits=True)
    import torch
    s = torch.cuda.Stream()
    plan = gm.anneal_prepare(37, 6, 7, 0.8, seed=5, use_graph=True, stream=s)
    for _ in range(2):   # replaying the graph twice gives the same search
        plan.launch(stream=s)
        r = plan.fetch()
        assert np.allclose(r["trace_f"][0], r_o["trace_f"], rtol=1e-11)
        assert np.allclose(r["x_best"][0], r_o["x_best"], rtol=1e-12, atol=1e-15)


def test_anneal_fp32_reaches_fp64_quality(gpu_lib):
    sk = synth.smile_2y()
    om, gm, _ = _markets(sk)
    r64 = gm.anneal(64, 100, 50, 0.9, seed=11, prec="fp64")
    r32 = gm.anneal(64, 100, 50, 0.9, seed=11, prec="fp32")
    # same search up to FP32 rounding: the final RMSEs agree to 1% of the FP64 value
    assert r32["rmse_volpt"][0] == pytest.approx(r64["rmse_volpt"][0], rel=1e-2)
    assert math.isfinite(r32["f_best"][0])


def test_load_market_rejects_bad_input(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    bad = sk.replace(cap_K=-sk.cap_K)
    with pytest.raises(lib.SabrLmmError) as e:
        lib.Market(bad, np.full(sk.n_cap, 0.2))
    assert e.value.status == 1 and "cap_K" in str(e.value)


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15"])
def test_anneal_fp32_same_search_at_every_cta_size(gpu_lib, name):
    # the FP32 level kernel comes in 4-chain CTAs and in one CTA of up to 28 chains per SM; a chain
    # is one warp either way, so every CTA size gives the same search bit for bit (100 chains: the
    # last 28-chain CTA is partial)
    sk = CASES[name]()
    om, gm, _ = _markets(sk)
    runs = [gm.anneal(100, 4, 12, 0.9, seed=13, prec="fp32", record_accepts=True, warps_per_block=w)
            for w in (1, 4, 7, 28, 0)]
    for r in runs[1:]:
        assert np.array_equal(r["bits"], runs[0]["bits"])
        assert np.array_equal(r["trace_f"], runs[0]["trace_f"])
        assert np.array_equal(r["x_best"], runs[0]["x_best"])
        assert np.array_equal(r["f_best"], runs[0]["f_best"])


def test_anneal_fp64_more_than_four_chains_per_cta_is_capped(gpu_lib):
    # FP64 (128 registers a thread) keeps 4-chain CTAs whatever is asked; the search is unchanged
    sk = synth.smile_2y()
    om, gm, _ = _markets(sk)
    r4 = gm.anneal(40, 3, 6, 0.9, seed=17, prec="fp64", record_accepts=True, warps_per_block=4)
    r28 = gm.anneal(40, 3, 6, 0.9, seed=17, prec="fp64", record_accepts=True, warps_per_block=28)
    assert np.array_equal(r4["bits"], r28["bits"])
    assert np.array_equal(r4["x_best"], r28["x_best"])
