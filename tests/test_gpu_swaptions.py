"""GPU-vs-oracle parity for markets with swaptions (S3 pair integrals, S5 quadratic forms, S6
swaption pricing), through the C-ABI: FP64 objective within 1e-12 relative away from the optimum,
FP64 vols within 1e-12 (see the prefix-sum note below), identical FP64 accept/reject
trajectories; FP32 vols within 2e-4 vol-pt, per-price errors (|dP| / vega of the search's own
pricer) within the bars of fp32_parity.py, feasibility as the oracle's, and the FP32 objective
within 1e-4 relative.  Markets: the 40-forward joint workload (300 caplets, 700 swaptions), a small
joint market, a swaptions-only market and two members of the uneven batch (random windows and
expiry groups).
"""
import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth
from fp32_parity import (assert_feasibility_rule, assert_point_feasibility_rule, check_per_price, feasible,
                         objective_bound_at_noise_floor, residual_errors)

pytestmark = pytest.mark.gpu


def _swaptions_only():
    sk = synth.joint_caplet_swaption(n_fwd=24, expiries=(1, 2, 4, 6), tenors=(1, 3, 5), swp_m=(-0.3, 0.0, 0.3))
    keep = np.arange(sk.n_cap, sk.n_instr)
    return sk.replace(cap_fwd=np.zeros(0, np.int32), cap_K=np.zeros(0), noise=sk.noise[keep])


CASES = {
    "joint_40f_300c_700s": lambda: synth.joint_caplet_swaption(),
    "joint_small": lambda: synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4)),
    "swaptions_only": _swaptions_only,
    "batch_member_3": lambda: synth.batch_market(3),
    "batch_member_11": lambda: synth.batch_market(11),
}


def _markets(sk):
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(sk)
    return om, lib.Market(sk, vols)


@pytest.mark.parametrize("name", list(CASES))
def test_swaption_objective_fp64_matches_oracle(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    n = 24 if sk.n_swp > 300 else 120
    X = synth.uniform_in_box(sk, n, seed=21)
    f_gpu = gm.objective(X, "fp64").cpu().numpy()
    f_orc = om.objective_batch(X, n_threads=8)
    fin = np.isfinite(f_orc)
    assert np.array_equal(fin, np.isfinite(f_gpu))
    rel = np.abs(f_gpu[fin] - f_orc[fin]) / np.abs(f_orc[fin])
    assert np.max(rel) <= 1e-12, np.max(rel)


@pytest.mark.parametrize("name", list(CASES))
def test_swaption_vols_fp64_match_oracle(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 6, seed=22), sk.theta_true[None, :]])
    v_gpu = gm.model_vols(X, "fp64").cpu().numpy()
    for i in range(X.shape[0]):
        v_orc = om.model_vols(X[i])
        ok = np.isfinite(v_orc) & (v_orc > 0)
        assert np.array_equal(ok, np.isfinite(v_gpu[i]))
        # X_ij(T_E) comes from differences of prefix sums taken from panel 0; a short window far
        # along a diagonal loses a factor ~ offset/length of the window: 1e-12, not 1e-13
        assert np.max(np.abs(v_gpu[i][ok] - v_orc[ok]) / v_orc[ok]) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_swaption_vols_fp32_error_bound(gpu_lib, name):
    # FP32 vols (caplets and swaptions) within 2e-4 vol-pt of the oracle, the caplet bar; every
    # instrument's feasibility as the oracle's (boundary rule in fp32_parity.py)
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 12, seed=23), sk.theta_true[None, :]])
    v32 = gm.model_vols(X, "fp32").cpu().numpy()
    errs = []
    for i in range(X.shape[0]):
        v_orc = om.model_vols(X[i])
        assert_feasibility_rule(np.isfinite(v32[i]), v_orc, where=f"{name} point {i}")
        ok = feasible(v_orc) & np.isfinite(v32[i])
        errs.append(np.abs(v32[i][ok] - v_orc[ok]) * 100.0)
    err = np.concatenate(errs)
    print(f"{name}: FP32 vol error max {err.max():.3e} p99 {np.quantile(err, 0.99):.3e} "
          f"median {np.median(err):.3e} vol-pt")
    assert err.max() <= 2e-4


@pytest.mark.parametrize("name", list(CASES))
def test_swaption_residuals_fp32_per_price(gpu_lib, name):
    # the search's own FP32 pricer (packed pairs of caplets and swaptions), per price |dP| / vega
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 8, seed=25), sk.theta_true[None, :]])
    err, mag = residual_errors(gm, om, X, "fp32")
    check_per_price(err, mag, -1, where=name)


@pytest.mark.parametrize("name", ["joint_40f_300c_700s", "batch_member_3"])
def test_swaption_objective_fp32_relative(gpu_lib, name):
    # FP32 objective within 1e-4 relative of the oracle at random points and at the generating point
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 16, seed=24), sk.theta_true[None, :]])
    f32 = gm.objective(X, "fp32").cpu().numpy()
    f64 = om.objective_batch(X, n_threads=8)
    assert_point_feasibility_rule(f32, f64, om, X, where=name)
    fin = np.isfinite(f64) & np.isfinite(f32)
    rel = np.abs(f32[fin] - f64[fin]) / f64[fin]
    print(f"{name}: FP32 objective relative error max {rel.max():.3e}, generating point {rel[-1]:.3e}")
    assert np.max(rel) <= 1e-4
    assert abs(f32[-1] - f64[-1]) <= objective_bound_at_noise_floor(f64[-1], sk.n_instr)


def test_swaption_objective_fp32_at_annealed_end_point(gpu_lib):
    sk = CASES["joint_small"]()
    om, gm = _markets(sk)
    r = gm.anneal(512, 10, 20, 0.9, seed=31, prec="fp32")
    fo = om.objective(r["x_best"][0])
    rel = abs(r["f_best"][0] - fo) / fo
    print(f"joint_small: final FP32 objective {r['f_best'][0]:.6e}, oracle {fo:.6e}, relative {rel:.2e}")
    assert rel <= 1e-4


def test_swaption_anneal_fp64_trajectory_identical(gpu_lib):
    sk = CASES["joint_small"]()
    om, gm = _markets(sk)
    r_o = om.anneal(24, 3, 6, 0.95, seed=9, want_bits=True, n_threads=8)
    r_g = gm.anneal(24, 3, 6, 0.95, seed=9, prec="fp64", record_accepts=True)
    diff = np.argwhere(r_g["bits"] != r_o["bits"])
    assert diff.size == 0, f"first differing (chain, level, step): {diff[:1]}"
    assert np.allclose(r_g["trace_f"][0], r_o["trace_f"], rtol=1e-11, atol=0)
    assert np.allclose(r_g["x_best"][0], r_o["x_best"], rtol=1e-12, atol=1e-15)


def test_swaption_anneal_fp32_runs_and_improves(gpu_lib):
    sk = CASES["joint_small"]()
    om, gm = _markets(sk)
    r = gm.anneal(256, 8, 20, 0.9, seed=5, prec="fp32")
    f0 = om.objective(sk.box_centre())
    assert np.isfinite(r["f_best"][0]) and r["f_best"][0] < f0
    # the returned point is scored consistently by the oracle
    assert om.objective(r["x_best"][0]) == pytest.approx(r["f_best"][0], rel=1e-4)


def test_market_info_geometry(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.joint_caplet_swaption()
    gm = lib.Market(sk, np.full(sk.n_instr, 0.2))
    d = gm.info()
    assert (d["n_fwd"], d["n_cap"], d["n_swp"]) == (40, 300, 700)
    assert d["n_swap"] == len(set(zip(sk.swp_start.tolist(), sk.swp_end.tolist()))) == 100
    # panels up to the last expiry (10y = 20) plus the widest offset inside a window (19)
    assert d["n_panels"] == 39 and 1 <= d["n_diag"] <= 20 and d["max_window"] <= 20
    assert 0 < d["smem_fp32"] < d["smem_fp64"] <= 227 * 1024
    assert d["batch_ctas_per_sm_fp32"] >= d["batch_ctas_per_sm_fp64"] >= 1
    cap = synth.caplet_term_structure()
    c = lib.Market(cap, np.full(cap.n_instr, 0.2)).info()
    assert (c["n_fwd"], c["n_cap"], c["n_swp"], c["n_swap"]) == (20, 300, 0, 0)
