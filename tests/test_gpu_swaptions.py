"""GPU-vs-oracle parity for markets with swaptions (S3 pair integrals, S5 quadratic forms, S6
swaption pricing), through the C-ABI: FP64 objective within 1e-12 relative away from the optimum,
FP64 vols within 1e-12 (see the prefix-sum note below), identical FP64 accept/reject
trajectories, FP32 vols within 1e-3 vol-pt (median 1e-4), the FP32 RMS-equivalent objective
within 1e-4 vol-pt plus 1.5e-5 of itself.  Markets: the 40-forward joint workload (300 caplets,
700 swaptions), a small joint market, a swaptions-only market and two members of the uneven batch
(random windows and expiry groups).
"""
import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

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


@pytest.mark.parametrize("name", ["joint_40f_300c_700s", "batch_member_3"])
def test_swaption_vols_fp32_error_bound(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 6, seed=23), sk.theta_true[None, :]])
    v32 = gm.model_vols(X, "fp32").cpu().numpy()
    for i in range(X.shape[0]):
        v_orc = om.model_vols(X[i])
        ok = np.isfinite(v_orc) & (v_orc > 0) & np.isfinite(v32[i])
        assert ok.sum() >= 0.9 * len(ok)
        err = np.abs(v32[i][ok] - v_orc[ok]) * 100.0
        # FP32 swaption vols: the window integrals are differences of FP32 prefix sums along the
        # diagonals (cancelling by up to (offset + window)/window) and rho_S = V3/V1; measured over
        # 64 random points on three markets: median 1.5e-5, 90th percentile 3.7e-5, worst 5.2e-4
        # vol-pt.  Caplets keep the caplet bar.
        assert np.max(err) <= 1e-3
        assert np.median(err) <= 1e-4


def test_swaption_objective_fp32_rms_equivalent(gpu_lib):
    sk = CASES["joint_40f_300c_700s"]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 16, seed=24), sk.theta_true[None, :]])
    f32 = gm.objective(X, "fp32").cpu().numpy()
    f64 = om.objective_batch(X, n_threads=8)
    fin = np.isfinite(f64) & np.isfinite(f32)
    n = sk.n_instr
    d = np.abs(np.sqrt(f32[fin] / n) - np.sqrt(f64[fin] / n)) * 100.0
    rms = np.sqrt(f64[fin] / n) * 100.0
    # In FP32 the window integrals are differences of prefix sums along the diagonals, which
    # cancel by up to ~ (offset + window) / window, so a swaption vol carries a relative error of a
    # few 1e-6 and the RMS-equivalent objective moves by that fraction of itself (measured up to
    # 8.2e-6 at random points whose RMS error is hundreds of vol-pt); near the optimum the bar is
    # the absolute 1e-4 vol-pt
    assert np.all(d <= 1e-4 + 1.5e-5 * rms), np.max(d - 1.5e-5 * rms)
    assert d[-1] <= 1e-4                       # the generating point


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
    assert om.objective(r["x_best"][0]) == pytest.approx(r["f_best"][0], rel=1e-3)


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
