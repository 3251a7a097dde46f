"""The pair-integral Grams of the swaption forms on the tensor cores (tcgen05, BF16 split).

Y = hi + lo with two bf16 terms keeps 16 significant bits per element, so the Grams, the swap-rate
SABR parameters and the swaption vols carry ~1e-5 relative error: the bars below are stated in vol
points against the FP64 oracle and against the FP32 ALU contraction.
"""
import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth
from fp32_parity import assert_feasibility_rule, assert_point_feasibility_rule, feasible

pytestmark = pytest.mark.gpu

CASES = {
    "joint_40f_300c_700s": lambda: synth.joint_caplet_swaption(),
    "joint_small": lambda: synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4)),
}


def _markets(sk):
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(sk)
    return om, lib.Market(sk, vols)


@pytest.mark.parametrize("name", list(CASES))
def test_bf16x3_swaption_vols_against_oracle(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 6, seed=41), sk.theta_true[None, :]])
    vt = gm.model_vols(X, "bf16x3").cpu().numpy()
    v32 = gm.model_vols(X, "fp32").cpu().numpy()
    worst, worst32 = 0.0, 0.0
    for i in range(X.shape[0]):
        vo = om.model_vols(X[i])
        assert_feasibility_rule(np.isfinite(vt[i]), vo, where=f"{name} bf16x3 point {i}")
        assert_feasibility_rule(np.isfinite(v32[i]), vo, where=f"{name} fp32 point {i}")
        ok = feasible(vo) & np.isfinite(vt[i]) & np.isfinite(v32[i])
        worst = max(worst, np.max(np.abs(vt[i][ok] - vo[ok])) * 100)
        worst32 = max(worst32, np.max(np.abs(v32[i][ok] - vo[ok])) * 100)
    print(f"{name}: bf16x3 max vol error {worst:.3e} vol-pt, fp32 {worst32:.3e} vol-pt")
    assert worst <= 1e-3          # measured 3.2e-4 (joint), 8.6e-5 (small)


def test_bf16x3_objective_close_to_fp32(gpu_lib):
    sk = CASES["joint_40f_300c_700s"]()
    om, gm = _markets(sk)
    X = np.vstack([synth.uniform_in_box(sk, 16, seed=42), sk.theta_true[None, :]])
    ft = gm.objective(X, "bf16x3").cpu().numpy()
    f64 = om.objective_batch(X, n_threads=8)
    assert_point_feasibility_rule(ft, f64, om, X, where="bf16x3")
    fin = np.isfinite(f64) & np.isfinite(ft)
    n = sk.n_instr
    d = np.abs(np.sqrt(ft[fin] / n) - np.sqrt(f64[fin] / n)) * 100.0
    print(f"bf16x3 RMS-equivalent objective error {np.max(d):.3e} vol-pt")
    assert np.max(d) <= 3e-4      # measured 6.3e-5


def test_bf16x3_anneal_runs_and_improves(gpu_lib):
    sk = CASES["joint_small"]()
    om, gm = _markets(sk)
    r = gm.anneal(256, 6, 16, 0.9, seed=5, prec="bf16x3")
    assert np.isfinite(r["f_best"][0]) and r["f_best"][0] < om.objective(sk.box_centre())
    assert om.objective(r["x_best"][0]) == pytest.approx(r["f_best"][0], rel=2e-2)


def test_precision_value_2_is_rejected(gpu_lib):
    # the enum has no TF32 split form: the value 2 is not a precision of the library
    import paper_2408_01470_b300 as lib
    sk = CASES["joint_small"]()
    om, gm = _markets(sk)
    with pytest.raises(lib.SabrLmmError) as e:
        gm.objective(sk.theta_true[None, :], 2)
    assert e.value.status == 1
