"""The hand-written adjoint (S9) and the Levenberg-Marquardt polish (S10), through the C-ABI.

Adjoint: FP64 gradient against the oracle's forward-mode dual numbers (an independent route) and
against central differences of the GPU objective; FP32 gradient against the oracle within the
FP32 pricing error.  LM: recovery of the generating point on noise-free quotes, agreement with the
oracle's LM, and the annealer's top-k polish.
"""
import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu

CASES = {
    "smile_2y": lambda: synth.smile_2y(),
    "smile_2y_paper": lambda: synth.smile_2y(formula=synth.FORMULA_PAPER),
    "caplets_20x15": lambda: synth.caplet_term_structure(),
    "caplets_20x15_paper": lambda: synth.caplet_term_structure(formula=synth.FORMULA_PAPER),
    "caplets_7x5": lambda: synth.caplet_term_structure(n_fwd=7, n_strikes=5),
}


def _markets(sk):
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(sk)
    return om, lib.Market(sk, vols)


def _points(sk, n, seed):
    X = synth.uniform_in_box(sk, n, seed=seed)
    if sk.model == synth.MODEL_REBONATO_LMM:
        X = 0.5 * (X + sk.theta_true[None, :])   # keep the vols in a sensible range
    return X


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_fp64_matches_oracle_dual_gradient(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = _points(sk, 40, seed=31)
    f, G = gm.objective_grad(X, "fp64")
    f, G = f.cpu().numpy(), G.cpu().numpy()
    for i in range(X.shape[0]):
        fo, go = om.objective_grad(X[i])
        if not np.isfinite(fo):
            assert not np.isfinite(f[i])
            continue
        assert f[i] == pytest.approx(fo, rel=1e-12)
        scale = np.max(np.abs(go))
        assert np.max(np.abs(G[i] - go)) <= 1e-9 * scale, (i, G[i], go)


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15"])
def test_adjoint_fp64_matches_central_differences(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = _points(sk, 4, seed=32)
    _, G = gm.objective_grad(X, "fp64")
    G = G.cpu().numpy()
    P = sk.n_param
    for i in range(X.shape[0]):
        h = 1e-6 * np.maximum(np.abs(X[i]), 1.0)
        Xp = np.repeat(X[i][None, :], 2 * P, axis=0)
        for k in range(P):
            Xp[2 * k, k] += h[k]
            Xp[2 * k + 1, k] -= h[k]
        fp = gm.objective(Xp, "fp64").cpu().numpy()
        fd = (fp[0::2] - fp[1::2]) / (2 * h)
        scale = np.max(np.abs(fd))
        assert np.max(np.abs(G[i] - fd)) <= 1e-6 * scale, (G[i], fd)


@pytest.mark.parametrize("name", ["smile_2y", "caplets_20x15"])
def test_adjoint_fp32_within_pricing_error(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X = _points(sk, 16, seed=33)
    _, G = gm.objective_grad(X, "fp32")
    G = G.cpu().numpy()
    for i in range(X.shape[0]):
        fo, go = om.objective_grad(X[i])
        if not np.isfinite(fo):
            continue
        scale = np.max(np.abs(go))
        assert np.max(np.abs(G[i] - go)) <= 2e-3 * scale


def test_adjoint_many_sets_sampled(gpu_lib):
    # the gradient workload: 65536 parameter sets on the caplet term structure, checked on a sample
    sk = synth.caplet_term_structure()
    om, gm = _markets(sk)
    X = _points(sk, 65536, seed=34)
    f, G = gm.objective_grad(X, "fp64")
    f, G = f.cpu().numpy(), G.cpu().numpy()
    for i in (0, 1, 777, 32768, 65535):
        fo, go = om.objective_grad(X[i])
        assert f[i] == pytest.approx(fo, rel=1e-12)
        assert np.max(np.abs(G[i] - go)) <= 1e-9 * np.max(np.abs(go))


def test_lm_recovers_generating_point_noise_free(gpu_lib):
    sk = synth.caplet_term_structure(noise_free=True, n_fwd=8, n_strikes=5)
    om, gm = _markets(sk)
    th0 = sk.theta_true.copy()
    th0[:9] *= 1.03
    X, f, r = gm.lm_polish(th0[None, :], max_iter=60)
    X = X.cpu().numpy()[0]
    assert r.cpu().numpy()[0] < 1e-6
    assert om.rmse_volpt(X) < 1e-6
    po = om.lm(th0, max_iter=200)
    assert np.max(np.abs(X[:9] - po["theta"][:9]) / np.maximum(np.abs(po["theta"][:9]), 1e-3)) < 1e-4


def test_lm_on_swaption_market_improves(gpu_lib):
    sk = synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4), noise_free=True)
    om, gm = _markets(sk)
    th0 = sk.theta_true * 1.02
    f0 = om.objective(th0)
    X, f, r = gm.lm_polish(th0[None, :], max_iter=30)
    assert f.cpu().numpy()[0] < 1e-3 * f0
    assert om.objective(X.cpu().numpy()[0]) == pytest.approx(f.cpu().numpy()[0], rel=1e-9)


def test_lm_zero_iterations_reports_the_start(gpu_lib):
    sk = synth.caplet_term_structure(n_fwd=7, n_strikes=5)
    om, gm = _markets(sk)
    X0 = _points(sk, 5, seed=11)
    X, f, r = gm.lm_polish(X0, max_iter=0)
    X, f, r = X.cpu().numpy(), f.cpu().numpy(), r.cpu().numpy()
    assert np.array_equal(X, X0)
    for i in range(5):
        assert f[i] == pytest.approx(om.objective(X0[i]), rel=1e-12)
        assert r[i] == pytest.approx(om.rmse_volpt(X0[i]), rel=1e-12)


def test_lm_f_and_rmse_are_those_of_the_returned_points(gpu_lib):
    sk = synth.caplet_term_structure(n_fwd=7, n_strikes=5)
    om, gm = _markets(sk)
    X0 = _points(sk, 6, seed=12)
    X, f, r = gm.lm_polish(X0, max_iter=8)
    X, f, r = X.cpu().numpy(), f.cpu().numpy(), r.cpu().numpy()
    for i in range(6):
        assert f[i] == pytest.approx(om.objective(X[i]), rel=1e-12)
        assert r[i] == pytest.approx(om.rmse_volpt(X[i]), rel=1e-12)
        assert f[i] <= om.objective(X0[i])
        assert np.all(X[i] >= sk.lo) and np.all(X[i] <= sk.hi)


@pytest.mark.parametrize("k", [1, 64])
def test_anneal_polish_top_k_bounds(gpu_lib, k):
    # k = 1 and k = n_chains (every chain polished) through the top-k selection
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    r0 = gm.anneal(64, 10, 20, 0.85, seed=5, prec="fp32")
    r1 = gm.anneal(64, 10, 20, 0.85, seed=5, prec="fp32", lm_top_k=k, lm_max_iter=10)
    # the polished result is an FP64 value, at most the FP64 objective of the search's best point
    assert r1["f_best"][0] <= om.objective(r0["x_best"][0]) * (1 + 1e-11)
    assert om.objective(r1["x_best"][0]) == pytest.approx(r1["f_best"][0], rel=1e-12)


def test_anneal_with_top_k_polish(gpu_lib):
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    r0 = gm.anneal(64, 30, 20, 0.85, seed=3, prec="fp32")
    r1 = gm.anneal(64, 30, 20, 0.85, seed=3, prec="fp32", lm_top_k=8, lm_max_iter=20)
    assert r1["f_best"][0] <= om.objective(r0["x_best"][0]) * (1 + 1e-11)
    assert r1["lm_seconds"] > 0.0
    # the polished point is a local minimum of the FP64 objective: LM from it moves nowhere
    p = om.lm(r1["x_best"][0], max_iter=20)
    assert p["f"] >= r1["f_best"][0] * (1 - 1e-9)
    assert om.objective(r1["x_best"][0]) == pytest.approx(r1["f_best"][0], rel=1e-12)


def test_autograd_function_backward_is_the_adjoint(gpu_lib):
    # CalibrationObjective: f from the library, X.grad = sum_i c_i df_i/dX_i from the reverse sweep,
    # compared with the oracle's dual-number gradient
    import torch
    sk = CASES["caplets_7x5"]()
    om, gm = _markets(sk)
    Xn = _points(sk, 4, seed=77)
    X = torch.tensor(Xn, dtype=torch.float64, device="cuda", requires_grad=True)
    f = gm.calibration_objective(X)
    c = torch.arange(1, 5, dtype=torch.float64, device="cuda")
    (c * f).sum().backward()
    g = X.grad.cpu().numpy()
    for i in range(4):
        fo, go = om.objective_grad(Xn[i])
        assert f[i].item() == pytest.approx(fo, rel=1e-12)
        assert np.max(np.abs(g[i] - (i + 1) * go)) <= 1e-9 * (i + 1) * np.max(np.abs(go))


def test_autograd_function_gradcheck(gpu_lib):
    # torch's own finite-difference check of the op (FP64, central differences)
    import torch
    sk = CASES["smile_2y"]()
    _, gm = _markets(sk)
    # points near the generating one keep f and its gradient of moderate size for the FD rounding
    rng = np.random.default_rng(78)
    Xn = sk.theta_true[None, :] * (1.0 + 0.05 * rng.standard_normal((2, sk.n_param)))
    X = torch.tensor(Xn, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: gm.calibration_objective(x), (X,), eps=1e-7, atol=1e-6, rtol=1e-4)


def _swaptions_only():
    sk = synth.joint_caplet_swaption(n_fwd=24, expiries=(1, 2, 4, 6), tenors=(1, 3, 5), swp_m=(-0.3, 0.0, 0.3))
    keep = np.arange(sk.n_cap, sk.n_instr)
    return sk.replace(cap_fwd=np.zeros(0, np.int32), cap_K=np.zeros(0), noise=sk.noise[keep])


SWAPTION_CASES = {
    "joint_small": lambda: synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4)),
    "joint_40f_300c_700s": lambda: synth.joint_caplet_swaption(),
    "swaptions_only": _swaptions_only,
    "batch_member_3": lambda: synth.batch_market(3),
}


@pytest.mark.parametrize("name", list(SWAPTION_CASES))
def test_swaption_adjoint_fp64_matches_oracle_dual_gradient(gpu_lib, name):
    # the reverse sweep through pricing, the swap-rate SABR parameters, the group forms, the window
    # integrals, the prefix tables, the Grams, the Y rows and the correlation tables: every one of
    # the 12 slots against the oracle's forward-mode dual numbers
    sk = SWAPTION_CASES[name]()
    om, gm = _markets(sk)
    X = np.vstack([_points(sk, 5, seed=35), sk.theta_true[None, :]])
    f, G = gm.objective_grad(X, "fp64")
    f, G = f.cpu().numpy(), G.cpu().numpy()
    worst = 0.0
    for i in range(X.shape[0]):
        fo, go = om.objective_grad(X[i])
        if not np.isfinite(fo):
            assert not np.isfinite(f[i])
            continue
        assert f[i] == pytest.approx(fo, rel=1e-12)
        scale = np.max(np.abs(go))
        worst = max(worst, np.max(np.abs(G[i] - go)) / scale)
        assert np.max(np.abs(G[i] - go)) <= 1e-9 * scale, (i, G[i], go)
    print(f"{name}: swaption adjoint, largest gradient error {worst:.2e} of the largest component")


def test_swaption_adjoint_matches_central_differences(gpu_lib):
    sk = SWAPTION_CASES["joint_small"]()
    om, gm = _markets(sk)
    X = _points(sk, 3, seed=36)
    _, G = gm.objective_grad(X, "fp64")
    G = G.cpu().numpy()
    P = sk.n_param
    for i in range(X.shape[0]):
        h = 1e-6 * np.maximum(np.abs(X[i]), 1.0)
        Xp = np.repeat(X[i][None, :], 2 * P, axis=0)
        for k in range(P):
            Xp[2 * k, k] += h[k]
            Xp[2 * k + 1, k] -= h[k]
        fp = gm.objective(Xp, "fp64").cpu().numpy()
        fd = (fp[0::2] - fp[1::2]) / (2 * h)
        assert np.max(np.abs(G[i] - fd)) <= 1e-6 * np.max(np.abs(fd)), (G[i], fd)


def test_swaption_adjoint_fp32_request_runs_in_fp64(gpu_lib):
    sk = SWAPTION_CASES["joint_small"]()
    om, gm = _markets(sk)
    X = _points(sk, 4, seed=37)
    f64, G64 = gm.objective_grad(X, "fp64")
    f32, G32 = gm.objective_grad(X, "fp32")
    assert np.array_equal(f64.cpu().numpy(), f32.cpu().numpy())
    assert np.allclose(G64.cpu().numpy(), G32.cpu().numpy(), rtol=1e-12, atol=0)


def test_swaption_adjoint_secondary_run_on_the_joint_market(gpu_lib):
    # the gradient workload's secondary run: many parameter sets on the 40-forward caplet + swaption
    # market (all 12 slots free), checked on a sample
    sk = synth.joint_caplet_swaption()
    om, gm = _markets(sk)
    X = _points(sk, 2048, seed=38)
    f, G = gm.objective_grad(X, "fp64")
    f, G = f.cpu().numpy(), G.cpu().numpy()
    for i in (0, 1023, 2047):
        fo, go = om.objective_grad(X[i])
        assert f[i] == pytest.approx(fo, rel=1e-12)
        assert np.max(np.abs(G[i] - go)) <= 1e-9 * np.max(np.abs(go))
