"""Edge cases through the C-ABI: empty point sets, infeasible points, invalid options, one chain."""
import math

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu


def _markets(sk):
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(sk)
    return om, lib.Market(sk, vols)


def test_empty_point_sets(gpu_lib):
    sk = synth.caplet_term_structure(n_fwd=7, n_strikes=5)
    om, gm = _markets(sk)
    X = np.zeros((0, sk.n_param))
    for prec in ("fp64", "fp32"):
        assert gm.objective(X, prec).numel() == 0
        assert gm.model_vols(X, prec).shape[0] == 0
    f, G = gm.objective_grad(X, "fp64")
    assert f.numel() == 0 and G.shape[0] == 0
    Xp, f, r = gm.lm_polish(X, max_iter=3)
    assert Xp.shape[0] == 0 and f.numel() == 0


def test_infeasible_points_are_infinite_like_the_oracle(gpu_lib):
    # alpha = 0, alpha < 0, rho > 1 (a negative radicand in x(z)), a Hagan correction that turns
    # the vol negative, a NaN parameter; the last point is feasible
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    X = np.array([[0.03, 1.5, 2.0], [0.0, -0.3, 0.4], [-0.01, 0.2, 0.4], [0.03, 0.999999, 50.0],
                  [math.nan, 0.1, 0.2], [0.03, -0.3, 0.4]])
    fo = np.array([om.objective(x) for x in X])
    assert np.all(np.isinf(fo[:-1])) and np.isfinite(fo[-1])
    f64 = gm.objective(X, "fp64").cpu().numpy()
    f32 = gm.objective(X, "fp32").cpu().numpy()
    assert np.all(np.isposinf(f64[:-1])) and np.all(np.isposinf(f32[:-1]))
    assert f64[-1] == pytest.approx(fo[-1], rel=1e-12)
    assert f32[-1] == pytest.approx(fo[-1], rel=1e-3)


def test_anneal_rejects_invalid_options(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    bad = [dict(n_chains=0, n_levels=1, steps=1), dict(n_chains=4, n_levels=0, steps=1),
           dict(n_chains=4, n_levels=1, steps=0), dict(n_chains=4, n_levels=1, steps=1, lm_top_k=5)]
    for b in bad:
        kw = {k: v for k, v in b.items() if k == "lm_top_k"}
        with pytest.raises(lib.SabrLmmError) as e:
            gm.anneal(b["n_chains"], b["n_levels"], b["steps"], 0.9, seed=1, **kw)
        assert e.value.status == 1, b   # EINVAL


def test_single_chain_fp64_trajectory(gpu_lib):
    sk = synth.caplet_term_structure(n_fwd=7, n_strikes=5)
    om, gm = _markets(sk)
    r_g = gm.anneal(1, 5, 20, 0.9, seed=4, prec="fp64", record_accepts=True)
    r_o = om.anneal(1, 5, 20, 0.9, seed=4, want_bits=True)
    assert r_g["n_evals"] == r_o["n_evals"] == 1 * (5 * 20 + 1)
    assert np.array_equal(r_g["bits"], r_o["bits"])
    assert np.allclose(r_g["x_best"][0], r_o["x_best"], rtol=1e-12, atol=1e-15)
    assert r_g["f_best"][0] == pytest.approx(r_o["f_best"], rel=1e-11)


def test_bounded_device_wait_gives_up_and_reports(gpu_lib):
    # a wait on an mbarrier phase that never completes: the library's bounded wait gives up, raises
    # its error word, and the call returns SABR_LMM_ETIMEOUT; the context stays usable
    import paper_2408_01470_b300 as lib
    assert lib.selftest_wait(4096) == 4
    assert lib.selftest_wait(1) == 4
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    x = sk.theta_true[None, :]
    assert gm.objective(x, "fp64").cpu().numpy()[0] == pytest.approx(om.objective(x[0]), rel=1e-12)


def test_bad_start_points_and_quotes_are_rejected(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    for x0 in (sk.hi + 0.1, np.array([math.nan, 0.0, 0.4])):
        with pytest.raises(lib.SabrLmmError) as e:
            gm.anneal(8, 1, 2, 0.9, seed=1, x0=x0)
        assert e.value.status == 1 and "x0" in str(e.value)
    r = gm.anneal(8, 1, 2, 0.9, seed=1, x0=sk.box_centre())   # inside: accepted
    assert np.isfinite(r["f_best"][0])
    vols = np.full(sk.n_cap, 0.2)
    vols[3] = math.nan
    with pytest.raises(lib.SabrLmmError) as e:
        lib.Market(sk, vols)
    assert e.value.status == 1 and "cap_vol" in str(e.value)


@pytest.mark.parametrize("maker", [synth.smile_2y,
                                   lambda: synth.joint_caplet_swaption(expiries=(1, 2), tenors=(1, 2),
                                                                       swp_m=(0.0,))])
def test_error_word_is_reported_once_then_cleared(gpu_lib, maker):
    # host-side injection only (no device wait is run out here): the market's error word is raised
    # from the host; the next sync reports ETIMEOUT once, the one after it OK; the same for the
    # annealing call, which reads and clears the word after its search; stream-ordered calls made
    # meanwhile still run and return their values
    import paper_2408_01470_b300 as lib
    sk = maker()
    om, gm = _markets(sk)
    x = sk.theta_true[None, :]
    gm.sync()
    gm.test_raise_error()
    f = gm.objective(x, "fp64").cpu().numpy()[0]
    assert f == pytest.approx(om.objective(x[0]), rel=1e-12)
    with pytest.raises(lib.SabrLmmError) as e:
        gm.sync()
    assert e.value.status == 4
    gm.sync()
    gm.test_raise_error()
    with pytest.raises(lib.SabrLmmError) as e:
        gm.anneal(8, 2, 3, 0.9, seed=1)
    assert e.value.status == 4
    r = gm.anneal(8, 2, 3, 0.9, seed=1)
    assert np.isfinite(r["f_best"][0])
    gm.sync()


def test_residuals_rows_of_infeasible_points_are_nan(gpu_lib):
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    X = np.array([[0.0, -0.3, 0.4], [0.03, -0.3, 0.4]])
    for prec in ("fp64", "fp32"):
        f, r = gm.residuals(X, prec)
        f, r = f.cpu().numpy(), r.cpu().numpy()
        assert np.isposinf(f[0]) and np.all(np.isnan(r[0]))
        r_or, _ = om.residuals_jac(X[1])
        assert np.all(np.isfinite(r[1])) and np.max(np.abs(r[1] - r_or)) <= (1e-12 if prec == "fp64" else 2e-6)
