"""The Nelder-Mead polish of the paper's hybrid scheme (SA, then a simplex search), through the C-ABI.

The GPU simplex runs the oracle's algorithm (same coefficients, projection, initial simplex and
vertex order) on the GPU's FP64 objective, which agrees with the oracle's to ~1e-15 relative: the
two searches take the same branches unless two vertex values tie within that rounding (near the
end, where the stopping test compares differences of that size), and end at the same point.
"""
import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu

CASES = {
    "smile_2y": lambda: synth.smile_2y(),
    "caplets_7x5": lambda: synth.caplet_term_structure(n_fwd=7, n_strikes=5),
    "joint_small": lambda: synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4)),
}


def _markets(sk):
    import paper_2408_01470_b300 as lib
    om, vols = oracle.quoted_market(sk)
    return om, lib.Market(sk, vols)


@pytest.mark.parametrize("name", list(CASES))
def test_nm_matches_the_oracle_simplex(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    X0 = 0.5 * (synth.uniform_in_box(sk, 4, seed=51) + sk.theta_true[None, :])
    iters = 60 if sk.n_swp else 150
    X, f, ev = gm.nm_polish(X0, max_iter=iters, step=0.02, ftol=1e-14)
    X, f, ev = X.cpu().numpy(), f.cpu().numpy(), ev.cpu().numpy()
    for i in range(X0.shape[0]):
        po = om.nm(X0[i], max_iter=iters, step=0.02, ftol=1e-14)
        assert f[i] == pytest.approx(po["f"], rel=1e-9), (i, f[i], po["f"])
        assert np.allclose(X[i], po["theta"], rtol=1e-7, atol=1e-12)
        # (near the end the vertex values differ by ~1e-15 relative, so the stopping test and the
        # last branches can fall either way and the evaluation counts are not compared)
        assert f[i] == pytest.approx(om.objective(X[i]), rel=1e-12)
    # the initial simplex alone: nf + 1 evaluations on both sides, the same best vertex
    X, f, ev = gm.nm_polish(X0, max_iter=0, step=0.02)
    for i in range(X0.shape[0]):
        po = om.nm(X0[i], max_iter=0, step=0.02)
        assert int(ev[i]) == po["evals"] == int(sk.free.sum()) + 1
        assert np.array_equal(X.cpu().numpy()[i], po["theta"])


def test_nm_recovers_the_generating_smile(gpu_lib):
    sk = synth.smile_2y(noise_free=True)
    om, gm = _markets(sk)
    th0 = sk.theta_true * np.array([1.05, 0.9, 1.1])
    X, f, _ = gm.nm_polish(th0[None, :], max_iter=2000, step=0.02, ftol=1e-15)
    X = X.cpu().numpy()[0]
    assert f.cpu().numpy()[0] < 1e-16
    assert np.max(np.abs(X - sk.theta_true) / np.abs(sk.theta_true)) < 1e-5


def test_hybrid_sa_then_nm_improves_the_search(gpu_lib):
    # the paper's hybrid: the annealer's best point, then Nelder-Mead
    sk = synth.caplet_term_structure()
    om, gm = _markets(sk)
    r = gm.anneal(512, 10, 20, 0.9, seed=3, prec="fp32")
    X, f, _ = gm.nm_polish(r["x_best"], max_iter=300)
    f = f.cpu().numpy()[0]
    assert f <= om.objective(r["x_best"][0]) * (1 + 1e-12)
    assert f == pytest.approx(om.objective(X.cpu().numpy()[0]), rel=1e-12)


def test_nm_rejects_bad_options_and_handles_empty_sets(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    om, gm = _markets(sk)
    for kw in (dict(max_iter=-1), dict(step=0.0), dict(step=1.5), dict(ftol=-1.0)):
        with pytest.raises(lib.SabrLmmError) as e:
            gm.nm_polish(sk.theta_true[None, :], **kw)
        assert e.value.status == 1
    X, f, ev = gm.nm_polish(np.zeros((0, 3)))
    assert X.shape[0] == 0 and f.numel() == 0


@pytest.mark.parametrize("name", ["caplets_7x5", "joint_small"])
def test_annealer_top_k_polish_by_nelder_mead(gpu_lib, name):
    sk = CASES[name]()
    om, gm = _markets(sk)
    r0 = gm.anneal(256, 6, 10, 0.9, seed=7, prec="fp32")
    r = gm.anneal(256, 6, 10, 0.9, seed=7, prec="fp32", lm_top_k=8, lm_max_iter=100, polish_nm=True)
    assert r["f_best"][0] <= om.objective(r0["x_best"][0]) * (1 + 1e-11)
    assert r["f_best"][0] == pytest.approx(om.objective(r["x_best"][0]), rel=1e-12)
    assert r["lm_seconds"] > 0.0
