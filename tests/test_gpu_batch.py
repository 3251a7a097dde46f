"""The batch path (S11): several uneven markets annealed by one persistent launch per temperature
level.  Each market keeps its own Philox stream (market index in the counter), chain state and
best-chain reduction, so in FP64 every market reproduces the oracle's search run with its index.
"""
import numpy as np
import pytest

import oracle
from fp32_parity import FAR_ABS_VOLPT, FAR_REL, objective_bound, residual_errors
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu


def _batch(js):
    import paper_2408_01470_b300 as lib
    sks = [synth.batch_market(j) for j in js]
    oms, vols = zip(*[oracle.quoted_market(sk) for sk in sks])
    return sks, oms, lib.Market(list(sks), list(vols))


@pytest.mark.parametrize("wpb", [0, 8])
def test_batch_fp64_reproduces_each_market_search(gpu_lib, wpb):
    # market 138 is the one caplet-only market of the batch family: in a batch with swaption
    # markets it runs on the CTA path, its caplets priced from diagonal 0 of the pair tables
    sks, oms, gm = _batch([0, 1, 138, 5])
    assert sks[2].n_swp == 0 and all(sk.n_swp > 0 for k, sk in enumerate(sks) if k != 2)
    C, L, N = 16, 3, 4
    r = gm.anneal(C, L, N, 0.9, seed=77, prec="fp64", record_accepts=True, warps_per_block=wpb)
    for j, om in enumerate(oms):
        ro = om.anneal(C, L, N, 0.9, seed=77, market_index=j, n_threads=8, want_bits=(j == 0))
        assert np.allclose(r["trace_f"][j], ro["trace_f"], rtol=1e-11, atol=0), j
        assert np.allclose(r["x_best"][j], ro["x_best"], rtol=1e-12, atol=1e-15), j
        assert r["f_best"][j] == pytest.approx(ro["f_best"], rel=1e-11)
        if j == 0:
            assert np.array_equal(r["bits"], ro["bits"])
    assert r["n_evals"] == C * (L * N + 1)


def test_batch_fp32_runs_every_market(gpu_lib):
    # every market's result: the FP32 search's value against the oracle's objective at the returned
    # point within the bound the per-price bars imply, and every price of that point (the search's
    # own pricer, through the residuals entry point) within the far-point bar
    sks, oms, gm = _batch(list(range(12)))
    r = gm.anneal(64, 4, 8, 0.9, seed=3, prec="fp32")
    for j, om in enumerate(oms):
        f0 = om.objective(sks[j].box_centre())
        x = r["x_best"][j]
        assert np.isfinite(r["f_best"][j])
        assert r["f_best"][j] <= f0
        f64 = om.objective(x)
        assert abs(r["f_best"][j] - f64) <= objective_bound(f64, sks[j].n_instr), (j, r["f_best"][j], f64)
        err, mag = residual_errors(gm, om, x[None, :], "fp32", market=j)
        ok = np.isfinite(err)
        assert ok.all(), j
        assert np.all(err[ok] <= FAR_ABS_VOLPT + FAR_REL * mag[ok]), (j, float(np.max(err)))


def test_batch_fp32_search_with_polish(gpu_lib):
    # the mixed-precision form on a batch: FP32 search, then the FP64 Levenberg-Marquardt polish of
    # each market's 8 best chains; every market's result is an FP64 value no worse than the FP64
    # objective of its search's best point, and is the oracle's objective at the returned point
    sks, oms, gm = _batch([0, 3, 4, 7])
    r0 = gm.anneal(64, 4, 8, 0.9, seed=21, prec="fp32")
    r1 = gm.anneal(64, 4, 8, 0.9, seed=21, prec="fp32", lm_top_k=8, lm_max_iter=10)
    assert r1["lm_seconds"] > 0.0
    for j, om in enumerate(oms):
        assert r1["f_best"][j] <= om.objective(r0["x_best"][j]) * (1 + 1e-11), j
        assert om.objective(r1["x_best"][j]) == pytest.approx(r1["f_best"][j], rel=1e-12), j
