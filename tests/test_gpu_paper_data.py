"""The paper's real-data caplet calibration (Section 4.1.1, Hagan model, Eq. sigmaHagan) on the GPU.

The 13 EURIBOR smiles of 21/11/2011 with the paper's schedule (w = 16384 chains, N = 10, cooling
0.99, T0 = 10 to T_min = 0.01: 688 levels) and its hybrid: the FP32 search, then Nelder-Mead from
the best chains in FP64.  The paper's cost is separable over the forwards (each smile has its own
alpha, rho, nu), so the 13 smiles are 13 searches of one call; together they price the same
number of caplets as the paper's single run over all of them (13 x 9 quotes x 112738304
evaluations).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu

FIXTURE = os.path.join(os.path.dirname(__file__), "golden", "paper_euribor_20111121.txt")


def test_paper_euribor_caplets_hybrid_search_reaches_the_published_mre(gpu_lib):
    import paper_2408_01470_b300 as lib
    sks, quotes, params, pub = synth.paper_euribor_caplet_smiles(FIXTURE)
    gm = lib.Market(sks, quotes)
    sk = sks[0]
    r = gm.anneal(sk.n_chains, sk.n_levels, sk.steps, sk.cooling, seed=20111121, prec="fp32", T0=10.0,
                  lm_top_k=8, lm_max_iter=2000, polish_nm=True)
    assert r["n_evals"] == int(pub["evaluations"])
    rel = []
    for j, (skj, q) in enumerate(zip(sks, quotes)):
        om = oracle.Market(skj, q)
        x = r["x_best"][j]
        assert np.all(x >= skj.lo) and np.all(x <= skj.hi)
        assert r["f_best"][j] == pytest.approx(om.objective(x), rel=1e-12)
        # no worse than the paper's own (4-digit) parameters
        assert r["f_best"][j] <= om.objective(params[j]) * (1 + 1e-9), j
        rel += list(np.abs(om.model_vols(x) - q) / q)
    assert float(np.mean(rel)) <= 1.80e-2 + 5e-5
