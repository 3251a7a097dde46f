"""The C-ABI library loads on a host without a GPU and exports every declared entry point.

No compute call is made here; argument validation runs before any CUDA call, so the EINVAL
paths are checked on the CPU too.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sabr_lmm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2408_01470_b300 import build
    build.build()
    import paper_2408_01470_b300 as pkg
    return pkg.open_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(sabr_lmm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_export():
    import paper_2408_01470_b300 as pkg
    assert set(declared_functions()) == set(pkg.EXPORTS)


def test_quadrature_rule_is_gauss_legendre(lib):
    import paper_2408_01470_b300 as pkg
    import mpmath as mp
    x, w = pkg.quadrature_rule(8)
    mp.mp.dps = 40
    for i in range(8):
        # each node is a root of P_8 and each weight 2 / ((1 - x^2) P_8'(x)^2), to 40 digits
        z = mp.findroot(lambda t: mp.legendre(8, t), mp.mpf(x[i]))
        dp = 8 * (z * mp.legendre(8, z) - mp.legendre(7, z)) / (z * z - 1)
        assert abs(x[i] - float(z)) <= 1.2e-16 * abs(float(z))
        assert abs(w[i] - float(2 / ((1 - z * z) * dp * dp))) <= 1.5e-16 * w[i]
    xr, wr = np.polynomial.legendre.leggauss(8)
    assert np.max(np.abs(x - xr)) < 1e-15 and np.max(np.abs(w - wr)) < 1e-15
    with pytest.raises(pkg.SabrLmmError):
        pkg.quadrature_rule(5)


def _desc(skel, **over):
    import paper_2408_01470_b300 as pkg
    vols = np.full(skel.n_instr, 0.2)
    d, keep = pkg.describe(skel, vols)
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("field,value,msg", [
    ("model", 7, "model"), ("formula", 3, "formula"), ("beta", 1.5, "beta"), ("n_fwd", 0, "n_fwd"),
    ("n_param", 5, "parameter slots"), ("panel", 0.0, "panel")])
def test_load_market_validates_before_any_cuda_call(lib, field, value, msg):
    from paper_2408_01470_b300 import synth
    sk = synth.caplet_term_structure()
    d, keep = _desc(sk, **{field: value})
    h = C.c_void_p()
    st = lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h))
    assert st == 1, st
    assert msg in lib.sabr_lmm_last_error().decode()
    assert h.value is None


def test_smile_model_rejects_swaptions_and_off_grid_times(lib):
    from paper_2408_01470_b300 import synth
    sk = synth.caplet_term_structure()
    T = sk.T.copy()
    T[3] += 0.1
    d, keep = _desc(sk.replace(T=T))
    h = C.c_void_p()
    assert lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h)) == 1
    assert "multiple of panel" in lib.sabr_lmm_last_error().decode()
    j = synth.joint_caplet_swaption(expiries=(1,), tenors=(1,))
    d, keep = _desc(j.replace(model=synth.MODEL_SABR_SMILE, lo=j.lo[:3], hi=j.hi[:3], free=j.free[:3],
                              theta_true=j.theta_true[:3]))
    assert lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h)) == 1
    assert "caplets only" in lib.sabr_lmm_last_error().decode()


def test_quad_nodes_other_than_8_not_supported(lib):
    from paper_2408_01470_b300 import synth
    sk = synth.caplet_term_structure()
    d, keep = _desc(sk, quad_nodes=6)
    h = C.c_void_p()
    assert lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h)) == 5


def test_mercurio_morini_shapes_validated_before_any_cuda_call(lib):
    # 2 n_fwd + 1 slots, at most 15 forwards, caplets only
    from paper_2408_01470_b300 import synth
    sk = synth.mercurio_morini_caplets()
    h = C.c_void_p()
    d, keep = _desc(sk, n_param=sk.n_param - 1)
    assert lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h)) == 1
    assert "2 n_fwd + 1" in lib.sabr_lmm_last_error().decode()
    wide = synth.mercurio_morini_caplets(n_fwd=16, n_strikes=2)
    d, keep = _desc(wide)
    assert lib.sabr_lmm_load_market(C.byref(d), 1, None, C.byref(h)) == 1
    assert "15 forwards" in lib.sabr_lmm_last_error().decode()


def _mc_desc(**over):
    import paper_2408_01470_b300 as pkg
    from paper_2408_01470_b300 import synth
    sk = synth.caplet_term_structure(n_fwd=6)
    model = dict(beta=0.5, eta1=0.8, lambda1=1.0, eta2=0.9, lambda2=1.0, lambda3=0.01, alpha=np.full(6, 0.2),
                 sigma=np.full(6, 0.3), phi=np.full(6, -0.3))
    model.update(over)
    return pkg.mc_describe(sk.T, sk.P, model, cap_fwd=[0, 3], cap_K=[0.01, 0.02], swp_start=[1], swp_end=[4],
                           swp_K=[0.02])


@pytest.mark.parametrize("over,opts,msg", [
    (dict(eta1=1.5), {}, "eta1"), (dict(beta=2.0), {}, "beta"), (dict(alpha=np.zeros(6)), {}, "alpha"),
    ({}, dict(n_paths=0), "n_paths"), ({}, dict(dt=0.0), "dt"), ({}, dict(prec=3), "prec")])
def test_mc_prepare_validates_before_any_cuda_call(lib, over, opts, msg):
    import paper_2408_01470_b300 as pkg
    d, keep = _mc_desc(**over)
    kw = dict(n_paths=100, dt=0.01, seed=1, prec=1, grid=0)
    kw.update(opts)
    o = pkg.McOpts()
    o.n_paths, o.dt, o.seed, o.prec, o.grid = kw["n_paths"], kw["dt"], kw["seed"], kw["prec"], kw["grid"]
    h = C.c_void_p()
    assert lib.sabr_lmm_mc_prepare(C.byref(d), C.byref(o), None, C.byref(h)) == 1
    assert msg in lib.sabr_lmm_last_error().decode()
    assert h.value is None


def test_mc_anneal_validates_its_box_before_any_cuda_call(lib):
    import paper_2408_01470_b300 as pkg
    d, keep = _mc_desc()
    o = pkg.McOpts()
    o.n_paths, o.dt, o.seed, o.prec, o.grid = 100, 0.01, 1, 1, 0
    lo, hi = np.zeros(5), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    bad_hi = hi.copy()
    bad_hi[0] = 1.5   # eta1 above 1
    fr = np.ones(5, np.uint8)
    qv = np.full(3, 0.3)
    for h_arr in (bad_hi,):
        a = pkg.McAnnealOpts()
        a.n_chains, a.n_levels, a.steps_per_level, a.cooling, a.step_frac, a.step_floor = 4, 2, 2, 0.9, 0.1, 1e-3
        a.lo, a.hi = lo.ctypes.data_as(pkg._D), h_arr.ctypes.data_as(pkg._D)
        a.free_mask = fr.ctypes.data_as(pkg._U8)
        r = pkg.McAnnealResult()
        st = lib.sabr_lmm_mc_anneal(C.byref(d), qv.ctypes.data_as(pkg._D), C.byref(o), C.byref(a), C.byref(r), None)
        assert st == 1 and "box" in lib.sabr_lmm_last_error().decode()
