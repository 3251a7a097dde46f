"""sabr_lmm_anneal_noalloc, the annealing call for code that may not allocate device memory.

Some callers cannot call cudaMalloc: a service that gives all device memory to its own pool at
start-up, a plug-in host that lends the library a stream but no allocator, a latency-critical
loop that cannot afford cudaMalloc's implicit device synchronisation.  For them the library keeps
the search's working state in a fixed array inside its own device image.  This test calls that
entry point directly through the C-ABI, twice in a row (the second call finds the first call's
leftovers in the array), and checks both results against sabr_lmm_anneal, which allocates its
state: the same kernels on the same uniforms give the same search, bit for bit, on caplet markets
and on markets with swaptions.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2408_01470_b300 import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(lib_pkg, gm, opts_kw, n_param, n_levels):
    import torch
    lib = lib_pkg.load()
    fn = lib.sabr_lmm_anneal_noalloc
    fn.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lib_pkg.AnnealOpts), C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p]
    o, keep = gm._opts(**opts_kw)
    x = torch.full((n_param,), float("nan"), dtype=torch.float64, device="cuda")
    f = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    tr = torch.full((n_levels,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    st = fn(gm.h, 0, C.byref(o), C.c_void_p(x.data_ptr()), C.c_void_p(f.data_ptr()), C.c_void_p(tr.data_ptr()),
            C.c_void_p(s.cuda_stream))
    assert st == 0, lib.sabr_lmm_last_error().decode()
    torch.cuda.synchronize()
    return x.cpu().numpy(), float(f.cpu().numpy()[0]), tr.cpu().numpy()


def _small_joint():
    return synth.joint_caplet_swaption(expiries=(1, 2, 3), tenors=(1, 2, 3), swp_m=(-0.4, 0.0, 0.4))


@pytest.mark.parametrize("maker,prec,C_,L,N,cool", [
    (synth.smile_2y, "fp64", 64, 20, 10, 0.9),
    (synth.caplet_term_structure, "fp32", 256, 6, 12, 0.95),
    (_small_joint, "fp64", 48, 3, 6, 0.9),
    (_small_joint, "fp32", 96, 3, 6, 0.9),
])
def test_noalloc_anneal_matches_allocating_anneal_twice(gpu_lib, maker, prec, C_, L, N, cool):
    # the same kernels on the same uniforms: the same search, bit for bit, on caplet markets (4-chain
    # CTAs here, whatever CTA size the allocating call picks: a chain is one warp either way) and on
    # markets with swaptions (one CTA per chain)
    import paper_2408_01470_b300 as lib
    sk = maker()
    _, vols = oracle.quoted_market(sk)
    gm = lib.Market(sk, vols)
    ref = gm.anneal(C_, L, N, cool, seed=17, prec=prec)
    kw = dict(n_chains=C_, n_levels=L, steps=N, cooling=cool, seed=17, prec=prec, T0=0.0, step_frac=0.1,
              step_floor=1e-3, x0=None, lm_top_k=0, lm_max_iter=0, target_rmse=0.0, warps_per_block=0,
              use_graph=False, record_accepts=False)
    for _ in range(2):
        x, f, tr = _call_noalloc(lib, gm, kw, sk.n_param, L)
        assert np.array_equal(x, ref["x_best"][0])
        assert f == ref["f_best"][0]
        assert np.array_equal(tr, ref["trace_f"][0])


def test_noalloc_given_start_point_and_a_second_stream(gpu_lib):
    # x0 given (it travels as a kernel argument), and the call made on a stream other than the one
    # the first call of this device used: the array's address lookup is per device, not per stream
    import torch
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    _, vols = oracle.quoted_market(sk)
    gm = lib.Market(sk, vols)
    x0 = sk.lo + 0.3 * (sk.hi - sk.lo)
    ref = gm.anneal(32, 5, 8, 0.9, seed=23, prec="fp64", x0=x0)
    kw = dict(n_chains=32, n_levels=5, steps=8, cooling=0.9, seed=23, prec="fp64", T0=0.0, step_frac=0.1,
              step_floor=1e-3, x0=x0, lm_top_k=0, lm_max_iter=0, target_rmse=0.0, warps_per_block=0,
              use_graph=False, record_accepts=False)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x, f, tr = _call_noalloc(lib, gm, kw, sk.n_param, 5)
    assert np.array_equal(x, ref["x_best"][0]) and f == ref["f_best"][0]


def test_noalloc_rejects_sizes_beyond_its_static_scratch(gpu_lib):
    import paper_2408_01470_b300 as lib
    sk = synth.smile_2y()
    _, vols = oracle.quoted_market(sk)
    gm = lib.Market(sk, vols)
    handle = lib.load()
    fn = handle.sabr_lmm_anneal_noalloc
    fn.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lib.AnnealOpts), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    o, keep = gm._opts(16385, 10, 10, 0.9, 1, "fp64", 0.0, 0.1, 1e-3, None, 0, 0, 0.0, 0, False, False)
    import torch
    x = torch.empty(3, dtype=torch.float64, device="cuda")
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    st = fn(gm.h, 0, C.byref(o), C.c_void_p(x.data_ptr()), C.c_void_p(f.data_ptr()), None, None)
    assert st == 1
    assert "static scratch limit" in handle.sabr_lmm_last_error().decode()
