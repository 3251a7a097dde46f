"""ORACLE -- test infrastructure only.

ctypes wrapper around ``oracle/sabr_oracle.cpp``: a plain FP64 CPU restatement of the
calibration objective, its gradient and the parallel simulated-annealing search of arXiv
2408.01470.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library (``paper_2408_01470_b300``);
both are fed the same seeded synthetic inputs from ``paper_2408_01470_b300.synth``, a module that
holds none of the method's arithmetic.

Parity status of each function is stated in ``sabr_oracle.cpp``'s header; every function there
is pinned by a ``-m "not gpu"`` test under ``tests/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sabr_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", _LIB_PATH + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Desc(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("formula", C.c_int32), ("beta", C.c_double),
        ("n_fwd", C.c_int32), ("T", C.POINTER(C.c_double)), ("P", C.POINTER(C.c_double)),
        ("n_cap", C.c_int32), ("cap_fwd", C.POINTER(C.c_int32)), ("cap_K", C.POINTER(C.c_double)),
        ("cap_vol", C.POINTER(C.c_double)), ("cap_w", C.POINTER(C.c_double)),
        ("n_swp", C.c_int32), ("swp_start", C.POINTER(C.c_int32)), ("swp_end", C.POINTER(C.c_int32)),
        ("swp_K", C.POINTER(C.c_double)), ("swp_vol", C.POINTER(C.c_double)),
        ("swp_w", C.POINTER(C.c_double)),
        ("n_param", C.c_int32), ("lo", C.POINTER(C.c_double)), ("hi", C.POINTER(C.c_double)),
        ("free_mask", C.POINTER(C.c_uint8)), ("panel", C.c_double), ("quad_nodes", C.c_int32),
    ]


class _SAOpts(C.Structure):
    _fields_ = [
        ("n_chains", C.c_int32), ("n_levels", C.c_int32), ("steps", C.c_int32),
        ("T0", C.c_double), ("cooling", C.c_double), ("step_frac", C.c_double),
        ("step_floor", C.c_double), ("seed", C.c_uint64), ("market_index", C.c_uint64),
        ("x0", C.POINTER(C.c_double)), ("n_threads", C.c_int32),
    ]


_D = C.POINTER(C.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            lib.orc_market_new.restype = C.c_void_p
            lib.orc_market_new.argtypes = [C.POINTER(_Desc)]
            lib.orc_market_free.argtypes = [C.c_void_p]
            for name in ("orc_normal_cdf",):
                getattr(lib, name).restype = C.c_double
                getattr(lib, name).argtypes = [C.c_double]
            for name in ("orc_black_call", "orc_black_put", "orc_black_otm", "orc_black_vega"):
                getattr(lib, name).restype = C.c_double
                getattr(lib, name).argtypes = [C.c_double] * 5
            lib.orc_z_over_x.restype = C.c_double
            lib.orc_z_over_x.argtypes = [C.c_double] * 2
            lib.orc_sabr_hagan2002.restype = C.c_double
            lib.orc_sabr_hagan2002.argtypes = [C.c_double] * 7
            lib.orc_sabr_paper.restype = C.c_double
            lib.orc_sabr_paper.argtypes = [C.c_double] * 6
            lib.orc_gl_nodes.argtypes = [C.c_int, _D, _D]
            lib.orc_market_info.argtypes = [C.c_void_p] + [_D] * 7
            lib.orc_rebonato_caplet.argtypes = [C.c_void_p, _D, C.c_double, _D]
            lib.orc_swap_params.argtypes = [C.c_void_p, _D, C.c_int, _D]
            lib.orc_model_vols.argtypes = [C.c_void_p, _D, _D]
            lib.orc_objective.restype = C.c_double
            lib.orc_objective.argtypes = [C.c_void_p, _D]
            lib.orc_objective_batch.argtypes = [C.c_void_p, _D, C.c_int64, _D, C.c_int]
            lib.orc_rmse_volpt.restype = C.c_double
            lib.orc_rmse_volpt.argtypes = [C.c_void_p, _D]
            lib.orc_objective_grad.restype = C.c_double
            lib.orc_objective_grad.argtypes = [C.c_void_p, _D, _D]
            lib.orc_residuals_jac.restype = C.c_int
            lib.orc_residuals_jac.argtypes = [C.c_void_p, _D, _D, _D]
            lib.orc_philox4x64_10.argtypes = [C.POINTER(C.c_uint64)] * 3
            lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            lib.orc_mc_normals4.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int, _D]
            _I = C.POINTER(C.c_int32)
            _MCI = [C.c_void_p, C.c_int, C.c_int, _D, _D, _D, _D, C.c_int, _I, _D, C.c_int, _I, _I, _D, _D, C.c_int64,
                    C.c_double, C.c_uint64]
            lib.orc_mc_objective.restype = C.c_double
            lib.orc_mc_objective.argtypes = _MCI + [_D, C.c_int]
            lib.orc_mc_anneal.restype = C.c_int
            lib.orc_mc_anneal.argtypes = _MCI + [_D, _D, C.POINTER(C.c_uint8), C.POINTER(_SAOpts), _D, _D, _D, _D, _D]
            lib.orc_mc_price.restype = C.c_int
            lib.orc_mc_price.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, _D, _D, _D, C.c_int, _I, _D, C.c_int, _I, _I,
                                         _D, C.c_int64, C.c_double, C.c_uint64, C.c_int, _D, _D,
                                         C.POINTER(C.c_int64)]
            lib.orc_step_uniforms.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_int, _D]
            lib.orc_anneal.restype = C.c_int
            lib.orc_anneal.argtypes = [C.c_void_p, C.POINTER(_SAOpts), _D, _D, _D, _D, _D, _D,
                                       C.POINTER(C.c_uint8), C.POINTER(C.c_int64), _D]
            lib.orc_nm.restype = C.c_int
            lib.orc_nm.argtypes = [C.c_void_p, _D, C.c_int, C.c_double, C.c_double, _D, _D,
                                   C.POINTER(C.c_int), C.POINTER(C.c_int)]
            lib.orc_lm.restype = C.c_int
            lib.orc_lm.argtypes = [C.c_void_p, _D, C.c_int, C.c_double, C.c_double, _D, _D, _D,
                                   C.POINTER(C.c_int)]
            _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- scalar formulas
def normal_cdf(x):
    return _lib_handle().orc_normal_cdf(float(x))


def black_call(F, K, T, sigma, D=1.0):
    return _lib_handle().orc_black_call(F, K, T, sigma, D)


def black_put(F, K, T, sigma, D=1.0):
    return _lib_handle().orc_black_put(F, K, T, sigma, D)


def black_otm(F, K, T, sigma, D=1.0):
    return _lib_handle().orc_black_otm(F, K, T, sigma, D)


def black_vega(F, K, T, sigma, D=1.0):
    return _lib_handle().orc_black_vega(F, K, T, sigma, D)


def z_over_x(z, rho):
    return _lib_handle().orc_z_over_x(z, rho)


def sabr_hagan2002(F, K, T, alpha, beta, rho, nu):
    return _lib_handle().orc_sabr_hagan2002(F, K, T, alpha, beta, rho, nu)


def sabr_paper(F, K, alpha, beta, rho, nu):
    return _lib_handle().orc_sabr_paper(F, K, alpha, beta, rho, nu)


def gl_nodes(n):
    x = np.zeros(n)
    w = np.zeros(n)
    _lib_handle().orc_gl_nodes(n, _dp(x), _dp(w))
    return x, w


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, np.uint64)
    P = C.POINTER(C.c_uint64)
    _lib_handle().orc_philox4x64_10(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P))
    return o


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    P = C.POINTER(C.c_uint32)
    _lib_handle().orc_philox4x32_10(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P))
    return o


def mc_normals4(seed, path, step, block):
    z = np.zeros(4)
    _lib_handle().orc_mc_normals4(seed, path, step, block, _dp(z))
    return z


def step_uniforms(seed, chain_word, level, step, count):
    u = np.zeros(count)
    _lib_handle().orc_step_uniforms(seed, chain_word, level, step, count, _dp(u))
    return u


# ---------------------------------------------------------------- market
class Market:
    """A market as the oracle sees it: a skeleton plus quotes in vol units."""

    def __init__(self, skel, vols=None, weights=None):
        self.skel = skel
        n_cap, n_swp = skel.n_cap, skel.n_swp
        if vols is None:
            vols = np.full(n_cap + n_swp, 0.2)
        vols = _f64(vols)
        self._keep = dict(
            T=_f64(skel.T), P=_f64(skel.P), cap_fwd=np.ascontiguousarray(skel.cap_fwd, np.int32),
            cap_K=_f64(skel.cap_K), cap_vol=_f64(vols[:n_cap]), swp_start=np.ascontiguousarray(skel.swp_start, np.int32),
            swp_end=np.ascontiguousarray(skel.swp_end, np.int32), swp_K=_f64(skel.swp_K),
            swp_vol=_f64(vols[n_cap:]), lo=_f64(skel.lo), hi=_f64(skel.hi),
            free=np.ascontiguousarray(skel.free, np.uint8))
        if weights is not None:
            w = _f64(weights)
            self._keep["cap_w"] = _f64(w[:n_cap])
            self._keep["swp_w"] = _f64(w[n_cap:])
        k = self._keep
        I32 = C.POINTER(C.c_int32)
        d = _Desc()
        d.model, d.formula, d.beta = skel.model, skel.formula, skel.beta
        d.n_fwd, d.T, d.P = skel.n_fwd, _dp(k["T"]), _dp(k["P"])
        d.n_cap = n_cap
        d.cap_fwd = k["cap_fwd"].ctypes.data_as(I32)
        d.cap_K, d.cap_vol = _dp(k["cap_K"]), _dp(k["cap_vol"])
        d.cap_w = _dp(k.get("cap_w"))
        d.n_swp = n_swp
        d.swp_start = k["swp_start"].ctypes.data_as(I32)
        d.swp_end = k["swp_end"].ctypes.data_as(I32)
        d.swp_K, d.swp_vol = _dp(k["swp_K"]), _dp(k["swp_vol"])
        d.swp_w = _dp(k.get("swp_w"))
        d.n_param, d.lo, d.hi = skel.n_param, _dp(k["lo"]), _dp(k["hi"])
        d.free_mask = k["free"].ctypes.data_as(C.POINTER(C.c_uint8))
        d.panel, d.quad_nodes = skel.panel, skel.quad_nodes
        self._desc = d
        self._lib = _lib_handle()
        self.h = self._lib.orc_market_new(C.byref(d))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._lib.orc_market_free(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def n_param(self):
        return self.skel.n_param

    @property
    def n_instr(self):
        return self.skel.n_instr

    def info(self):
        s = self.skel
        F = np.zeros(s.n_fwd)
        cpm, cw = np.zeros(s.n_cap), np.zeros(s.n_cap)
        spm, sw, sS, sA = (np.zeros(s.n_swp) for _ in range(4))
        self._lib.orc_market_info(self.h, _dp(F), _dp(cpm), _dp(cw), _dp(spm), _dp(sw), _dp(sS), _dp(sA))
        return dict(F=F, cap_price=cpm, cap_w=cw, swp_price=spm, swp_w=sw, swp_S=sS, swp_A=sA)

    def rebonato_caplet(self, theta, Ti):
        o = np.zeros(4)
        self._lib.orc_rebonato_caplet(self.h, _dp(_f64(theta)), float(Ti), _dp(o))
        return dict(G=o[0], X=o[1], alpha=o[2], nu=o[3])

    def swap_params(self, theta, s):
        o = np.zeros(6)
        self._lib.orc_swap_params(self.h, _dp(_f64(theta)), int(s), _dp(o))
        return dict(V1=o[0], V2=o[1], V3=o[2], alpha=o[3], nu=o[4], rho=o[5])

    def model_vols(self, theta):
        v = np.zeros(self.n_instr)
        self._lib.orc_model_vols(self.h, _dp(_f64(theta)), _dp(v))
        return v

    def objective(self, theta):
        return self._lib.orc_objective(self.h, _dp(_f64(theta)))

    def objective_batch(self, X, n_threads=1):
        X = _f64(np.atleast_2d(X))
        f = np.zeros(X.shape[0])
        self._lib.orc_objective_batch(self.h, _dp(X), X.shape[0], _dp(f), int(n_threads))
        return f

    def rmse_volpt(self, theta):
        return self._lib.orc_rmse_volpt(self.h, _dp(_f64(theta)))

    def objective_grad(self, theta):
        g = np.zeros(self.n_param)
        f = self._lib.orc_objective_grad(self.h, _dp(_f64(theta)), _dp(g))
        return f, g

    def residuals_jac(self, theta):
        """(r, J): the weighted residuals and their Jacobian (dual numbers, at most 12 slots; J is
        None beyond that), or (None, None) at an infeasible point."""
        r = np.zeros(self.n_instr)
        J = np.zeros((self.n_instr, self.n_param)) if self.n_param <= 12 else None
        rc = self._lib.orc_residuals_jac(self.h, _dp(_f64(theta)), _dp(r), _dp(J))
        return (r, J) if rc == 0 else (None, None)

    def anneal(self, n_chains, n_levels, steps, cooling, seed, T0=0.0, step_frac=0.1,
               step_floor=1e-3, x0=None, market_index=0, n_threads=1, want_bits=False,
               want_chains=False):
        P = self.n_param
        o = _SAOpts()
        o.n_chains, o.n_levels, o.steps = n_chains, n_levels, steps
        o.T0, o.cooling, o.step_frac, o.step_floor = T0, cooling, step_frac, step_floor
        o.seed, o.market_index = seed, market_index
        x0a = None if x0 is None else _f64(x0)
        o.x0 = _dp(x0a)
        o.n_threads = n_threads
        xb, fb = np.zeros(P), np.zeros(1)
        cxb = np.zeros((n_chains, P)) if want_chains else None
        cfb = np.zeros(n_chains) if want_chains else None
        tf, tx = np.zeros(n_levels), np.zeros((n_levels, P))
        bits = np.zeros((n_chains, n_levels, steps), np.uint8) if want_bits else None
        ne = C.c_int64(0)
        t0 = np.zeros(1)
        self._lib.orc_anneal(self.h, C.byref(o), _dp(xb), _dp(fb), _dp(cxb), _dp(cfb), _dp(tf), _dp(tx),
                             None if bits is None else bits.ctypes.data_as(C.POINTER(C.c_uint8)),
                             C.byref(ne), _dp(t0))
        return dict(x_best=xb, f_best=fb[0], chain_xb=cxb, chain_fb=cfb, trace_f=tf, trace_x=tx,
                    bits=bits, n_evals=ne.value, T0=t0[0])

    def nm(self, theta0, max_iter=500, step=0.02, ftol=1e-12):
        """Nelder-Mead on the free slots (see sabr_oracle.cpp)."""
        th, f = np.zeros(self.n_param), np.zeros(1)
        it, ev = C.c_int(0), C.c_int(0)
        self._lib.orc_nm(self.h, _dp(_f64(theta0)), int(max_iter), float(step), float(ftol), _dp(th), _dp(f),
                         C.byref(it), C.byref(ev))
        return dict(theta=th, f=f[0], iters=it.value, evals=ev.value)

    def lm(self, theta0, max_iter=50, target_rmse=0.0, mu0=1e-3):
        P = self.n_param
        th, f, r = np.zeros(P), np.zeros(1), np.zeros(1)
        it = C.c_int(0)
        self._lib.orc_lm(self.h, _dp(_f64(theta0)), int(max_iter), float(target_rmse), float(mu0),
                         _dp(th), _dp(f), _dp(r), C.byref(it))
        return dict(theta=th, f=f[0], rmse=r[0], iters=it.value)


def mc_price(market, model, cap_fwd=(), cap_K=(), swp_a=(), swp_b=(), swp_K=(), n_paths=1000, dt=0.01,
             seed=1, n_threads=1):
    """Monte Carlo prices of caplets and swaptions under the Hagan SABR/LIBOR model, or with
    model["model"] = 2 the Mercurio & Morini one (see sabr_oracle.cpp mc_price), on `market`'s
    tenor structure.  model: dict with M, beta, eta1, lambda1, eta2, lambda2, lambda3 and per-forward
    alpha, sigma, phi (Mercurio & Morini: sigma[0] is the common vol of vol, phi_i = corr(W_i, Z)).  Returns (price, stderr,
    n_bad), n_bad the paths stopped at a non-finite state, or None on a bad input."""
    M = int(model["M"])
    par = _f64([model["beta"], model["eta1"], model["lambda1"], model["eta2"], model["lambda2"], model["lambda3"]])
    al, sg, ph = (_f64(model[k])[:M] for k in ("alpha", "sigma", "phi"))
    cf = np.ascontiguousarray(cap_fwd, np.int32)
    ck = _f64(cap_K)
    sa = np.ascontiguousarray(swp_a, np.int32)
    sb = np.ascontiguousarray(swp_b, np.int32)
    sk = _f64(swp_K)
    ni = len(cf) + len(sa)
    price, sq = np.zeros(max(ni, 1)), np.zeros(max(ni, 1))
    nb = C.c_int64(0)
    _I = C.POINTER(C.c_int32)
    rc = market._lib.orc_mc_price(market.h, M, int(model.get("model", 0)), _dp(par), _dp(al), _dp(sg), _dp(ph), len(cf), cf.ctypes.data_as(_I),
                                  _dp(ck), len(sa), sa.ctypes.data_as(_I), sb.ctypes.data_as(_I), _dp(sk),
                                  int(n_paths), float(dt), int(seed), int(n_threads), _dp(price), _dp(sq),
                                  C.byref(nb))
    if rc != 0:
        return None
    price, sq = price[:ni], sq[:ni]
    se = np.sqrt(np.maximum(sq - price * price, 0.0) / max(int(n_paths) - 1, 1))
    return price, se, nb.value


def _mc_args(market, model, cap_fwd, cap_K, swp_a, swp_b, swp_K, quote_vol):
    M = int(model["M"])
    keep = dict(par=_f64([model["beta"], model.get("eta1", 0.0), model.get("lambda1", 0.0), model.get("eta2", 0.0),
                          model.get("lambda2", 0.0), model.get("lambda3", 0.0)]),
                al=_f64(model["alpha"])[:M], sg=_f64(model["sigma"])[:M], ph=_f64(model["phi"])[:M],
                cf=np.ascontiguousarray(cap_fwd, np.int32), ck=_f64(cap_K), sa=np.ascontiguousarray(swp_a, np.int32),
                sb=np.ascontiguousarray(swp_b, np.int32), sk=_f64(swp_K), qv=_f64(quote_vol))
    _I = C.POINTER(C.c_int32)
    args = [market.h, M, int(model.get("model", 0)), _dp(keep["par"]), _dp(keep["al"]), _dp(keep["sg"]), _dp(keep["ph"]), len(keep["cf"]),
            keep["cf"].ctypes.data_as(_I), _dp(keep["ck"]), len(keep["sa"]), keep["sa"].ctypes.data_as(_I),
            keep["sb"].ctypes.data_as(_I), _dp(keep["sk"]), _dp(keep["qv"])]
    return args, keep


def mc_objective(market, model, y, quote_vol, cap_fwd=(), cap_K=(), swp_a=(), swp_b=(), swp_K=(), n_paths=1000,
                 dt=0.01, mc_seed=1, n_threads=1):
    """f_s(y) = sum_k (P_k^Black - P_k^MC(y))^2 at the correlation parameters y = (eta1, lambda1,
    eta2, lambda2, lambda3) (see sabr_oracle.cpp mc_objective)."""
    args, keep = _mc_args(market, model, cap_fwd, cap_K, swp_a, swp_b, swp_K, quote_vol)
    yy = _f64(y)
    return market._lib.orc_mc_objective(*args, int(n_paths), float(dt), int(mc_seed), _dp(yy), int(n_threads))


def mc_anneal(market, model, quote_vol, lo, hi, free, n_chains, n_levels, steps, cooling, seed, cap_fwd=(), cap_K=(),
              swp_a=(), swp_b=(), swp_K=(), n_paths=1000, dt=0.01, mc_seed=1, T0=0.0, step_frac=0.1, step_floor=1e-3,
              y0=None, n_threads=1):
    """The annealing search of f_s over the correlation box (see sabr_oracle.cpp orc_mc_anneal)."""
    args, keep = _mc_args(market, model, cap_fwd, cap_K, swp_a, swp_b, swp_K, quote_vol)
    lo, hi = _f64(lo), _f64(hi)
    fr = np.ascontiguousarray(free, np.uint8)
    o = _SAOpts()
    o.n_chains, o.n_levels, o.steps = int(n_chains), int(n_levels), int(steps)
    o.T0, o.cooling, o.step_frac, o.step_floor = float(T0), float(cooling), float(step_frac), float(step_floor)
    o.seed, o.market_index, o.n_threads = int(seed), 0, int(n_threads)
    y0a = None if y0 is None else _f64(y0)
    o.x0 = _dp(y0a)
    yb, fb, tr, tx, t0 = np.zeros(5), np.zeros(1), np.zeros(n_levels), np.zeros((n_levels, 5)), np.zeros(1)
    market._lib.orc_mc_anneal(*args, int(n_paths), float(dt), int(mc_seed), _dp(lo), _dp(hi),
                              fr.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(o), _dp(yb), _dp(fb), _dp(tr), _dp(tx),
                              _dp(t0))
    return dict(y_best=yb, f_best=fb[0], trace_f=tr, trace_x=tx, T0=t0[0])


def quoted_market(skel, noise=True):
    """The market whose quotes are the oracle's model vols at skel.theta_true (+ skel.noise)."""
    m0 = Market(skel)
    v = m0.model_vols(skel.theta_true)
    if noise:
        v = v + skel.noise
    return Market(skel, v), v
