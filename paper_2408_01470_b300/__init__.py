"""B300-native SABR/LIBOR market-model calibration (arXiv 2408.01470), ctypes binding.

This module only marshals arguments into the C-ABI of ``libsabr_lmm.so`` (declared in
``include/sabr_lmm.h``); every number of the hot path is computed by the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: ``load()`` raises if the
library is missing or no CUDA device is visible.

Entry points (same names as the C-ABI, without the ``sabr_lmm_`` prefix):
    Market(...)                 sabr_lmm_load_market / sabr_lmm_free_market
    Market.objective(X, prec)   sabr_lmm_objective
    Market.model_vols(X, prec)  sabr_lmm_model_vols
    Market.residuals(X, prec)   sabr_lmm_residuals
    Market.nm_polish(X, ...)    sabr_lmm_nm_polish (the hybrid scheme's Nelder-Mead)
    Market.sync(stream)         sabr_lmm_sync (device-side wait timeouts of stream-ordered calls)
    Market.objective_grad(...)  sabr_lmm_objective_grad
    Market.anneal(...)          sabr_lmm_anneal
    Market.anneal_prepare(...)  sabr_lmm_anneal_prepare / _launch / _fetch / _plan_free
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsabr_lmm.so")

FP64, FP32, FP32_BF16X3 = 0, 1, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16x3": FP32_BF16X3}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTSUP"}

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)


class SabrLmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sabr_lmm {STATUS.get(status, status)}: {msg}")
        self.status = status


class MarketDesc(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("formula", C.c_int32), ("beta", C.c_double),
        ("n_fwd", C.c_int32), ("T", _D), ("P", _D),
        ("n_cap", C.c_int32), ("cap_fwd", _I32), ("cap_K", _D), ("cap_vol", _D), ("cap_w", _D),
        ("n_swp", C.c_int32), ("swp_start", _I32), ("swp_end", _I32), ("swp_K", _D),
        ("swp_vol", _D), ("swp_w", _D),
        ("n_param", C.c_int32), ("lo", _D), ("hi", _D), ("free_mask", _U8),
        ("panel", C.c_double), ("quad_nodes", C.c_int32),
    ]


class AnnealOpts(C.Structure):
    _fields_ = [
        ("n_chains", C.c_int32), ("n_levels", C.c_int32), ("steps_per_level", C.c_int32),
        ("T0", C.c_double), ("cooling", C.c_double), ("step_frac", C.c_double),
        ("step_floor", C.c_double), ("seed", C.c_uint64), ("x0", _D), ("prec", C.c_int32),
        ("lm_top_k", C.c_int32), ("lm_max_iter", C.c_int32), ("target_rmse_volpt", C.c_double),
        ("warps_per_block", C.c_int32), ("use_graph", C.c_int32), ("record_accepts", C.c_int32),
        ("polish_nm", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("x_best", _D), ("f_best", _D), ("rmse_volpt", _D), ("trace_f", _D),
        ("accept_bits", _U8), ("n_evals", C.c_int64), ("seconds", C.c_double),
        ("lm_seconds", C.c_double), ("T0_used", C.c_double), ("trace_x", _D), ("trace_seconds", _D),
    ]


class PlanConfig(C.Structure):
    _fields_ = [
        ("chains_per_cta", C.c_int32), ("grid", C.c_int32), ("cta_threads_swaptions", C.c_int32),
        ("n_buckets", C.c_int32), ("bucket_markets", C.c_int32 * 16), ("bucket_threads", C.c_int32 * 16),
        ("bucket_grid", C.c_int32 * 16), ("bucket_ctas_per_sm", C.c_int32 * 16),
    ]


class MarketInfo(C.Structure):
    _fields_ = [
        ("n_fwd", C.c_int32), ("n_cap", C.c_int32), ("n_swp", C.c_int32), ("n_swap", C.c_int32),
        ("n_panels", C.c_int32), ("n_diag", C.c_int32), ("max_window", C.c_int32),
        ("smem_fp64", C.c_uint32), ("smem_fp32", C.c_uint32),
        ("batch_ctas_per_sm_fp64", C.c_int32), ("batch_ctas_per_sm_fp32", C.c_int32),
    ]


class McDesc(C.Structure):
    _fields_ = [
        ("n_fwd", C.c_int32), ("T", _D), ("P", _D), ("beta", C.c_double), ("alpha", _D), ("sigma", _D),
        ("phi", _D), ("eta1", C.c_double), ("lambda1", C.c_double), ("eta2", C.c_double),
        ("lambda2", C.c_double), ("lambda3", C.c_double), ("n_cap", C.c_int32), ("cap_fwd", _I32),
        ("cap_K", _D), ("n_swp", C.c_int32), ("swp_start", _I32), ("swp_end", _I32), ("swp_K", _D),
        ("model", C.c_int32),
    ]


class McOpts(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("dt", C.c_double), ("seed", C.c_uint64), ("prec", C.c_int32),
                ("grid", C.c_int32)]


class McAnnealOpts(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("n_levels", C.c_int32), ("steps_per_level", C.c_int32),
                ("T0", C.c_double), ("cooling", C.c_double), ("step_frac", C.c_double), ("step_floor", C.c_double),
                ("seed", C.c_uint64), ("y0", _D), ("lo", _D), ("hi", _D), ("free_mask", _U8)]


class McAnnealResult(C.Structure):
    _fields_ = [("y_best", C.c_double * 5), ("f_best", C.c_double), ("T0_used", C.c_double), ("n_evals", C.c_int64),
                ("seconds", C.c_double), ("trace_f", _D), ("trace_y", _D)]


_lock = threading.Lock()
_lib = None

EXPORTS = ("sabr_lmm_load_market", "sabr_lmm_free_market", "sabr_lmm_objective", "sabr_lmm_model_vols",
           "sabr_lmm_objective_grad", "sabr_lmm_anneal", "sabr_lmm_anneal_prepare", "sabr_lmm_anneal_launch",
           "sabr_lmm_anneal_fetch", "sabr_lmm_anneal_plan_free", "sabr_lmm_anneal_noalloc", "sabr_lmm_lm_polish",
           "sabr_lmm_market_info", "sabr_lmm_selftest_wait", "sabr_lmm_quadrature_rule", "sabr_lmm_last_error",
           "sabr_lmm_version", "sabr_lmm_residuals", "sabr_lmm_sync", "sabr_lmm_test_raise_error",
           "sabr_lmm_nm_polish", "sabr_lmm_anneal_plan_config", "sabr_lmm_mc_prepare", "sabr_lmm_mc_launch",
           "sabr_lmm_mc_plan_free", "sabr_lmm_mc_price", "sabr_lmm_mc_anneal")


def open_library(path: str = LIB_PATH):
    """dlopen the library and declare its signatures (no CUDA call is made)."""
    if not os.path.exists(path):
        raise ImportError(f"the CUDA library {path} is missing; build it with "
                          "`python -m paper_2408_01470_b300.build`")
    lib = C.CDLL(path)
    lib.sabr_lmm_load_market.argtypes = [C.POINTER(MarketDesc), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.sabr_lmm_free_market.argtypes = [C.c_void_p]
    lib.sabr_lmm_free_market.restype = None
    for name in ("sabr_lmm_objective", "sabr_lmm_model_vols"):
        getattr(lib, name).argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    lib.sabr_lmm_objective_grad.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
    lib.sabr_lmm_residuals.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    lib.sabr_lmm_sync.argtypes = [C.c_void_p, C.c_void_p]
    lib.sabr_lmm_test_raise_error.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    lib.sabr_lmm_anneal.argtypes = [C.c_void_p, C.POINTER(AnnealOpts), C.POINTER(Result)]
    lib.sabr_lmm_anneal_prepare.argtypes = [C.c_void_p, C.POINTER(AnnealOpts), C.c_void_p, C.POINTER(C.c_void_p)]
    lib.sabr_lmm_anneal_launch.argtypes = [C.c_void_p, C.c_void_p]
    lib.sabr_lmm_anneal_fetch.argtypes = [C.c_void_p, C.POINTER(Result)]
    lib.sabr_lmm_anneal_plan_config.argtypes = [C.c_void_p, C.POINTER(PlanConfig)]
    lib.sabr_lmm_anneal_plan_free.argtypes = [C.c_void_p]
    lib.sabr_lmm_anneal_plan_free.restype = None
    lib.sabr_lmm_lm_polish.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_double,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sabr_lmm_nm_polish.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_double,
                                       C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sabr_lmm_market_info.argtypes = [C.c_void_p, C.c_int32, C.POINTER(MarketInfo)]
    lib.sabr_lmm_selftest_wait.argtypes = [C.c_int64, C.c_void_p]
    lib.sabr_lmm_quadrature_rule.argtypes = [C.c_int32, _D, _D]
    lib.sabr_lmm_mc_prepare.argtypes = [C.POINTER(McDesc), C.POINTER(McOpts), C.c_void_p, C.POINTER(C.c_void_p)]
    lib.sabr_lmm_mc_launch.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sabr_lmm_mc_plan_free.argtypes = [C.c_void_p]
    lib.sabr_lmm_mc_plan_free.restype = None
    lib.sabr_lmm_mc_price.argtypes = [C.POINTER(McDesc), C.POINTER(McOpts), _D, _D, C.POINTER(C.c_int64), C.c_void_p]
    lib.sabr_lmm_mc_anneal.argtypes = [C.POINTER(McDesc), _D, C.POINTER(McOpts), C.POINTER(McAnnealOpts),
                                       C.POINTER(McAnnealResult), C.c_void_p]
    lib.sabr_lmm_last_error.restype = C.c_char_p
    lib.sabr_lmm_version.restype = C.c_char_p
    return lib


def load():
    """The library, loaded once; raises if it is missing or no CUDA device is visible."""
    global _lib
    with _lock:
        if _lib is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("paper_2408_01470_b300 needs a CUDA device (B300, sm_103a); none is visible")
            torch.cuda.init()
            _lib = open_library()
    return _lib


def _check(status):
    if status != 0:
        raise SabrLmmError(status, _lib.sabr_lmm_last_error().decode())


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def selftest_wait(polls=4096, stream=None):
    """sabr_lmm_selftest_wait: the status of a bounded device wait that cannot complete (4 =
    SABR_LMM_ETIMEOUT is the expected outcome)."""
    lib = load()
    return lib.sabr_lmm_selftest_wait(int(polls), _stream_ptr(stream))


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def describe(skel, vols, weights=None):
    """A MarketDesc for a synth.Skeleton and quotes; returns (desc, keep-alive arrays)."""
    n_cap = skel.n_cap
    vols = _f64(vols)
    keep = dict(T=_f64(skel.T), P=_f64(skel.P), cap_fwd=np.ascontiguousarray(skel.cap_fwd, np.int32),
                cap_K=_f64(skel.cap_K), cap_vol=_f64(vols[:n_cap]),
                swp_start=np.ascontiguousarray(skel.swp_start, np.int32),
                swp_end=np.ascontiguousarray(skel.swp_end, np.int32), swp_K=_f64(skel.swp_K),
                swp_vol=_f64(vols[n_cap:]), lo=_f64(skel.lo), hi=_f64(skel.hi),
                free=np.ascontiguousarray(skel.free, np.uint8))
    d = MarketDesc()
    d.model, d.formula, d.beta = skel.model, skel.formula, skel.beta
    d.n_fwd = skel.n_fwd
    d.T, d.P = keep["T"].ctypes.data_as(_D), keep["P"].ctypes.data_as(_D)
    d.n_cap = n_cap
    d.cap_fwd = keep["cap_fwd"].ctypes.data_as(_I32)
    d.cap_K, d.cap_vol = keep["cap_K"].ctypes.data_as(_D), keep["cap_vol"].ctypes.data_as(_D)
    d.n_swp = skel.n_swp
    d.swp_start = keep["swp_start"].ctypes.data_as(_I32)
    d.swp_end = keep["swp_end"].ctypes.data_as(_I32)
    d.swp_K, d.swp_vol = keep["swp_K"].ctypes.data_as(_D), keep["swp_vol"].ctypes.data_as(_D)
    if weights is not None:
        w = _f64(weights)
        keep["cap_w"], keep["swp_w"] = _f64(w[:n_cap]), _f64(w[n_cap:])
        d.cap_w = keep["cap_w"].ctypes.data_as(_D)
        d.swp_w = keep["swp_w"].ctypes.data_as(_D)
    d.n_param = skel.n_param
    d.lo, d.hi = keep["lo"].ctypes.data_as(_D), keep["hi"].ctypes.data_as(_D)
    d.free_mask = keep["free"].ctypes.data_as(_U8)
    d.panel, d.quad_nodes = skel.panel, skel.quad_nodes
    return d, keep


class Market:
    """One or more markets loaded on the device (sabr_lmm_load_market)."""

    def __init__(self, skels, vols, weights=None, stream=None):
        import torch
        lib = load()
        if not isinstance(skels, (list, tuple)):
            skels, vols = [skels], [vols]
            weights = [weights]
        elif weights is None:
            weights = [None] * len(skels)
        self.skels = list(skels)
        descs = (MarketDesc * len(skels))()
        self._keep = []
        for j, (s, v, w) in enumerate(zip(skels, vols, weights)):
            d, keep = describe(s, v, w)
            descs[j] = d
            self._keep.append(keep)
        h = C.c_void_p()
        _check(lib.sabr_lmm_load_market(descs, len(skels), _stream_ptr(stream), C.byref(h)))
        self.h = h
        self._lib = lib
        self._torch = torch

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            self._lib.sabr_lmm_free_market(self.h)
            self.h = C.c_void_p()

    def _X(self, X, j):
        t = self._torch
        if not isinstance(X, t.Tensor):
            X = t.as_tensor(np.atleast_2d(X), dtype=t.float64)
        X = X.to(device="cuda", dtype=t.float64).contiguous()
        if X.dim() == 1:
            X = X[None, :]
        assert X.shape[1] == self.skels[j].n_param
        return X

    def objective(self, X, prec="fp64", market=0, stream=None):
        X = self._X(X, market)
        f = self._torch.empty(X.shape[0], dtype=self._torch.float64, device="cuda")
        _check(self._lib.sabr_lmm_objective(self.h, market, C.c_void_p(X.data_ptr()), X.shape[0], _prec(prec),
                                            C.c_void_p(f.data_ptr()), _stream_ptr(stream)))
        return f

    def model_vols(self, X, prec="fp64", market=0, stream=None):
        X = self._X(X, market)
        n_instr = self.skels[market].n_instr
        v = self._torch.empty((X.shape[0], n_instr), dtype=self._torch.float64, device="cuda")
        _check(self._lib.sabr_lmm_model_vols(self.h, market, C.c_void_p(X.data_ptr()), X.shape[0], _prec(prec),
                                             C.c_void_p(v.data_ptr()), _stream_ptr(stream)))
        return v

    def residuals(self, X, prec="fp64", market=0, stream=None):
        """sabr_lmm_residuals: (f, r) with r[i, k] = sqrt(w_k) (P_k(X[i]) - P_k^mkt) from the pricer
        the search runs at this precision (device tensors)."""
        X = self._X(X, market)
        n_instr = self.skels[market].n_instr
        f = self._torch.empty(X.shape[0], dtype=self._torch.float64, device="cuda")
        r = self._torch.empty((X.shape[0], n_instr), dtype=self._torch.float64, device="cuda")
        _check(self._lib.sabr_lmm_residuals(self.h, market, C.c_void_p(X.data_ptr()), X.shape[0], _prec(prec),
                                            C.c_void_p(f.data_ptr()), C.c_void_p(r.data_ptr()), _stream_ptr(stream)))
        return f, r

    def sync(self, stream=None):
        """sabr_lmm_sync: synchronise the stream and raise SabrLmmError (ETIMEOUT) if a device-side
        wait of a call on these markets gave up since the last check."""
        _check(self._lib.sabr_lmm_sync(self.h, _stream_ptr(stream)))

    def test_raise_error(self, market=0, stream=None):
        """sabr_lmm_test_raise_error: raise the market's error word from the host (failure-detection
        tests)."""
        _check(self._lib.sabr_lmm_test_raise_error(self.h, market, _stream_ptr(stream)))

    def objective_grad(self, X, prec="fp64", market=0, stream=None):
        X = self._X(X, market)
        n = X.shape[0]
        f = self._torch.empty(n, dtype=self._torch.float64, device="cuda")
        G = self._torch.empty_like(X)
        _check(self._lib.sabr_lmm_objective_grad(self.h, market, C.c_void_p(X.data_ptr()), n, _prec(prec),
                                                 C.c_void_p(f.data_ptr()), C.c_void_p(G.data_ptr()),
                                                 _stream_ptr(stream)))
        return f, G

    def calibration_objective(self, X, prec="fp64", market=0):
        """f(X) as a differentiable torch op: the forward and the backward both come from
        sabr_lmm_objective_grad (the hand-written adjoint), through CalibrationObjective."""
        return CalibrationObjective.apply(X, self, prec, market)

    def info(self, market=0):
        """sabr_lmm_market_info: geometry and per-CTA resources of one market, as a dict."""
        out = MarketInfo()
        _check(self._lib.sabr_lmm_market_info(self.h, market, C.byref(out)))
        return {name: getattr(out, name) for name, _ in MarketInfo._fields_}

    def lm_polish(self, X, max_iter=50, target_rmse=0.0, market=0, stream=None):
        """sabr_lmm_lm_polish: returns (X polished, f, rmse in vol points) as device tensors."""
        X = self._X(X, market).clone()
        n = X.shape[0]
        f = self._torch.empty(n, dtype=self._torch.float64, device="cuda")
        r = self._torch.empty(n, dtype=self._torch.float64, device="cuda")
        _check(self._lib.sabr_lmm_lm_polish(self.h, market, C.c_void_p(X.data_ptr()), n, int(max_iter),
                                            float(target_rmse), C.c_void_p(f.data_ptr()), C.c_void_p(r.data_ptr()),
                                            _stream_ptr(stream)))
        return X, f, r

    def nm_polish(self, X, max_iter=500, step=0.02, ftol=1e-12, market=0, stream=None):
        """sabr_lmm_nm_polish: returns (X polished, f, evaluations) as device tensors."""
        X = self._X(X, market).clone()
        n = X.shape[0]
        f = self._torch.empty(n, dtype=self._torch.float64, device="cuda")
        ev = self._torch.zeros(n, dtype=self._torch.int32, device="cuda")
        _check(self._lib.sabr_lmm_nm_polish(self.h, market, C.c_void_p(X.data_ptr()), n, int(max_iter), float(step),
                                            float(ftol), C.c_void_p(f.data_ptr()), C.c_void_p(ev.data_ptr()),
                                            _stream_ptr(stream)))
        return X, f, ev

    def _opts(self, n_chains, n_levels, steps, cooling, seed, prec, T0, step_frac, step_floor, x0,
              lm_top_k, lm_max_iter, target_rmse, warps_per_block, use_graph, record_accepts, polish_nm=False):
        o = AnnealOpts()
        o.n_chains, o.n_levels, o.steps_per_level = n_chains, n_levels, steps
        o.T0, o.cooling, o.step_frac, o.step_floor = T0, cooling, step_frac, step_floor
        o.seed = seed
        keep = None
        if x0 is not None:
            keep = _f64(x0).reshape(-1)
            o.x0 = keep.ctypes.data_as(_D)
        o.prec = _prec(prec)
        o.lm_top_k, o.lm_max_iter, o.target_rmse_volpt = lm_top_k, lm_max_iter, target_rmse
        o.warps_per_block, o.use_graph, o.record_accepts = warps_per_block, int(use_graph), int(record_accepts)
        o.polish_nm = int(polish_nm)
        return o, keep

    def _result(self, n_chains, n_levels, steps, record_accepts):
        nm = len(self.skels)
        P = self.skels[0].n_param
        arrs = dict(x_best=np.zeros((nm, P)), f_best=np.zeros(nm), rmse=np.zeros(nm),
                    trace_f=np.zeros((nm, n_levels)), trace_x=np.zeros((nm, n_levels, P)),
                    trace_seconds=np.zeros((nm, n_levels)))
        bits = np.zeros((n_chains, n_levels, steps), np.uint8) if record_accepts else None
        r = Result()
        r.x_best = arrs["x_best"].ctypes.data_as(_D)
        r.f_best = arrs["f_best"].ctypes.data_as(_D)
        r.rmse_volpt = arrs["rmse"].ctypes.data_as(_D)
        r.trace_f = arrs["trace_f"].ctypes.data_as(_D)
        r.trace_x = arrs["trace_x"].ctypes.data_as(_D)
        r.trace_seconds = arrs["trace_seconds"].ctypes.data_as(_D)
        if bits is not None:
            r.accept_bits = bits.ctypes.data_as(_U8)
        return r, arrs, bits

    @staticmethod
    def _pack(r, arrs, bits):
        return dict(x_best=arrs["x_best"], f_best=arrs["f_best"], rmse_volpt=arrs["rmse"],
                    trace_f=arrs["trace_f"], trace_x=arrs["trace_x"], trace_seconds=arrs["trace_seconds"],
                    bits=bits, n_evals=r.n_evals, seconds=r.seconds, lm_seconds=r.lm_seconds, T0=r.T0_used)

    def anneal(self, n_chains, n_levels, steps, cooling, seed, prec="fp64", T0=0.0, step_frac=0.1,
               step_floor=1e-3, x0=None, lm_top_k=0, lm_max_iter=50, target_rmse=0.0,
               warps_per_block=0, use_graph=False, record_accepts=False, polish_nm=False):
        o, keep = self._opts(n_chains, n_levels, steps, cooling, seed, prec, T0, step_frac, step_floor, x0,
                             lm_top_k, lm_max_iter, target_rmse, warps_per_block, use_graph, record_accepts,
                             polish_nm)
        r, arrs, bits = self._result(n_chains, n_levels, steps, record_accepts)
        _check(self._lib.sabr_lmm_anneal(self.h, C.byref(o), C.byref(r)))
        del keep
        return self._pack(r, arrs, bits)

    def anneal_prepare(self, n_chains, n_levels, steps, cooling, seed, prec="fp64", T0=0.0, step_frac=0.1,
                       step_floor=1e-3, x0=None, lm_top_k=0, lm_max_iter=50, target_rmse=0.0,
                       warps_per_block=0, use_graph=True, stream=None, polish_nm=False):
        o, keep = self._opts(n_chains, n_levels, steps, cooling, seed, prec, T0, step_frac, step_floor, x0,
                             lm_top_k, lm_max_iter, target_rmse, warps_per_block, use_graph, False, polish_nm)
        h = C.c_void_p()
        _check(self._lib.sabr_lmm_anneal_prepare(self.h, C.byref(o), _stream_ptr(stream), C.byref(h)))
        return AnnealPlan(self, h, (n_chains, n_levels, steps))


class AnnealPlan:
    """sabr_lmm_anneal_prepare / launch / fetch / plan_free."""

    def __init__(self, market, h, dims):
        self.market, self.h, self.dims = market, h, dims
        self._lib = market._lib

    def launch(self, stream=None):
        _check(self._lib.sabr_lmm_anneal_launch(self.h, _stream_ptr(stream)))

    def config(self):
        """sabr_lmm_anneal_plan_config: the launch configuration the plan chose, as a dict."""
        c = PlanConfig()
        _check(self._lib.sabr_lmm_anneal_plan_config(self.h, C.byref(c)))
        nb = c.n_buckets
        return {"chains_per_cta": c.chains_per_cta, "grid": c.grid,
                "cta_threads_swaptions": c.cta_threads_swaptions,
                "buckets": [{"markets": c.bucket_markets[i], "threads": c.bucket_threads[i],
                             "grid": c.bucket_grid[i], "ctas_per_sm": c.bucket_ctas_per_sm[i]}
                            for i in range(nb)]}

    def fetch(self):
        C_, L, N = self.dims
        r, arrs, bits = self.market._result(C_, L, N, False)
        _check(self._lib.sabr_lmm_anneal_fetch(self.h, C.byref(r)))
        return Market._pack(r, arrs, bits)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            self._lib.sabr_lmm_anneal_plan_free(self.h)
            self.h = C.c_void_p()


def quadrature_rule(q: int = 8):
    lib = _lib or open_library()
    x, w = np.zeros(q), np.zeros(q)
    st = lib.sabr_lmm_quadrature_rule(q, x.ctypes.data_as(_D), w.ctypes.data_as(_D))
    if st != 0:
        raise SabrLmmError(st, lib.sabr_lmm_last_error().decode())
    return x, w


def _autograd_function():
    import torch

    class CalibrationObjective(torch.autograd.Function):
        """f = sum_k w_k (P_k(theta) - P_k^mkt)^2 per row of X (n x n_param, float64, CUDA) with the
        gradient of the library's reverse sweep: forward runs sabr_lmm_objective_grad once and keeps
        G = df/dtheta; backward returns grad_f[:, None] * G.  Second derivatives are not provided."""

        @staticmethod
        def forward(ctx, X, market, prec="fp64", index=0):
            f, G = market.objective_grad(X.detach(), prec=prec, market=index)
            ctx.save_for_backward(G)
            return f

        @staticmethod
        def backward(ctx, grad_f):
            (G,) = ctx.saved_tensors
            return grad_f[:, None] * G, None, None, None

    return CalibrationObjective


class _LazyFunction:
    """Defers `import torch` until first use (the binding imports without torch for ABI checks)."""

    def __init__(self):
        self._cls = None

    def apply(self, *args):
        if self._cls is None:
            self._cls = _autograd_function()
        return self._cls.apply(*args)


CalibrationObjective = _LazyFunction()


# ---------------------------------------------------------------- Monte Carlo pricer
def mc_describe(T, P, model, cap_fwd=(), cap_K=(), swp_start=(), swp_end=(), swp_K=()):
    """An McDesc for a tenor structure (T, P) and a model dict: beta, eta1, lambda1, per-forward
    alpha, sigma, phi; for the Hagan dynamics also eta2, lambda2, lambda3; "model": 2 selects the
    Mercurio & Morini dynamics (sigma[0] the common vol of vol).  Returns (desc, keep-alive arrays)."""
    n_fwd = len(T) - 1
    keep = dict(T=_f64(T), P=_f64(P), alpha=_f64(np.resize(model["alpha"], n_fwd)),
                sigma=_f64(np.resize(model["sigma"], n_fwd)), phi=_f64(np.resize(model["phi"], n_fwd)),
                cap_fwd=np.ascontiguousarray(cap_fwd, np.int32), cap_K=_f64(cap_K),
                swp_start=np.ascontiguousarray(swp_start, np.int32), swp_end=np.ascontiguousarray(swp_end, np.int32),
                swp_K=_f64(swp_K))
    d = McDesc()
    d.n_fwd = n_fwd
    d.T, d.P = keep["T"].ctypes.data_as(_D), keep["P"].ctypes.data_as(_D)
    d.beta = float(model["beta"])
    d.alpha, d.sigma, d.phi = (keep[k].ctypes.data_as(_D) for k in ("alpha", "sigma", "phi"))
    d.eta1, d.lambda1, d.eta2 = float(model["eta1"]), float(model["lambda1"]), float(model.get("eta2", 0.0))
    d.lambda2, d.lambda3 = float(model.get("lambda2", 0.0)), float(model.get("lambda3", 0.0))
    d.model = int(model.get("model", 0))
    d.n_cap = len(keep["cap_fwd"])
    d.cap_fwd, d.cap_K = keep["cap_fwd"].ctypes.data_as(_I32), keep["cap_K"].ctypes.data_as(_D)
    d.n_swp = len(keep["swp_start"])
    d.swp_start, d.swp_end = keep["swp_start"].ctypes.data_as(_I32), keep["swp_end"].ctypes.data_as(_I32)
    d.swp_K = keep["swp_K"].ctypes.data_as(_D)
    return d, keep


def _mc_opts(n_paths, dt, seed, prec, grid):
    o = McOpts()
    o.n_paths, o.dt, o.seed, o.prec, o.grid = int(n_paths), float(dt), int(seed), _prec(prec), int(grid)
    return o


def mc_price(T, P, model, cap_fwd=(), cap_K=(), swp_start=(), swp_end=(), swp_K=(), n_paths=100000, dt=0.01,
             seed=1, prec="fp32", grid=0, stream=None):
    """sabr_lmm_mc_price: Monte Carlo prices (caplets, then swaptions), their standard errors and
    the count of stopped paths, as numpy arrays (synchronous)."""
    lib = load()
    d, keep = mc_describe(T, P, model, cap_fwd, cap_K, swp_start, swp_end, swp_K)
    o = _mc_opts(n_paths, dt, seed, prec, grid)
    ni = d.n_cap + d.n_swp
    price, se, nb = np.zeros(max(ni, 1)), np.zeros(max(ni, 1)), C.c_int64(0)
    _check(lib.sabr_lmm_mc_price(C.byref(d), C.byref(o), price.ctypes.data_as(_D), se.ctypes.data_as(_D),
                                 C.byref(nb), _stream_ptr(stream)))
    del keep
    return price[:ni], se[:ni], nb.value


class McPlan:
    """sabr_lmm_mc_prepare / launch / plan_free: the model's constants and device buffers, priced
    again and again (launch is stream-ordered; outputs are device tensors)."""

    def __init__(self, T, P, model, cap_fwd=(), cap_K=(), swp_start=(), swp_end=(), swp_K=(), n_paths=100000,
                 dt=0.01, seed=1, prec="fp32", grid=0, stream=None):
        import torch
        self._lib = load()
        d, keep = mc_describe(T, P, model, cap_fwd, cap_K, swp_start, swp_end, swp_K)
        o = _mc_opts(n_paths, dt, seed, prec, grid)
        h = C.c_void_p()
        _check(self._lib.sabr_lmm_mc_prepare(C.byref(d), C.byref(o), _stream_ptr(stream), C.byref(h)))
        del keep
        self.h = h
        self.n_instr = d.n_cap + d.n_swp
        dev = torch.device("cuda", torch.cuda.current_device())
        self.price = torch.zeros(self.n_instr, dtype=torch.float64, device=dev)
        self.stderr = torch.zeros(self.n_instr, dtype=torch.float64, device=dev)
        self.n_bad = torch.zeros(1, dtype=torch.int64, device=dev)

    def launch(self, stream=None):
        _check(self._lib.sabr_lmm_mc_launch(self.h, C.c_void_p(self.price.data_ptr()),
                                            C.c_void_p(self.stderr.data_ptr()), C.c_void_p(self.n_bad.data_ptr()),
                                            _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.sabr_lmm_mc_plan_free(self.h)
            self.h = None


def mc_anneal(T, P, model, quote_vol, lo, hi, free, n_chains, n_levels, steps, cooling, seed, cap_fwd=(), cap_K=(),
              swp_start=(), swp_end=(), swp_K=(), n_paths=10000, dt=0.02, mc_seed=1, prec="fp32", T0=0.0,
              step_frac=0.1, step_floor=1e-3, y0=None, stream=None):
    """sabr_lmm_mc_anneal: the correlation parameters (eta1, lambda1, eta2, lambda2, lambda3) by
    simulated annealing over the Monte Carlo objective; returns a dict (synchronous)."""
    lib = load()
    d, keep = mc_describe(T, P, model, cap_fwd, cap_K, swp_start, swp_end, swp_K)
    mo = _mc_opts(n_paths, dt, mc_seed, prec, 0)
    qv = _f64(quote_vol)
    lo, hi = _f64(lo), _f64(hi)
    fr = np.ascontiguousarray(free, np.uint8)
    o = McAnnealOpts()
    o.n_chains, o.n_levels, o.steps_per_level = int(n_chains), int(n_levels), int(steps)
    o.T0, o.cooling, o.step_frac, o.step_floor, o.seed = float(T0), float(cooling), float(step_frac), \
        float(step_floor), int(seed)
    y0a = None if y0 is None else _f64(y0)
    o.y0 = None if y0a is None else y0a.ctypes.data_as(_D)
    o.lo, o.hi, o.free_mask = lo.ctypes.data_as(_D), hi.ctypes.data_as(_D), fr.ctypes.data_as(_U8)
    tf, ty = np.zeros(n_levels), np.zeros((n_levels, 5))
    r = McAnnealResult()
    r.trace_f, r.trace_y = tf.ctypes.data_as(_D), ty.ctypes.data_as(_D)
    _check(lib.sabr_lmm_mc_anneal(C.byref(d), qv.ctypes.data_as(_D), C.byref(mo), C.byref(o), C.byref(r),
                                  _stream_ptr(stream)))
    del keep
    return dict(y_best=np.array(r.y_best[:]), f_best=r.f_best, T0=r.T0_used, n_evals=r.n_evals, seconds=r.seconds,
                trace_f=tf, trace_y=ty)
