"""Benchmark: instrument prices per second inside the simulated-annealing objective.

One step = one complete annealing search of the Rebonato SABR/LIBOR caplet term structure
(20 semi-annual forwards x 15 strikes = 300 caplets; 4096 chains x 200 temperatures x 100
Metropolis steps, cooling 0.95): proposal (S1), per-forward SABR parameters by quadrature (S2),
caplet pricing (S4), objective sum (S7), Metropolis and the per-temperature best-chain
reduction (S8).  Inputs are synthetic (seeded), resident in HBM before the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64] [--impl reference]

Besides the headline value the line carries `variants.fp64` (the FP64 plain form of the same
search), `workloads` (the joint 40-forward caplet + swaption market over its full 200-level
schedule in FP32 with its own roofline and oracle baseline, one level of it in FP64 and with the
BF16-split tensor-core Grams, the paper's real-data caplet calibration over its full schedule, one
level of the 256-market batch) and `time_to_target` (0.05 vol-pt and the FP64 form's final true
vol RMSE: FP64 plain, FP32, and the FP32 search with the Levenberg-Marquardt polish).  Shortened
samples say so (`extrapolated`, `levels_timed` against `levels_of_schedule`).

Other modes: `--workload joint|batch|caplets` (that workload's full schedule as its own line),
`--quality --workload W --seeds S` (final true vol RMSE of FP32 against FP64 over S seeds, with and
without the polish), `--profile` (one search, for ncu launch lists).

Multi-GPU runs (torchrun, one process per GPU) are independent replicas: the search does not
shard, so no collective touches the data path; rank r anneals with seed + r and the aggregate
counts every rank's prices over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "instrument prices/s in SA objective; time-to-target-RMSE vs FP64 plain form"
UNIT = "prices/s"
WORKLOAD = "rebonato_caplets_20fwd_x_15k_4096ch_x_200T_x_100steps"
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # FP32 FMA lanes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 1.25                              # nominal B300 FP64 rate
# DRAM bytes (read + write) of one FP32 level launch of sa_level_kernel on this workload, from an ncu
# capture of the kernel as it is built now (dram__bytes_read.sum 510,976 B, dram__bytes_write.sum 0 B,
# second level of a 3-level search of 28-chain CTAs); the market and chain state stay in L2 across
# launches
LEVEL_TRAFFIC_BYTES_FP32 = 510_976
TARGET_RMSE_VOLPT = 0.05


def flops_per_chain_step(skel, info=None) -> float:
    """Algorithmic floating-point operations of one objective evaluation plus one Metropolis step.

    Counted from the arithmetic as written (add, mul = 1; fma = 2; div, sqrt, exp, log1p, erfc = 1):
      S2 (caplet forwards), per (panel, node): g and h (5 each), eight inner nodes (8 each), three
          weighted sums (5) = 79; per forward: 4 per panel + 6;
      S4 / S6, per instrument: SABR with z/x(z) 35, Black 15, weighted residual 3 = 53;
      S1 + S8: 6 per free slot + 4;
    and for markets with swaptions (info = the market's geometry, sabr_lmm_market_info):
      S3, Y rows: per (absolute panel, outer node) g and h at the node = 24;
          pair Grams per (diagonal, panel) cell: G and H (8 products each, 16 flop each) and the
          inner-rule bilinear form at 8 nodes (6 fma + 2) = 144; prefix sums 24 per cell
          (float-float G and G x H prefixes);
          window integrals per (expiry group, pair of its window) 16;
      S5, per swap: 3 quadratic forms over its window's L (L + 1) / 2 pairs (1 fma each);
      swap-rate SABR parameters per swap 20.
    """
    free = int(np.asarray(skel.free).sum())
    s1 = 6 * free + 4
    s4 = 53 * (skel.n_cap + skel.n_swp)
    s2 = 0
    if skel.model == 1 and skel.n_cap > 0:
        fwds = sorted(set(np.asarray(skel.cap_fwd).tolist()))
        NP = int(round(max(skel.T[i] for i in fwds) / skel.panel))
        s2 = NP * 8 * 79 + sum(4 * int(round(skel.T[i] / skel.panel)) + 6 for i in fwds)
    s3 = s5 = 0
    if skel.n_swp > 0:
        NA, ND = int(info["n_panels"]), int(info["n_diag"])
        cells = sum(NA - e for e in range(ND))
        swaps = sorted(set(zip(np.asarray(skel.swp_start).tolist(), np.asarray(skel.swp_end).tolist())))
        glen = {}
        for a, b in swaps:
            glen[a] = max(glen.get(a, 0), b - a)
        pairs_g = sum(L * (L + 1) // 2 for L in glen.values())
        s3 = NA * 8 * 24 + cells * (144 + 24) + 16 * pairs_g + 20 * len(swaps)
        s5 = sum(3 * 2 * ((b - a) * (b - a + 1) // 2) for a, b in swaps)
    return float(s1 + s2 + s3 + s4 + s5)


def measure_peaks(stream_ptr=None):
    """Pipe throughputs measured on this GPU (libsabr_peaks.so, CUDA events, 8 CTAs of 256 threads
    per SM, 8 independent chains per thread, best of 3): FP32 FMA (scalar and on register pairs),
    FP64 FMA, MUFU ex2.  TFLOP/s count 2 flop per FMA."""
    import ctypes as C
    import torch
    from paper_2408_01470_b300 import build
    lib = C.CDLL(build.PEAKS_LIB)
    lib.sabr_peak_probe.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    iters = {0: 1 << 15, 1: 1 << 14, 2: 1 << 9, 3: 1 << 13}
    out = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32x2_fma"), (2, "fp64_fma"), (3, "mufu_ex2")):
        best = 0.0
        for _ in range(3):
            sec, ops = C.c_double(), C.c_double()
            rc = lib.sabr_peak_probe(kind, nsm * 8, 256, iters[kind], stream_ptr, C.byref(sec), C.byref(ops))
            if rc != 0:
                raise RuntimeError(f"sabr_peak_probe({kind}) failed: CUDA error {rc}")
            best = max(best, ops.value / sec.value)
        out[name] = best
    return {"fp32_tflops": 2 * max(out["fp32_fma"], out["fp32x2_fma"]) / 1e12,
            "fp32_scalar_tflops": 2 * out["fp32_fma"] / 1e12, "fp32x2_tflops": 2 * out["fp32x2_fma"] / 1e12,
            "fp64_tflops": 2 * out["fp64_fma"] / 1e12, "mufu_gops": out["mufu_ex2"] / 1e9, "sms": nsm,
            "how": "libsabr_peaks.so: FMA / ex2 chains, 8 CTAs x 256 threads per SM, best of 3, CUDA events"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int, out_dir: str = ""):
        self.gpu = gpu
        self.p = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(), f"clocks_gpu{gpu}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.fh.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(local_seconds: float, units_per_rank: float, ws: int):
    """Whole-job throughput of ws replicas: every rank's units over the slowest rank's time.
    Returns (units per second, the max-over-ranks seconds)."""
    t = reduce_max(local_seconds, ws)
    return ws * units_per_rank / t, t


def replica_seed(base: int, rank: int) -> int:
    """Rank r runs an independent replica of the search with seed base + r."""
    return base + rank


WORKLOADS = {
    "caplets": "rebonato_caplets_20fwd_x_15k_4096ch_x_200T_x_100steps",
    "joint": "rebonato_joint_40fwd_300caplets_700swaptions_16384ch_x_200T_x_100steps",
    "batch": "rebonato_batch_256_markets_10to60fwd_50to1000instr_4096ch_x_100T_x_50steps",
}
PREC_DTYPE = {"fp32": "f32", "fp64": "f64", "bf16x3": "f32+bf16x3"}


def workload_markets(lib, name, markets=0):
    """(Market, skeletons, quotes list, chains, levels, steps, cooling) of a named workload (the
    batch: its first `markets` markets when markets > 0).  The quotes are the library's own FP64
    model vols at the generating point plus the noise draws."""
    from paper_2408_01470_b300 import synth
    if name == "caplets":
        sks = [synth.caplet_term_structure()]
    elif name == "joint":
        sks = [synth.joint_caplet_swaption()]
    else:
        sks = [synth.batch_market(j) for j in range(markets if markets > 0 else 256)]
    vols = []
    for sk in sks:
        placeholder = lib.Market(sk, np.full(sk.n_instr, 0.2))
        v = placeholder.model_vols(sk.theta_true, "fp64").cpu().numpy()[0]
        del placeholder
        vols.append(v + sk.noise)
    gm = lib.Market(sks, vols) if len(sks) > 1 else lib.Market(sks[0], vols[0])
    s0 = sks[0]
    return gm, sks, vols, s0.n_chains, s0.n_levels, s0.steps, s0.cooling


def market_from_library(lib, skel):
    """Quotes for the bench made by the library itself: model vols at the generating point + noise."""
    import torch
    placeholder = lib.Market(skel, np.full(skel.n_instr, 0.2))
    v = placeholder.model_vols(skel.theta_true, "fp64").cpu().numpy()[0]
    del placeholder
    torch.cuda.synchronize()
    vols = v + skel.noise
    return lib.Market(skel, vols), vols


def cpu_baseline(skel, vols, levels=1, steps=100, chains=None, threads=None):
    """The oracle as it stands on the host cores, on a bounded sample of the workload."""
    import oracle
    om = oracle.Market(skel, vols)
    threads = threads or os.cpu_count() or 1
    chains = chains or skel.n_chains
    t0 = time.perf_counter()
    r = om.anneal(chains, levels, steps, skel.cooling, seed=240801470, n_threads=threads)
    dt = time.perf_counter() - t0
    prices = r["n_evals"] * skel.n_instr
    return {"value": prices / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "chain_steps_per_s": chains * levels * steps / dt,
            "sample": f"{chains} chains x {levels} temperature level x {steps} steps of the same market "
                      f"({r['n_evals']} objective evaluations, {dt:.1f} s wall, {threads} threads)"}


def run_reference(args):
    from paper_2408_01470_b300 import synth
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    skel = synth.caplet_term_structure()
    om0 = oracle.Market(skel)
    vols = om0.model_vols(skel.theta_true) + skel.noise
    vals = []
    base = None
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(skel, vols, levels=1, steps=20)
        if i >= args.warmup:
            vals.append(b["value"])
            base = b
    value = statistics.median(vals)
    step_s = skel.n_chains * (skel.n_levels * skel.steps + 1) * skel.n_instr / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": base["sample"]},
            "extrapolated": {"ms_per_step": True, "value": False,
                             "how": "value is measured on the sample; ms_per_step is the full workload "
                                    "(4096 x (200 x 100 + 1) evaluations x 300 caplets) at that rate"},
            "cpu_baseline": {**base, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """One search of a workload (levels shortened with --levels), for ncu captures."""
    import paper_2408_01470_b300 as lib
    import torch
    lib.load()
    gm, sks, _, C, L0, N, cooling = workload_markets(lib, args.workload)
    L = args.levels or L0
    C = args.chains or C
    s = torch.cuda.Stream()
    plan = gm.anneal_prepare(C, L, N, cooling, 240801470, prec=args.prec,
                             use_graph=False, stream=s, warps_per_block=args.warps_per_block,
                             lm_top_k=args.lm_top_k, lm_max_iter=50, target_rmse=TARGET_RMSE_VOLPT)
    for _ in range(2):
        plan.launch(stream=s)
        r = plan.fetch()
    prices = sum(sk.n_instr for sk in sks) * r["n_evals"]
    print(json.dumps({"profile": True, "workload": args.workload, "chains": C, "levels": L, "prec": args.prec,
                      "f_best": float(r["f_best"][0]), "seconds": r["seconds"],
                      "prices_per_s": prices / r["seconds"], "ms_per_level": 1e3 * r["seconds"] / L,
                      "lm_top_k": args.lm_top_k, "lm_seconds": r["lm_seconds"],
                      "rmse_volpt": float(r["rmse_volpt"][0])}))


def run_mc_profile(args):
    """Three launches of the Monte Carlo pricer on the paper's Hagan model (its 117 caplets, FP32),
    or with --mc-model mm its Mercurio & Morini model on the same caplets, --mc-paths paths at
    --mc-dt, for ncu captures."""
    import paper_2408_01470_b300 as lib
    import torch
    from paper_2408_01470_b300 import synth
    lib.load()
    sk, model, cf, ck, _ = synth.paper_hagan_mc_model(PAPER_DATA, PAPER_MM, PAPER_MC)
    if args.mc_model == "mm":
        sk, model = synth.paper_mm_mc_model(PAPER_DATA, PAPER_MM)
    s = torch.cuda.Stream()
    plan = lib.McPlan(sk.T, sk.P, model, cf, ck, n_paths=args.mc_paths, dt=args.mc_dt, seed=1, prec=args.prec,
                      stream=s)
    for _ in range(3):
        plan.launch(s)
    s.synchronize()
    print(json.dumps({"mc_profile": True, "model": args.mc_model, "paths": args.mc_paths, "dt": args.mc_dt, "prec": args.prec,
                      "price_first": float(plan.price[0].item()), "n_bad": int(plan.n_bad.item())}))


def rmse_per_level(gm, trace_x, quotes, market=0):
    """The true vol RMSE (vol points) of each level's start point: FP64 model vols against the quotes."""
    v = gm.model_vols(trace_x, "fp64", market=market).cpu().numpy()
    return 100.0 * np.sqrt(np.mean((v - np.asarray(quotes)[None, :]) ** 2, axis=1))


def rmse_trace(gm, r, quotes):
    """(true vol RMSE, device seconds) of each level's best end point and, last, of the search's
    result (the best point ever accepted, taken by the final reduction right after the last level)."""
    rm = rmse_per_level(gm, r["trace_x"][0], quotes)
    sec = np.asarray(r["trace_seconds"][0], dtype=np.float64)
    return np.append(rm, float(r["rmse_volpt"][0])), np.append(sec, sec[-1])


def first_hit(rmse, seconds, target):
    """(level, device seconds from the search's start) of the first entry of a trace that reaches the
    target RMSE, or None (level L + 1: the search's final result)."""
    hit = np.nonzero(rmse <= target)[0]
    return None if hit.size == 0 else {"level": int(hit[0]) + 1, "seconds": float(seconds[hit[0]])}


def roofline_alu(flops_per_launch, level_s, peak_tflops, traffic, kernel, source):
    achieved = flops_per_launch / level_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic, "kernel": kernel, "peak_source": source}


def search_record(lib, name, prec, seed, stream, peaks, levels=None, cpu=None, e2e=True, chains=None,
                  warps_per_block=0):
    """One timed search of a named workload (after a 2-level warm-up of the same kernels), with its
    rate, roofline, quality, end-to-end rate and (cpu = dict of sample sizes) the oracle baseline."""
    import torch
    gm, sks, vols, C, L0, N, cool = workload_markets(lib, name)
    C = chains or C
    L = levels or L0
    warm = gm.anneal_prepare(C, min(2, L), N, cool, seed, prec=prec, use_graph=True, stream=stream,
                             warps_per_block=warps_per_block)
    warm.launch(stream=stream)
    warm.fetch()
    del warm
    plan = gm.anneal_prepare(C, L, N, cool, seed, prec=prec, use_graph=True, stream=stream,
                             warps_per_block=warps_per_block)
    tuning = plan.config()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    stream.synchronize()
    t = a.elapsed_time(b) / 1e3
    r = plan.fetch()
    del plan
    n_instr = sum(sk.n_instr for sk in sks)
    rec = {"workload": WORKLOADS[name] if L == L0 and C == sks[0].n_chains else
           f"{name}: {C} chains x {L} levels x {N} steps", "prec": prec, "chains": C, "levels_timed": L,
           "levels_of_schedule": L0, "extrapolated": L != L0, "value": r["n_evals"] * n_instr / t, "unit": UNIT,
           "seconds": t, "ms_per_level": 1e3 * t / L, "chain_steps_per_s": C * L * N * len(sks) / t,
           "rmse_volpt": float(np.median(r["rmse_volpt"])), "tuning": tuning}
    if len(sks) == 1:
        info = gm.info()
        fl = C * N * flops_per_chain_step(sks[0], info)
        peak, src = ((peaks["fp32_tflops"], "measured FP32 FMA rate (libsabr_peaks.so)") if prec != "fp64" else
                     (peaks["fp64_tflops"], "measured FP64 FMA rate (libsabr_peaks.so)"))
        kern = "sa_level_cta_kernel" if sks[0].n_swp > 0 else "sa_level_kernel"
        rec["roofline"] = roofline_alu(fl, t / L, peak, None, kern, src)
        rec["flops_per_chain_step"] = flops_per_chain_step(sks[0], info)
    if cpu:
        rec["cpu_baseline"] = cpu_baseline(sks[0], vols[0], **cpu)
    if e2e:
        h2d = sum(np.asarray(x).nbytes for sk, v in zip(sks, vols)
                  for x in (sk.T, sk.P, sk.cap_fwd, sk.cap_K, sk.swp_start, sk.swp_end, sk.swp_K, v, sk.lo, sk.hi,
                            sk.free))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = lib.Market(sks if len(sks) > 1 else sks[0], vols if len(sks) > 1 else vols[0])
        r2 = m2.anneal(C, L, N, cool, seed, prec=prec, warps_per_block=warps_per_block)
        del m2
        te = time.perf_counter() - t0
        rec["e2e"] = {"value": r2["n_evals"] * n_instr / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(len(sks) * (sks[0].n_param + 2 + L) * 8)}
    return rec, r, gm, sks, vols


PAPER_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "paper_euribor_20111121.txt")
PAPER_MM = os.path.join(os.path.dirname(PAPER_DATA), "paper_mm_20111121.txt")
PAPER_MC = os.path.join(os.path.dirname(PAPER_DATA), "paper_hagan_mc_20111121.txt")
PAPER_SWP = os.path.join(os.path.dirname(PAPER_DATA), "paper_swaptions_20111121.txt")


def paper_data_record(lib, seed, stream):
    """The paper's real-data caplet calibration (Section 4.1.1): the 13 EURIBOR smiles, the paper's
    schedule (16384 chains, N = 10, cooling 0.99, T0 = 10 to 0.01: 688 levels) and hybrid (the search,
    then Nelder-Mead from the best chains), FP32 search and FP64 simplex; device time of each part
    and the mean relative vol error, beside the paper's own figures (another GPU: context)."""
    import torch
    from paper_2408_01470_b300 import synth
    sks, quotes, params, pub = synth.paper_euribor_caplet_smiles(PAPER_DATA)
    gm = lib.Market(sks, quotes)
    sk = sks[0]
    kw = dict(prec="fp32", T0=10.0, lm_top_k=8, lm_max_iter=2000, polish_nm=True, use_graph=True, stream=stream)
    warm = gm.anneal_prepare(sk.n_chains, 2, sk.steps, sk.cooling, seed, **kw)
    warm.launch(stream=stream)
    warm.fetch()
    del warm
    plan = gm.anneal_prepare(sk.n_chains, sk.n_levels, sk.steps, sk.cooling, seed, **kw)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    stream.synchronize()
    t = a.elapsed_time(b) / 1e3
    r = plan.fetch()
    del plan
    rel = []
    for j, q in enumerate(quotes):
        v = gm.model_vols(r["x_best"][j][None, :], "fp64", market=j).cpu().numpy()[0]
        rel += list(np.abs(v - q) / q)
    n_prices = r["n_evals"] * len(sks) * sk.n_cap
    return {"workload": f"paper_euribor_caplets_13x9_{sk.n_chains}ch_x_{sk.n_levels}T_x_{sk.steps}steps",
            "how": "13 smiles, one search each in one call (the paper's cost is separable over the forwards); "
                   "device time of the whole call (CUDA events), of which the Nelder-Mead polish",
            "seconds": t, "sa_seconds": t - float(r["lm_seconds"]), "nm_seconds": float(r["lm_seconds"]),
            "mre": float(np.mean(rel)), "evaluations_per_smile": int(r["n_evals"]),
            "prices_per_s": n_prices / t, "f_best": [float(x) for x in r["f_best"]],
            "paper": {"mre": float(pub["mre"]), "sa_seconds": float(pub["sa_seconds"]),
                      "nm_seconds": float(pub["nm_seconds"]), "total_seconds": float(pub["total_seconds"]),
                      "evaluations": int(pub["evaluations"]), "hardware": pub["hardware"]}}


def mm_paper_record(lib, seed, stream):
    """The paper's Mercurio & Morini caplet calibration (Section 4.2.1): one search over the 27
    parameters [phi_i, sigma, alpha_i] of the 13 EURIBOR smiles (coupled through sigma and the drift of
    Eq. haganForMercurio), the paper's schedule and hybrid; device time and the mean relative vol
    error beside the paper's figures (another GPU: context)."""
    import torch
    from paper_2408_01470_b300 import synth
    sk, q, pr, pv, pub = synth.paper_euribor_mm_market(PAPER_DATA, PAPER_MM)
    gm = lib.Market(sk, q)
    kw = dict(prec="fp32", T0=10.0, lm_top_k=8, lm_max_iter=20000, polish_nm=True, use_graph=True, stream=stream)
    warm = gm.anneal_prepare(sk.n_chains, 2, sk.steps, sk.cooling, seed, **kw)
    warm.launch(stream=stream)
    warm.fetch()
    del warm
    plan = gm.anneal_prepare(sk.n_chains, sk.n_levels, sk.steps, sk.cooling, seed, **kw)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.launch(stream=stream)
    b.record(stream)
    stream.synchronize()
    t = a.elapsed_time(b) / 1e3
    r = plan.fetch()
    del plan
    v = gm.model_vols(r["x_best"][0][None, :], "fp64").cpu().numpy()[0]
    return {"workload": f"paper_euribor_mercurio_morini_27params_{sk.n_chains}ch_x_{sk.n_levels}T_x_{sk.steps}steps",
            "how": "one search over all 27 slots (warp kernels, one slot per lane), then Nelder-Mead (FP64) from "
                   "the 8 best chains; device time of the whole call (CUDA events), of which the polish",
            "seconds": t, "sa_seconds": t - float(r["lm_seconds"]), "nm_seconds": float(r["lm_seconds"]),
            "mre": float(np.mean(np.abs(v - q) / q)), "evaluations": int(r["n_evals"]),
            "prices_per_s": r["n_evals"] * sk.n_cap / t, "f_best": float(r["f_best"][0]),
            "paper": {"mre": float(pub["mre"]), "sa_seconds": float(pub["sa_seconds"]),
                      "nm_seconds": float(pub["nm_seconds"]), "total_seconds": float(pub["total_seconds"]),
                      "evaluations": int(pub["evaluations"]), "hardware": pub["hardware"]}}


def mc_flops_per_path(M, nsteps):
    """Algorithmic floating-point operations of one Monte Carlo path (add, mul = 1; fma = 2; log,
    sqrt, sin, cos, exp, reciprocal = 1), summed over the steps of every interval k with a = M - k
    forwards alive: normals 2a (Box-Muller per pair: log, sqrt, sin, cos and 4 products = 8);
    correlated increments, rows r < 2a of L: r + 1 fma each; per alive forward: V = exp(ln V),
    F^b (log, exp), x (4 + reciprocal), two drift sums over its a - u partners (2 fma each), the F
    step (5) and the ln V step (6)."""
    total = 0.0
    for k in range(M):
        a = M - k
        per = 8 * a + sum(2 * (r + 1) for r in range(2 * a))
        per += sum(1 + 2 + 5 + 4 * (a - u) + 5 + 6 for u in range(a))
        total += nsteps[k] * per
    return total


def mc_record(lib, stream, peaks, cpu=True):
    """The Monte Carlo pricer on the paper's calibrated Hagan SABR/LIBOR model (13 EURIBOR forwards,
    its 117 caplets), at the (paths, dt) of Table tab:haganMCpricer, FP32 as in the paper: device time
    per pricing (CUDA events around the launch on its stream, after one untimed launch), path-steps/s
    and the paper's GPU seconds (one GTX 470: context).  The roofline of the largest configuration
    against the measured FP32 FMA rate, and the oracle's Monte Carlo on the host cores on a sample."""
    import torch
    from paper_2408_01470_b300 import synth
    sk, model, cf, ck, rows = synth.paper_hagan_mc_model(PAPER_DATA, PAPER_MM, PAPER_MC)
    out = {"workload": "paper_hagan_lmm_mc_13fwd_117caplets", "precision": "fp32", "configs": []}
    big = None
    for paths, dt, cpu_s, gpu_s, _ in rows:
        plan = lib.McPlan(sk.T, sk.P, model, cf, ck, n_paths=int(paths), dt=float(dt), seed=20111121, prec="fp32",
                          stream=stream)
        plan.launch(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5 if paths * (1 / dt) < 1e8 else 2
        a.record(stream)
        for _ in range(reps):
            plan.launch(stream)
        b.record(stream)
        stream.synchronize()
        t = a.elapsed_time(b) / 1e3 / reps
        nsteps = [max(1, int(np.ceil((sk.T[k] - (sk.T[k - 1] if k else 0.0)) / dt - 1e-9))) for k in range(sk.n_fwd)]
        steps = sum(nsteps)
        rec = {"paths": int(paths), "dt": float(dt), "seconds": t, "path_steps_per_s": paths * steps / t,
               "n_bad": int(plan.n_bad.item()), "paper_gpu_seconds": float(gpu_s), "paper_cpu_seconds": float(cpu_s),
               "time_steps": steps}
        out["configs"].append(rec)
        big = (rec, nsteps)
        del plan
    rec, nsteps = big
    # the Mercurio & Morini dynamics (one vol process, 1 + a normals a step) at the largest configuration
    skm, mmod = synth.paper_mm_mc_model(PAPER_DATA, PAPER_MM)
    plan = lib.McPlan(skm.T, skm.P, mmod, cf, ck, n_paths=rec["paths"], dt=rec["dt"], seed=20111121, prec="fp32",
                      stream=stream)
    plan.launch(stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(2):
        plan.launch(stream)
    b.record(stream)
    stream.synchronize()
    t = a.elapsed_time(b) / 1e3 / 2
    out["mercurio_morini"] = {"paths": rec["paths"], "dt": rec["dt"], "seconds": t,
                              "path_steps_per_s": rec["paths"] * rec["time_steps"] / t,
                              "n_bad": int(plan.n_bad.item())}
    del plan
    flops = mc_flops_per_path(sk.n_fwd, nsteps) * rec["paths"]
    out["roofline"] = roofline_alu(flops, rec["seconds"], peaks["fp32_tflops"], None, "mc_path_kernel<float>",
                                   "measured FP32 FMA rate (libsabr_peaks.so)")
    out["flops_per_path"] = mc_flops_per_path(sk.n_fwd, nsteps)
    if cpu:
        import oracle
        om = oracle.Market(sk, np.full(sk.n_cap, 0.5))
        threads = os.cpu_count() or 1
        n, dt = 20000, float(rec["dt"])
        t0 = time.perf_counter()
        oracle.mc_price(om, model, cap_fwd=cf, cap_K=ck, n_paths=n, dt=dt, seed=1, n_threads=threads)
        tc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n * rec["time_steps"] / tc, "unit": "path-steps/s", "cores": threads,
                               "kind": "oracle", "sample": f"{n} paths at dt = {dt} (FP64)"}
    return out


def mc_calibration_record(lib, stream, chains=64, levels=20, steps=5, n_paths=10000, dt=0.02, model="hagan"):
    """The paper's swaption calibration of the Hagan model over a Monte Carlo objective (Section 4.1.2):
    the correlation parameters (eta1, lambda1, eta2, lambda2, lambda3) against the 180 swaptions of
    Table tab:smilesTS, the caplet-calibrated alpha_i, sigma_i, phi_ii of Table tab:paramsHaganVolas
    fixed; FP32 paths with common random numbers, every step's proposals of all chains in one launch.
    Reports the search's wall time (against the paper's ~2 hours on two GTX 470s: context), f_s, and
    the mean absolute error of the swaption prices in percent of the notional (the paper's MAE
    6.19e-2; Black prices here with the annuity of the real accruals).  model="mm": the same for the
    Mercurio & Morini model of Section 4.2 (alpha_i, phi_i, sigma of Table tab:paramsMercurioVolas
    fixed; eta1, lambda1 searched; the paper's MAE 5.50e-2)."""
    from paper_2408_01470_b300 import synth
    from scipy.special import ndtr
    sk, sa, sb, sK, vol, pub = synth.paper_swaption_smiles(PAPER_DATA, PAPER_MM, PAPER_SWP)
    mm = model == "mm"
    if mm:
        _, model = synth.paper_mm_mc_model(PAPER_DATA, PAPER_MM)
        mmpub = {r[0]: float(r[1]) for r in synth.read_paper_market(PAPER_MM)["published_swaptions"]}
        pub = {"mae_percent": mmpub["mae_percent"], "calibration_hours": pub["calibration_hours"]}
    else:
        _, model, _, _, _ = synth.paper_hagan_mc_model(PAPER_DATA, PAPER_MM, PAPER_MC)
    lo, hi = np.array([0.0, 0.0, 0.0, 0.0, 0.0]), np.array([1.0, 5.0, 1.0, 5.0, 0.5])
    free = np.array([1, 1, 0, 0, 0]) if mm else np.ones(5)
    kw = dict(swp_start=sa, swp_end=sb, swp_K=sK, n_paths=n_paths, dt=dt, mc_seed=20111121, prec="fp32")
    r = lib.mc_anneal(sk.T, sk.P, model, vol, lo, hi, free, chains, levels, steps, 0.8, 20111121, stream=stream,
                      **kw)
    m_best = dict(model, eta1=r["y_best"][0], lambda1=r["y_best"][1], eta2=r["y_best"][2], lambda2=r["y_best"][3],
                  lambda3=r["y_best"][4])
    mc, _, _ = lib.mc_price(sk.T, sk.P, m_best, (), (), sa, sb, sK, n_paths=n_paths, dt=dt, seed=20111121, prec="fp32",
                            stream=stream)
    tau = np.diff(sk.T)
    A = np.array([sum(tau[k] * sk.P[k + 1] for k in range(a, b)) for a, b in zip(sa, sb)])
    S = (sk.P[sa] - sk.P[sb]) / A
    sd = vol * np.sqrt(sk.T[sa])
    d1 = np.log(S / sK) / sd + 0.5 * sd
    black = A * (S * ndtr(d1) - sK * ndtr(d1 - sd))
    name = "mercurio_morini" if mm else "hagan"
    return {"workload": f"paper_{name}_swaption_calibration_mc_180swaptions_{chains}ch_x_{levels}T_x_{steps}steps_"
                        f"{n_paths}paths_dt{dt}",
            "how": "sabr_lmm_mc_anneal: host-driven annealing (the paper's own split), every step's proposals priced "
                   "in one batched Monte Carlo launch, their constants built by a pool of host threads; wall time of the "
                   "whole search",
            "seconds": r["seconds"], "evaluations": int(r["n_evals"]), "f_best": r["f_best"],
            "y_best": [float(x) for x in r["y_best"]],
            "mae_percent": float(100.0 * np.mean(np.abs(mc - black))),
            "path_steps_per_s": r["n_evals"] * n_paths * int(np.ceil(sk.T[3] / dt)) / r["seconds"],
            "paper": {"mae_percent": float(pub["mae_percent"]), "calibration_hours": float(pub["calibration_hours"]),
                      "y": [model[k] for k in (("eta1", "lambda1") if mm else
                                                ("eta1", "lambda1", "eta2", "lambda2", "lambda3"))],
                      "hardware": "2x NVIDIA GeForce GTX 470 (Fermi)"}}


def lm_schedule_to_target(gm, C, N, cool, seed, target, schedule=(1, 2, 3, 5, 10, 20, 40, 80, 200)):
    """The mixed-precision, adjoint-polished form: the shortest FP32 search of the schedule (the same
    cooling, fewer levels) whose Levenberg-Marquardt polish of its 64 best chains reaches the target
    vol RMSE; device time of that search plus its polish, both measured (each run once untimed)."""
    for Ls in schedule:
        for _ in range(2):
            rp = gm.anneal(C, Ls, N, cool, seed, prec="fp32", lm_top_k=64, lm_max_iter=50, target_rmse=target)
        if rp["rmse_volpt"][0] <= target:
            return {"levels": Ls, "search_s": float(rp["seconds"]), "polish_s": float(rp["lm_seconds"]),
                    "seconds": float(rp["seconds"] + rp["lm_seconds"]), "rmse_volpt": float(rp["rmse_volpt"][0])}
    return None


def run_quality(args):
    """FP32 against FP64: the final vol RMSE of --seeds seeds of a workload's search, and of that
    search's best point after the Levenberg-Marquardt polish (adjoint gradient), on one GPU.  Prints
    one JSON line (per-seed rows on stderr)."""
    import paper_2408_01470_b300 as lib
    import torch
    lib.load()
    gm, sks, vols, C, L, N, cool = workload_markets(lib, args.workload, args.markets)
    C = args.chains or C
    nm = len(sks)
    rows = []
    for k in range(args.seeds):
        seed = 240801470 + 7919 * k
        row = {"seed": seed}
        for prec in ("fp64", "fp32"):
            r = gm.anneal(C, L, N, cool, seed, prec=prec)
            # the adjoint-driven Levenberg-Marquardt polish of each market's best point (FP64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rps = []
            for j in range(nm):
                Xp, fp, rp = gm.lm_polish(r["x_best"][j:j + 1], max_iter=50, market=j)
                rps.append(float(rp.cpu().numpy()[0]))
            tp = time.perf_counter() - t0
            # batches: the mean over the markets of each market's final vol RMSE
            row[prec] = {"rmse_volpt": float(np.mean(r["rmse_volpt"][:nm])), "seconds": float(r["seconds"]),
                         "polished_rmse_volpt": float(np.mean(rps)), "polish_s": tp}
            if nm > 1:
                row[prec]["per_market_rmse_volpt"] = [float(x) for x in r["rmse_volpt"][:nm]]
                row[prec]["per_market_polished_rmse_volpt"] = rps
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"quality": True, "workload": args.workload, "chains": C, "levels": L, "steps": N, "seeds": args.seeds,
           "markets": nm}
    for key in ("rmse_volpt", "polished_rmse_volpt"):
        a64 = np.array([r["fp64"][key] for r in rows])
        a32 = np.array([r["fp32"][key] for r in rows])
        out[key] = {"fp64_mean": float(a64.mean()), "fp32_mean": float(a32.mean()),
                    "fp64_std": float(a64.std(ddof=1)) if len(a64) > 1 else 0.0,
                    "fp32_std": float(a32.std(ddof=1)) if len(a32) > 1 else 0.0,
                    "mean_ratio_fp32_over_fp64": float(a32.mean() / a64.mean()),
                    "fp64": a64.tolist(), "fp32": a32.tolist()}
    out["seconds_fp64_mean"] = float(np.mean([r["fp64"]["seconds"] for r in rows]))
    out["seconds_fp32_mean"] = float(np.mean([r["fp32"]["seconds"] for r in rows]))
    print(json.dumps(out))


def run_workload_line(args):
    """--workload joint|batch without --profile: that workload's full schedule as its own line."""
    import paper_2408_01470_b300 as lib
    import torch
    lib.load()
    peaks = measure_peaks()
    s = torch.cuda.Stream()
    cpu = ({"chains": 64, "levels": 1, "steps": 16} if args.workload == "joint" else
           {"chains": 4096, "levels": 1, "steps": 20} if args.workload == "caplets" else None)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), args.clocks_dir) as clk:
        rec, r, gm, sks, vols = search_record(lib, args.workload, args.prec, 240801470, s, peaks, cpu=None,
                                              e2e=True)
    if args.workload == "batch":
        sub = [synth_market for synth_market in sks[:4]]
        import oracle
        t0 = time.perf_counter()
        n_ev = 0
        for sk, v in zip(sub, vols[:4]):
            rr = oracle.Market(sk, v).anneal(16, 1, 4, sk.cooling, seed=240801470, n_threads=os.cpu_count() or 1)
            n_ev += rr["n_evals"] * sk.n_instr
        dt = time.perf_counter() - t0
        rec["cpu_baseline"] = {"value": n_ev / dt, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"batch markets 0-3, 16 chains x 1 level x 4 steps each ({dt:.1f} s wall)"}
    elif cpu:
        rec["cpu_baseline"] = cpu_baseline(sks[0], vols[0], **cpu)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": rec["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": PREC_DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": rec["workload"], "precision": args.prec,
                       "l2": "inputs resident; warm-up: a 2-level search of the same kernels"},
            **{k: rec[k] for k in rec if k in ("roofline", "e2e", "cpu_baseline")},
            "chain_steps_per_s": rec["chain_steps_per_s"], "ms_per_level": rec["ms_per_level"],
            "rmse_volpt_median": rec["rmse_volpt"], "clocks": clk.summary(), "peaks": peaks,
            "gpu_launches": rec["levels_timed"] * max(1, len(rec["tuning"]["buckets"])) + 2,
            "tuning": rec["tuning"]}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "bf16x3"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64-variant", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-joint-variant", action="store_true")
    ap.add_argument("--no-batch-variant", action="store_true")
    ap.add_argument("--no-paper-data", action="store_true")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--clocks-dir", default="", help="folder for the raw nvidia-smi clock samples (default: temp dir)")
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--profile", action="store_true",
                    help="run the workload's search once (optionally shortened) and exit: the ncu target")
    ap.add_argument("--quality", action="store_true",
                    help="FP32 against FP64 final RMSE over --seeds seeds of --workload (one JSON line)")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--markets", type=int, default=0, help="with --quality --workload batch: the first K markets")
    ap.add_argument("--levels", type=int, default=0, help="with --profile: temperature levels (0 = workload's)")
    ap.add_argument("--chains", type=int, default=0, help="with --profile / --quality: chains per market")
    ap.add_argument("--lm-top-k", type=int, default=0,
                    help="with --profile: Levenberg-Marquardt polish of the k best chains after the search")
    ap.add_argument("--workload", default="", choices=[""] + list(WORKLOADS),
                    help="with --profile / --quality: the search to run; alone: that workload's full line")
    ap.add_argument("--mc-profile", action="store_true",
                    help="three launches of the Monte Carlo pricer (--mc-paths, --mc-dt), for ncu captures")
    ap.add_argument("--mc-calibration", action="store_true",
                    help="the paper's swaption calibration over the Monte Carlo objective alone (--mc-chains, "
                         "--mc-levels, --mc-steps, --mc-paths, --mc-dt)")
    ap.add_argument("--mc-model", default="hagan", choices=["hagan", "mm"],
                    help="with --mc-calibration or --mc-profile: the Hagan or the Mercurio & Morini dynamics")
    ap.add_argument("--mc-chains", type=int, default=64)
    ap.add_argument("--mc-levels", type=int, default=20)
    ap.add_argument("--mc-steps", type=int, default=5)
    ap.add_argument("--mc-paths", type=int, default=100000)
    ap.add_argument("--mc-dt", type=float, default=0.01)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mc_profile:
        return run_mc_profile(args)
    if args.mc_calibration:
        import paper_2408_01470_b300 as lib
        import torch
        lib.load()
        print(json.dumps(mc_calibration_record(lib, torch.cuda.Stream(), args.mc_chains, args.mc_levels,
                                               args.mc_steps, args.mc_paths, args.mc_dt, args.mc_model)))
        return None
    if args.profile:
        args.workload = args.workload or "caplets"
        return run_profile(args)
    if args.quality:
        args.workload = args.workload or "caplets"
        return run_quality(args)
    if args.workload:
        return run_workload_line(args)

    ws, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    from paper_2408_01470_b300 import build as _build
    _build.build()
    import paper_2408_01470_b300 as lib
    from paper_2408_01470_b300 import synth
    lib.load()
    peaks = measure_peaks()

    skel = synth.caplet_term_structure()
    gm, vols = market_from_library(lib, skel)
    C, L, N = skel.n_chains, skel.n_levels, skel.steps
    seed = replica_seed(240801470, rank)
    s = torch.cuda.Stream()
    plan = gm.anneal_prepare(C, L, N, skel.cooling, seed, prec=args.prec, use_graph=True, stream=s,
                             warps_per_block=args.warps_per_block)
    tuning = plan.config()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        plan.launch(stream=s)
        s.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local, args.clocks_dir) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(s):
                flush.zero_()          # L2 flush between timed steps (outside the events)
            evs[k][0].record(s)
            plan.launch(stream=s)
            evs[k][1].record(s)
        s.synchronize()
    torch.cuda.synchronize()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) / 1e3
    res = plan.fetch()
    n_evals = res["n_evals"]
    prices_per_step = n_evals * skel.n_instr
    value, total_s_max = job_rate(total_s, args.steps * prices_per_step, ws)
    ms_per_step = 1e3 * total_s_max / args.steps

    # roofline of the dominant kernel (the per-temperature level kernel, >99% of the step) against
    # the FP32 (FP64) FMA rate measured on this GPU
    level_s = (total_s / args.steps) / L
    info = gm.info()
    flops_launch = C * N * flops_per_chain_step(skel, info)
    peak, src = ((peaks["fp32_tflops"], "measured FP32 FMA rate (libsabr_peaks.so)") if args.prec != "fp64" else
                 (peaks["fp64_tflops"], "measured FP64 FMA rate (libsabr_peaks.so)"))
    roofline = roofline_alu(flops_launch, level_s, peak,
                            LEVEL_TRAFFIC_BYTES_FP32 if args.prec == "fp32" and not args.warps_per_block else None,
                            "sa_level_kernel", src)

    rmse32, sec32 = rmse_trace(gm, res, vols)
    quality = {"f_best": float(res["f_best"][0]), "rmse_volpt": float(res["rmse_volpt"][0]),
               "rmse_volpt_last_level": float(rmse32[-2])}

    # e2e: through the public API from host buffers (H2D of the market, D2H of the results)
    e2e_vals = []
    h2d = sum(a.nbytes for a in (skel.T, skel.P, skel.cap_fwd, skel.cap_K, vols, skel.lo, skel.hi, skel.free))
    d2h = (skel.n_param + 2 + L) * 8
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = lib.Market(skel, vols)
        r2 = m2.anneal(C, L, N, skel.cooling, seed, prec=args.prec, warps_per_block=args.warps_per_block)
        del m2
        e2e_vals.append(r2["n_evals"] * skel.n_instr / (time.perf_counter() - t0))
    e2e_local = statistics.median(e2e_vals) if e2e_vals else float("nan")
    e2e = {"value": ws * e2e_local, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # time to target, measured on the device: each level's best point is recorded with the GPU's
    # global timer when the level ends; its true vol RMSE (FP64 model vols against the quotes) decides
    # when a target is reached.  Targets: 0.05 vol-pt and the final RMSE of the plain FP64 form.
    variants = {}
    ttt = {"how": "device global timer at the end of the first level whose best point's true vol RMSE "
                  "reaches the target (searches); search + polish device time of the shortest schedule "
                  "reaching it (polished form)"}
    if args.prec == "fp32" and not args.no_fp64_variant:
        plan64 = gm.anneal_prepare(C, L, N, skel.cooling, seed, prec="fp64", use_graph=True, stream=s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan64.launch(stream=s)
        b.record(s)
        s.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        r64 = plan64.fetch()
        del plan64
        rmse64, sec64 = rmse_trace(gm, r64, vols)
        R64 = float(r64["rmse_volpt"][0])
        variants["fp64"] = {"value": prices_per_step / t64, "ms_per_step": t64 * 1e3, "rmse_volpt": R64,
                            "f_best": float(r64["f_best"][0]), "chain_steps_per_s": C * L * N / t64,
                            "roofline": roofline_alu(flops_launch, t64 / L, peaks["fp64_tflops"], None,
                                                     "sa_level_kernel", "measured FP64 FMA rate (libsabr_peaks.so)")}
        for name, target in (("target_0p05", TARGET_RMSE_VOLPT), ("target_fp64_final", R64)):
            ttt[name] = {"target_rmse_volpt": target,
                         "fp64": first_hit(rmse64, sec64, target),
                         "fp32": first_hit(rmse32, sec32, target),
                         "fp32_lm_polished": lm_schedule_to_target(gm, C, N, skel.cooling, seed, target)}

    # the joint caplet + swaption market (CTA-per-chain kernels) over its full schedule, and shortened
    # samples of the other precision forms (labelled extrapolated)
    workloads = {}
    if args.prec == "fp32" and not args.no_joint_variant:
        rec, _, _, _, _ = search_record(lib, "joint", "fp32", seed, s, peaks,
                                        cpu=None if args.no_cpu_baseline else {"chains": 64, "levels": 1, "steps": 16})
        workloads["joint_fp32"] = rec
        for jprec in ("fp64", "bf16x3"):
            rec, _, _, _, _ = search_record(lib, "joint", jprec, seed, s, peaks, levels=1, e2e=False)
            workloads["joint_" + jprec] = rec
    # the paper's real-data caplet calibration, full schedule
    if args.prec == "fp32" and not args.no_paper_data:
        workloads["paper_euribor_caplets"] = paper_data_record(lib, seed, s)
    # the paper's Mercurio & Morini calibration (27 coupled parameters), full schedule
    if args.prec == "fp32" and not args.no_paper_data:
        workloads["paper_euribor_mercurio_morini"] = mm_paper_record(lib, seed, s)
    # the Monte Carlo pricer at the configurations of Table tab:haganMCpricer
    if args.prec == "fp32" and not args.no_mc:
        workloads["mc_hagan_caplets"] = mc_record(lib, s, peaks, cpu=not args.no_cpu_baseline)
        workloads["mc_swaption_calibration"] = mc_calibration_record(lib, s)
        workloads["mc_swaption_calibration_mm"] = mc_calibration_record(lib, s, model="mm")
    # the 256-market batch: one level (its full 100-level schedule: bench.py --workload batch)
    if args.prec == "fp32" and not args.no_batch_variant:
        rec, _, _, _, _ = search_record(lib, "batch", "fp32", seed, s, peaks, levels=1, e2e=False)
        workloads["batch_fp32"] = rec

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PREC_DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains": C, "levels": L, "steps_per_level": N,
                       "instruments": skel.n_instr, "n_evals_per_step": n_evals, "precision": args.prec,
                       "l2": "flushed between timed steps (256 MB write)", "graph": True,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps * (L + 2), "clocks": clocks,
            "chain_steps_per_s": ws * C * L * N * args.steps / total_s_max, "peaks": peaks,
            "quality": quality, "time_to_target": ttt, "variants": variants, "workloads": workloads,
            "tuning": tuning}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(skel, vols, levels=1, steps=100)
        cb1 = cpu_baseline(skel, vols, levels=1, steps=4, threads=1)
        cb["single_thread"] = {k: cb1[k] for k in ("value", "chain_steps_per_s", "cores", "sample")}
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
