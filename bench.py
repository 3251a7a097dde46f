"""Benchmark: instrument prices per second inside the simulated-annealing objective.

One step = one complete annealing search of the Rebonato SABR/LIBOR caplet term structure
(20 semi-annual forwards x 15 strikes = 300 caplets; 4096 chains x 200 temperatures x 100
Metropolis steps, cooling 0.95): proposal (S1), per-forward SABR parameters by quadrature (S2),
caplet pricing (S4), objective sum (S7), Metropolis and the per-temperature best-chain
reduction (S8).  Inputs are synthetic (seeded), resident in HBM before the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64] [--impl reference]

Besides the headline value the line carries `variants` (the FP64 plain form of the same search;
the joint caplet + swaption market in FP32, FP64 and with the BF16-split tensor-core Grams; one
level of the 256-market batch) and `time_to_target` (0.05 vol-pt RMS: FP64 plain, FP32, and the
FP32 search with the Levenberg-Marquardt polish).

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
# capture of the kernel as it is built now (dram__bytes_read.sum 513,280 B, dram__bytes_write.sum 0 B,
# second level of a 3-level search); the market and chain state stay in L2 across launches
LEVEL_TRAFFIC_BYTES_FP32 = 513_280
TARGET_RMSE_VOLPT = 0.05


def flops_per_chain_step(skel) -> float:
    """Algorithmic floating-point operations of one objective evaluation plus one Metropolis step.

    Counted from the arithmetic as written (add, mul = 1; fma = 2; div, sqrt, exp, log1p, erfc = 1):
      S2, per (panel, node): g and h (5 each), eight inner nodes (8 each), three weighted sums (5)
          = 79; per forward: 4 per panel + 6;
      S4, per caplet: SABR with z/x(z) 35, Black 15, weighted residual 3 = 53;
      S1 + S8: 6 per free slot + 4.
    """
    NP = int(round(max(skel.T[i] for i in set(skel.cap_fwd.tolist())) / skel.panel))
    if skel.model == 1:
        s2 = NP * 8 * 79 + sum(4 * int(round(skel.T[i] / skel.panel)) + 6 for i in set(skel.cap_fwd.tolist()))
    else:
        s2 = 0
    s4 = 53 * skel.n_cap
    s1 = 6 * int(skel.free.sum()) + 4
    return float(s2 + s4 + s1)


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


def workload_markets(lib, name):
    """(Market, skeletons, vols list, chains, levels, steps, cooling) of a named workload."""
    from paper_2408_01470_b300 import synth
    if name == "caplets":
        sks = [synth.caplet_term_structure()]
    elif name == "joint":
        sks = [synth.joint_caplet_swaption()]
    else:
        sks = [synth.batch_market(j) for j in range(256)]
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
            "sample": f"{chains} chains x {levels} temperature level x {steps} steps of the same market "
                      f"({r['n_evals']} objective evaluations, {dt:.1f} s wall)"}


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
    times, vals = [], []
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
            "cpu_baseline": {**base, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """One search of the bench workload (levels shortened with --levels), for ncu captures."""
    import torch
    import paper_2408_01470_b300 as lib
    from paper_2408_01470_b300 import synth
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
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--clocks-dir", default="", help="folder for the raw nvidia-smi clock samples (default: temp dir)")
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--profile", action="store_true",
                    help="run the workload's search once (optionally shortened) and exit: the ncu target")
    ap.add_argument("--levels", type=int, default=0, help="with --profile: temperature levels (0 = workload's)")
    ap.add_argument("--chains", type=int, default=0, help="with --profile: chains per market (0 = workload's)")
    ap.add_argument("--lm-top-k", type=int, default=0,
                    help="with --profile: Levenberg-Marquardt polish of the k best chains after the search")
    ap.add_argument("--workload", default="caplets", choices=list(WORKLOADS),
                    help="with --profile: the search to run (the timed line is always the caplet workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    ws, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    from paper_2408_01470_b300 import build as _build
    _build.build()
    import paper_2408_01470_b300 as lib
    from paper_2408_01470_b300 import synth
    lib.load()

    skel = synth.caplet_term_structure()
    gm, vols = market_from_library(lib, skel)
    C, L, N = skel.n_chains, skel.n_levels, skel.steps
    seed = replica_seed(240801470, rank)
    s = torch.cuda.Stream()
    plan = gm.anneal_prepare(C, L, N, skel.cooling, seed, prec=args.prec, use_graph=True, stream=s,
                             warps_per_block=args.warps_per_block)
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

    # roofline of the dominant kernel (the per-temperature level kernel, >99% of the step)
    level_s = (total_s / args.steps) / L
    flops_launch = C * N * flops_per_chain_step(skel)
    peak = FP32_PEAK_TFLOPS if args.prec == "fp32" else FP64_PEAK_TFLOPS
    achieved = flops_launch / level_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": LEVEL_TRAFFIC_BYTES_FP32 if args.prec == "fp32" and not args.warps_per_block else None,
                "kernel": "sa_level_kernel", "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2032 MHz"
                if args.prec == "fp32" else "nominal B300 FP64 1.25 TFLOP/s"}

    quality = {"f_best": float(res["f_best"][0]), "rmse_volpt": float(res["rmse_volpt"][0])}
    trace_rmse = 100.0 * np.sqrt(np.maximum(res["trace_f"][0], 0.0) / skel.n_instr)
    hit = np.nonzero(trace_rmse <= TARGET_RMSE_VOLPT)[0]
    ttt = {"target_rmse_volpt": TARGET_RMSE_VOLPT,
           args.prec + "_s": (float((hit[0] + 1) * level_s) if hit.size else None)}

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

    variants = {}
    if not args.no_fp64_variant and args.prec == "fp32":
        plan64 = gm.anneal_prepare(C, L, N, skel.cooling, seed, prec="fp64", use_graph=True, stream=s)
        plan64.launch(stream=s)
        s.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan64.launch(stream=s)
        b.record(s)
        s.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        r64 = plan64.fetch()
        tr64 = 100.0 * np.sqrt(np.maximum(r64["trace_f"][0], 0.0) / skel.n_instr)
        hit64 = np.nonzero(tr64 <= TARGET_RMSE_VOLPT)[0]
        ttt["fp64_s"] = float((hit64[0] + 1) * t64 / L) if hit64.size else None
        ach64 = flops_launch / (t64 / L) / 1e12
        variants["fp64"] = {"value": prices_per_step / t64, "ms_per_step": t64 * 1e3,
                            "rmse_volpt": float(r64["rmse_volpt"][0]), "f_best": float(r64["f_best"][0]),
                            "roofline": {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                                         "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS}}
        del plan64

    # the mixed-precision, adjoint-polished form: a shortened FP32 search (the same cooling, fewer
    # levels), then the Levenberg-Marquardt polish (adjoint gradient) of its 64 best chains; the
    # shortest schedule that reaches the target
    if args.prec == "fp32":
        pol = None
        for Ls in (1, 2, 3, 5, 10, 20, 40, 80):
            for _ in range(2):   # the first call of a schedule is its warm-up
                rp = gm.anneal(C, Ls, N, skel.cooling, seed, prec="fp32", lm_top_k=64, lm_max_iter=50,
                               target_rmse=TARGET_RMSE_VOLPT)
            if rp["rmse_volpt"][0] <= TARGET_RMSE_VOLPT:
                pol = {"levels": Ls, "search_s": float(rp["seconds"]), "polish_s": float(rp["lm_seconds"]),
                       "rmse_volpt": float(rp["rmse_volpt"][0])}
                break
        ttt["fp32_lm_polished_s"] = pol["search_s"] + pol["polish_s"] if pol else None
        ttt["fp32_lm_polished"] = pol

    # the joint caplet + swaption market (CTA-per-chain kernels), a shortened search for its rate in
    # each precision form: FP32 (5 levels), FP64 plain and FP32 with the BF16-split tensor-core
    # Grams (1 level each)
    if args.prec == "fp32" and not args.no_joint_variant:
        jm, jsks, _, jC, _, jN, jcool = workload_markets(lib, "joint")
        for jprec, jL in (("fp32", 5), ("fp64", 1), ("bf16x3", 1)):
            jplan = jm.anneal_prepare(jC, jL, jN, jcool, seed, prec=jprec, use_graph=True, stream=s)
            jplan.launch(stream=s)
            s.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            jplan.launch(stream=s)
            b.record(s)
            s.synchronize()
            tj = a.elapsed_time(b) / 1e3
            rj = jplan.fetch()
            variants["joint_" + jprec] = {"workload": WORKLOADS["joint"], "levels_timed": jL,
                                          "value": rj["n_evals"] * jsks[0].n_instr / tj, "unit": UNIT,
                                          "ms_per_level": tj * 1e3 / jL,
                                          "rmse_volpt": float(rj["rmse_volpt"][0])}
            del jplan
        del jm

    # the 256-market batch (one persistent launch per shared-memory bucket and level), one level
    if args.prec == "fp32" and not args.no_batch_variant:
        bm, bsks, _, bC, _, bN, bcool = workload_markets(lib, "batch")
        bL = 1
        bplan = bm.anneal_prepare(bC, bL, bN, bcool, seed, prec="fp32", use_graph=True, stream=s)
        bplan.launch(stream=s)
        s.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        bplan.launch(stream=s)
        b.record(s)
        s.synchronize()
        tb = a.elapsed_time(b) / 1e3
        rb = bplan.fetch()
        variants["batch_fp32"] = {"workload": WORKLOADS["batch"], "levels_timed": bL,
                                  "value": rb["n_evals"] * sum(sk.n_instr for sk in bsks) / tb, "unit": UNIT,
                                  "ms_per_level": tb * 1e3 / bL}
        del bplan, bm

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains": C, "levels": L, "steps_per_level": N,
                       "instruments": skel.n_instr, "n_evals_per_step": n_evals, "precision": args.prec,
                       "l2": "flushed between timed steps (256 MB write)", "graph": True,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps * (L + 2), "clocks": clocks,
            "quality": quality, "time_to_target": ttt, "variants": variants}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(skel, vols, levels=1, steps=100)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
