#!/usr/bin/env python
"""Throughput of the whole hot path: pivoted partial Cholesky of the implicit
Gaussian kernel matrix -> bistochastic normalisation -> top-k eigenpairs.

One step = rpchol_factor + bistoch_normalize + eig_topk on one synthetic
problem (default: 200,000 KS states in R^64, FP64, ARPC b=64, r=1,024, top-64
eigenpairs).  `value` is accepted pivots per second of the whole step,
aggregated over ranks (each rank solves its own independent problem: weak
scaling, no collective on the data path); `ms_per_step` is the end-to-end
top-k eigenpair time.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pivots/s + end-to-end top-k eigpairs time, fp64 vs mixed, at equal trace error"
FP64_PEAK_GFLOPS = 1250.0       # nominal FP64 rate of the GB300 (profiling recipe table)
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="ks200k")
    p.add_argument("--n", type=int, default=None, help="truncate the workload to n points (profiling cases)")
    p.add_argument("--precision", default=None, choices=["fp64", "bf16x3", "both", "lowmem"],
                   help="fp64 path, precision form, or both (default: both for ks workloads, bf16x3 for vsa); "
                        "lowmem: the FP64 low-memory form (pivots and W = F(S,:) only)")
    p.add_argument("--rsweep", default=None,
                   help="comma-separated ranks: time factorisation and eigen stage per r (Section 4.2's scaling)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(v, device, world):
    """Max of a float over ranks (identity for a single process)."""
    if world == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def reduce_sum(v, device, world):
    """Sum of a float over ranks (identity for a single process)."""
    if world == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0])


def replica_seed(name, rank):
    """Data seed of rank `rank`: rank 0 uses the workload's own seed, others their own problem."""
    from datagen import CONFIGS
    return CONFIGS[name]["seed"] + 1000 * rank


def workload(name, rank, n=None):
    from datagen import make_config
    X, eps, cfg = make_config(name, N=n, seed=replica_seed(name, rank))
    return X, eps, cfg


def config_json(cfg, name, world):
    return {"workload": "%s: %d KS-derived points in R^%d, %s input, %s b=%d, r=%d, top-%d" % (
        name, cfg["N"], cfg["d"], cfg["dtype"], cfg["method"], cfg["b"], cfg["r"], cfg["k"]),
        "N": cfg["N"], "d": cfg["d"], "r": cfg["r"], "b": cfg["b"], "k": cfg["k"], "eps_rule": "median sq. distance",
        "seed": 1000 + 2, "l2": "flushed (256 MiB write) before every timed step; F (N*r*8 B) exceeds L2",
        "parallelism": "replicas%d" % world}


# ---------------------------------------------------------------------------
# CPU arm: the oracle as it stands, timed on the host cores
# ---------------------------------------------------------------------------
def oracle_step(X, eps, cfg, seed):
    from oracle.pchol import arpc, greedy_pchol
    from oracle.alg1 import bistochastic_evd
    t0 = time.perf_counter()
    if cfg["method"] == "greedy":
        F = greedy_pchol(X, eps, cfg["r"])[0]
    else:
        F = arpc(X, eps, cfg["r"], cfg["b"], seed)["F"]
    lam, U = bistochastic_evd(F, cfg["k"])
    return time.perf_counter() - t0, F.shape[1]


def cpu_sample(X, eps, cfg, n_sample):
    n = min(n_sample, X.shape[0])
    Xs = np.ascontiguousarray(X[:n], dtype=np.float64)
    dt, rank = oracle_step(Xs, eps, cfg, 1000 + 2)
    scale = X.shape[0] / n                       # every stage is linear in N at fixed r
    full_s = dt * scale
    return dict(value=rank / full_s, unit="pivots/s", cores=os.cpu_count(), kind="oracle",
                sample="first %d of %d points, r=%d, b=%d, k=%d; %.2f s measured, scaled by N/n=%.1f "
                       "(all stages linear in N at fixed r)" % (n, X.shape[0], cfg["r"], cfg["b"], cfg["k"], dt, scale),
                seconds_full_extrapolated=full_s)


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    X, eps, cfg = workload(args.config, 0, args.n)
    n_sample = 12000
    for _ in range(args.warmup):
        cpu_sample(X, eps, cfg, n_sample // 4)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_sample(X, eps, cfg, n_sample))
    secs = float(np.mean([v["seconds_full_extrapolated"] for v in vals]))
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pivots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1000, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(cfg, args.config, 1),
            "cpu_baseline": {"value": value, "unit": "pivots/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": "pivots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


HBM_PEAK_GBS = 6783.5          # MEASURED_PEAKS.json copy bandwidth of the GB300s
BF16_PEAK_TFLOPS = 1924.8       # MEASURED_PEAKS.json cuBLAS bf16 (burst)


# DRAM traffic of one Gram launch from ncu captures of the two Gram kernels
# (dram__bytes_read.sum + dram__bytes_write.sum, bytes, at the captured N and rank).
# Both kernels read F once per (tile pair, split) with L2 absorbing the re-reads, so the
# traffic scales with N * rank; the bench scales the captured figure to its own launch.
GRAM_TRAFFIC = {
    "k_gram": (436.7e6 + 70.7e6, 60000, 803),      # FP64, ks200k points truncated to N = 60,000
    "k_gram32": (8.661e9 + 0.159e9, 300000, 1848),  # FP32, vsa2m points truncated to N = 300,000
}


def gram_traffic(kernel, N, rank):
    b, n0, r0 = GRAM_TRAFFIC[kernel]
    return b * (float(N) * rank) / (float(n0) * r0)


def roofline(path, stages, out, cfg, steps):
    """Roofline entry of the dominant kernel of one path from the traced stage times."""
    N, d = cfg["N"], cfg["d"]
    rank = out["rank"]
    eng_ms = stages["engine"][0] / steps
    gram_ms = stages["gram"][0] / steps
    # per round N (2 d m + 2 k m + m^2); summed, 2 sum k m = rank^2 - sum m^2 cancels the m^2 terms
    eng_flops = N * (2.0 * d * rank + float(rank) ** 2)
    gram_flops = 2.0 * N * rank * (rank + 1)
    if path == "lowmem":
        # factor panel loop per round: K(p, S u T) (2 d (k+m) per row), R = K(p,T) - K(p,S) Z (2 k m),
        # G = R L^-T (m^2); sum k m = (rank^2 - sum m^2) / 2.  Normalisation pass 3: K(p,S) (2 d r),
        # F_p = K(p,S) W^-T (r^2), Grams (2 r (r+1)).
        eng_fl = N * (2.0 * d * (out["sum_k"] + rank) + float(rank) ** 2)
        p3_fl = N * (2.0 * d * rank + float(rank) ** 2 + 2.0 * rank * (rank + 1))
        cand = {"factor panel loop (cuBLAS DGEMM/DTRSM + k_lm_kexp + k_lm_rho)": (eng_ms, eng_fl),
                "normalisation pass 3 (DGEMM + k_lm_kexp + DTRSM + k_gram)": (gram_ms, p3_fl)}
        dom = max(cand, key=lambda n: cand[n][0])
        ms, fl = cand[dom]
        ach = fl / (ms / 1e3) / 1e9
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": ach / FP64_PEAK_GFLOPS, "traffic": None, "ms_per_step": ms,
                "peak_source": "nominal FP64 rate of the recipe table (1.25 TFLOP/s); cuBLAS DGEMM measured 1.04",
                "stages": {n: {"ms": v[0], "gflop": v[1] / 1e9, "frac": v[1] / (v[0] / 1e3) / 1e9 / FP64_PEAK_GFLOPS}
                           for n, v in cand.items()},
                "sum_k": out["sum_k"], "sum_m_sq": out["sum_m_sq"]}
    if path == "fp64":
        cand = {"k_engine": (eng_ms, eng_flops), "k_gram": (gram_ms, gram_flops)}
        dom = max(cand, key=lambda n: cand[n][0])
        ms, fl = cand[dom]
        ach = fl / (ms / 1e3) / 1e9
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": ach / FP64_PEAK_GFLOPS,
                "traffic": gram_traffic("k_gram", N, rank) if dom == "k_gram" else None, "ms_per_step": ms,
                "peak_source": "nominal FP64 rate of the recipe table (1.25 TFLOP/s); cuBLAS DGEMM measured 1.04"}
    # precision form: the engine reads F(:, :k) and X once per round (HBM-bound), writes the m new
    # columns, and reads + writes rho
    eng_bytes = 4.0 * N * (out["sum_k"] + d * out["engine_rounds"] + rank) + 16.0 * N * out["engine_rounds"]
    cand = {"k_engine_tc": eng_ms, "k_gram32": gram_ms}
    dom = max(cand, key=lambda n: cand[n])
    if dom == "k_engine_tc":
        ach = eng_bytes / (eng_ms / 1e3) / 1e9
        return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": ach / HBM_PEAK_GBS, "traffic": None, "ms_per_step": eng_ms,
                "algorithmic_bytes_per_step": eng_bytes,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    ach = gram_flops / (gram_ms / 1e3) / 1e12
    return {"kernel": dom, "bound": "alu", "achieved": ach * 1e3, "peak": 70000.0, "unit": "GFLOP/s",
            "frac": ach * 1e3 / 70000.0, "traffic": gram_traffic("k_gram32", N, rank), "ms_per_step": gram_ms,
            "peak_source": "FP32 FFMA, cuBLAS SGEMM measured 69.8 TFLOP/s on this pool"}


def lowmem_launches(N, out, steps):
    """Kernels of this library that one low-memory step launches (cuBLAS calls not counted)."""
    rank, rounds, er = out["rank"], out["rounds"], out["engine_rounds"]
    P = min((N + 63) // 64 * 64, max(64, ((1 << 24) // max(rank, 1)) // 64 * 64))
    npan = (N + P - 1) // P
    factor = 1 + 5 * rounds + er * (1 + 2 * npan) + 1
    normalize = 3 + npan * (3 + 1 + 1 + 2)
    eig = 2 + npan + 9
    return int(steps * (factor + normalize + eig))


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2510_26574_gb300.build import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    import paper_2510_26574_gb300 as kevd

    X, eps, cfg = workload(args.config, rank, args.n)
    N, d, r, b, k = cfg["N"], cfg["d"], cfg["r"], cfg["b"], cfg["k"]
    seed = 1000 + 2 + rank
    mode = cfg["method"]
    prec = args.precision or ("both" if cfg["dtype"] == "f64" else "bf16x3")
    paths = ["fp64", "bf16x3"] if prec == "both" else [prec]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def make_step(path):
        tau = 1e-6 if path == "bf16x3" else 1e-13
        if path == "lowmem":
            def step_lm(Xd):
                out = kevd.rpchol_factor_lowmem(Xd, eps, r, mode=mode, b=b, seed=seed)
                dt, qt, A, C = kevd.bistoch_normalize_lowmem(Xd, eps, out["pivots"], out["W"], out["rank"])
                ev, U, kept = kevd.eig_topk_lowmem(Xd, eps, out["pivots"], out["W"], out["rank"], dt, A, C, k, tau=tau)
                return out, ev, U
            return step_lm

        def step(Xd):
            out = kevd.rpchol_factor(Xd, eps, r, mode=mode, b=b, seed=seed)
            dt, qt, A, C = kevd.bistoch_normalize(out["F"], out["rank"])
            ev, U, kept = kevd.eig_topk(out["F"], out["rank"], dt, A, C, k, tau=tau)
            return out, ev, U
        return step

    results = {}
    for path in paths:
        xdt = np.float32 if path == "bf16x3" else np.float64
        Xp = np.ascontiguousarray(X, dtype=xdt)
        Xg = torch.from_numpy(Xp).to(dev)
        step = make_step(path)
        for _ in range(max(args.warmup, 3)):
            out, ev, U = step(Xg)
        kevd.trace_reset()
        kevd.trace_enable(True)
        clocks = Clocks(local)
        clocks.start()
        times = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out, ev, U = step(Xg)
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
        clk = clocks.stop()
        kevd.trace_enable(False)
        stages = kevd.trace_read()
        ms = reduce_max(float(np.mean(times)), dev, world)
        piv = reduce_sum(float(out["rank"]), dev, world)
        res = {"value": piv / (ms / 1e3), "ms_per_step": ms, "accepted_rank": out["rank"], "rounds": out["rounds"],
               "trace_err_rel": out["trace_err"] / N, "clocks": clk, "top_eigs": [float(x) for x in ev[:4].cpu()],
               "stage_ms_per_step": {s_: v[0] / args.steps for s_, v in stages.items()},
               "roofline": roofline(path, stages, out, cfg, args.steps),
               "gpu_launches": int(args.steps * ((1 + 5 * (r // b if mode == "arpc" else r) + 2) + 9 + 9
                                                 + (r // b if path == "bf16x3" else 0)))}
        if path == "lowmem":
            res["gpu_launches"] = lowmem_launches(N, out, args.steps)
            res["workspace_bytes"] = {
                "factor": kevd.workspace_bytes(kevd.kevd.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1,
                                               kevd.kevd.make_opts(mode, b, seed)),
                "stored_F_factor_plus_F": kevd.workspace_bytes(kevd.kevd.KEVD_WS_FACTOR, N, d, r, 1,
                                                               kevd.kevd.make_opts(mode, b, seed)) + 8 * N * r}
        # end to end through the public API with host buffers
        if not args.no_e2e:
            Xh = torch.from_numpy(Xp).pin_memory()
            et = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                barrier()
                t0 = time.perf_counter()
                Xd = Xh.to(dev, non_blocking=True)
                o2, ev2, U2 = step(Xd)
                evh = ev2.cpu()
                Uh = U2.cpu()
                barrier()
                et.append(time.perf_counter() - t0)
            es = reduce_max(float(np.mean(et)), dev, world)
            res["e2e"] = {"value": piv / es, "unit": "pivots/s", "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size()),
                          "d2h_bytes_per_step": int(evh.numel() * 8 + Uh.numel() * 8), "seconds_per_step": es}
            del Xh
        results[path] = res
        del Xg, out, U
        torch.cuda.empty_cache()

    if world > 1 and rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return 0

    main_path = paths[0]
    mres = results[main_path]
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = cpu_sample(X, eps, cfg, 12000 if N <= 300000 else 6000)
        cpu.pop("seconds_full_extrapolated", None)
    line = {"metric": METRIC, "value": mres["value"], "unit": "pivots/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": mres["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3" if main_path == "bf16x3" else "f64",
            "data": "synthetic (seeded KS, ETDRK4, 1,000 t.u. spin-up)",
            "config": config_json(cfg, args.config, world), "clocks": mres["clocks"], "e2e": mres.get("e2e"),
            "gpu_launches": mres["gpu_launches"], "roofline": mres["roofline"], "cpu_baseline": cpu,
            "accepted_rank": mres["accepted_rank"], "rounds": mres["rounds"], "trace_err_rel": mres["trace_err_rel"],
            "top_eigs": mres["top_eigs"], "stage_ms_per_step": mres["stage_ms_per_step"]}
    if main_path == "lowmem":
        line["form"] = "low-memory (pivots and W = F(S,:) only; F rebuilt in row panels)"
        line["workspace_bytes"] = mres["workspace_bytes"]
    if args.config == "paper32k":
        line["paper_context"] = {"trace_err_rel": 0.0891, "hardware": "1x A100 40 GiB, FP32",
                                 "note": "Section 4.1: NM = 32,768, J = 64, eps = 32, r = 4096, b = 64"}
    if len(paths) == 2:
        mx = results["bf16x3"]
        line["mixed"] = {k_: mx[k_] for k_ in ("value", "ms_per_step", "accepted_rank", "trace_err_rel", "top_eigs",
                                               "roofline", "stage_ms_per_step", "e2e", "clocks")}
        line["mixed"]["dtype"] = "f32 storage, bf16x3 tensor-core products, fp64 rho/H/L/degrees/eigensolve"
        line["mixed"]["speedup_vs_fp64"] = results["fp64"]["ms_per_step"] / mx["ms_per_step"]
        line["mixed"]["trace_err_ratio_vs_fp64"] = mx["trace_err_rel"] / results["fp64"]["trace_err_rel"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """64 independent Gaussian-mixture problems (uneven N, d, eps, r), batched FP64 ARPC
    behind a CUDA graph with autotuned b, then normalisation and top-16 eigenpairs each."""
    import torch
    from datagen import batched_problems
    rank_, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as kevd
    from paper_2510_26574_gb300.autotune import tune
    raw = batched_problems(64, seed=4 + 1000 * rank_)
    probs = [dict(X=torch.from_numpy(p["X"]).to(dev), eps=p["eps"], r=p["r"], b=p["b"], seed=p["seed"], k=p["k"])
             for p in raw]
    t0 = time.perf_counter()
    bs = tune(probs)
    tune_s = time.perf_counter() - t0
    for p, b in zip(probs, bs):
        p["b"] = b
    batch = kevd.Batch(probs, use_graph=True)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    # normalisation and top-k of the 64 problems: small, latency-bound r x r work, so
    # WORKERS host threads drive it on their own streams (the library keeps one
    # cuSOLVER/cuBLAS handle per thread); the main stream waits for all of them
    from concurrent.futures import ThreadPoolExecutor
    workers = 8
    wstreams = [torch.cuda.Stream(dev) for _ in range(workers)]
    pool = ThreadPoolExecutor(workers)

    def finish(wk, outs):
        torch.cuda.set_device(dev)
        res = {}
        with torch.cuda.stream(wstreams[wk]):
            for i in range(wk, len(probs), workers):
                o = outs[i]
                dt, qt, A, C = kevd.bistoch_normalize(o["F"], o["rank"])
                ev, U, kept = kevd.eig_topk(o["F"], o["rank"], dt, A, C, probs[i]["k"])
                res[i] = ev
        return res

    fac_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step():
        fac_ev[0].record(stream)
        outs = batch.run()
        fac_ev[1].record(stream)
        for ws in wstreams:
            ws.wait_event(fac_ev[1])
        evs = {}
        for f in [pool.submit(finish, wk, outs) for wk in range(workers)]:
            evs.update(f.result())
        for ws in wstreams:
            stream.wait_stream(ws)
        return outs, [evs[i] for i in range(len(probs))]

    for _ in range(max(args.warmup, 3)):
        outs, evs = step()
    clocks = Clocks(local)
    clocks.start()
    times, fac_times = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs, evs = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
        fac_times.append(fac_ev[0].elapsed_time(fac_ev[1]))
    clk = clocks.stop()
    pool.shutdown()
    ms = float(np.mean(times))
    factor_ms = float(np.mean(fac_times))
    # stage breakdown from one extra traced step with the per-problem stages run in sequence
    kevd.trace_reset()
    kevd.trace_enable(True)
    batch.run()
    for p, o in zip(probs, outs):
        dt, qt, A, C = kevd.bistoch_normalize(o["F"], o["rank"])
        kevd.eig_topk(o["F"], o["rank"], dt, A, C, p["k"])
    torch.cuda.synchronize(dev)
    kevd.trace_enable(False)
    stages = kevd.trace_read()
    pivots = sum(o["rank"] for o in outs)
    flops = sum(p["X"].shape[0] * (2.0 * p["X"].shape[1] * o["rank"] + float(o["rank"]) ** 2)
                for p, o in zip(probs, outs))
    # the same factorisations as independent single-problem calls (plain FP64 path)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for p in probs:
        kevd.rpchol_factor(p["X"], p["eps"], p["r"], mode="arpc", b=p["b"], seed=p["seed"])
    torch.cuda.synchronize(dev)
    single_ms = (time.perf_counter() - t1) * 1e3
    ach = flops / (factor_ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": pivots / (ms / 1e3), "unit": "pivots/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (64 seeded Gaussian mixtures around KS states)",
            "config": {"workload": "batched: 64 problems, N~U[5k,100k], d in {32,64,128}, eps in {0.25..2}x median, "
                                   "r~U[128,512], top-16, autotuned b, CUDA graph",
                       "n_problems": 64, "total_points": int(sum(p["X"].shape[0] for p in probs)),
                       "b_choices": sorted(set(bs)), "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas%d" % world},
            "clocks": clk, "e2e": None, "gpu_launches": None,
            "roofline": {"kernel": "batched factorisation (graph: propose..engine x rounds)", "bound": "alu",
                         "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": ach / FP64_PEAK_GFLOPS,
                         "traffic": None, "ms_per_step": factor_ms},
            "batched_factor_ms": factor_ms, "single_calls_factor_ms": single_ms,
            "batching_speedup": single_ms / factor_ms, "autotune_s": tune_s,
            "finish_streams": workers,
            "stage_ms_sequential_step": {s_: v[0] for s_, v in stages.items()}}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def run_rsweep(args):
    """Wall-clock of the factorisation and of the eigen stage (normalisation + top-k) as r grows
    on one workload (the paper's scaling experiment, Fig. 5, reports both as quadratic in r)."""
    import torch
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as kevd
    X, eps, cfg = workload(args.config, 0, args.n)
    prec = args.precision or ("fp64" if cfg["dtype"] == "f64" else "bf16x3")
    Xg = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64 if prec == "fp64" else np.float32)).cuda()
    rows = []
    for r in [int(x) for x in args.rsweep.split(",")]:
        b = min(cfg["b"], r)
        k = min(cfg["k"], r // 2)
        for _ in range(max(args.warmup, 1)):           # warm both stages (solver kernels load lazily)
            out = kevd.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=1000)
            dt, qt, A, C = kevd.bistoch_normalize(out["F"], out["rank"])
            kevd.eig_topk(out["F"], out["rank"], dt, A, C, min(k, out["rank"]), tau=1e-13 if prec == "fp64" else 1e-6)
        fac, eig = [], []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = kevd.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=1000)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            dt, qt, A, C = kevd.bistoch_normalize(out["F"], out["rank"])
            ev, U, kept = kevd.eig_topk(out["F"], out["rank"], dt, A, C, min(k, out["rank"]),
                                        tau=1e-13 if prec == "fp64" else 1e-6)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fac.append(t1 - t0)
            eig.append(t2 - t1)
        rows.append({"r": r, "rank": out["rank"], "factor_s": float(np.median(fac)), "eig_s": float(np.median(eig)),
                     "trace_err_rel": out["trace_err"] / cfg["N"]})
        del out
        torch.cuda.empty_cache()
    print(json.dumps({"rsweep": rows, "config": config_json(cfg, args.config, 1), "precision": prec}), flush=True)
    return 0


def main():
    args = parse()
    if args.rsweep:
        return run_rsweep(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batched":
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
