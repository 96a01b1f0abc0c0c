#!/usr/bin/env python3
"""Benchmark of the fast ordering ICA hot path on GB300: time to all components and
algorithmic TFLOP/s of the BF16 fused tcgen05 path with the learned restart pruner (the
headline), beside the same path without the pruner and the plain FP32 matrix form (cuBLAS
SGEMM, Z in device memory) on the same GPU, and the FP64 CPU oracle as a baseline.

One step = one whole fit of one synthetic data set: whitening (ica_whiten) plus every
component (ica_order_fit), inputs resident in device memory when the timed region starts.
Default workload: EEG-like mixture, N = 256 channels, T = 1,000,000 samples, M = 8192
restarts, all 256 components, at most 30 fixed-point iterations, tolerance 1e-6 (--config
eeg128: N = 128, T = 500,000, M = 4096; eeg64: N = 64, T = 200,000, M = 1024).

Algorithmic FLOPs: 4 n M_act T per fused update of M_act active restarts on n reduced
dimensions (two products of n x T per restart; the rows actually updated, counted on the
device), 2 n M T per kurtosis pass, summed over the fit. `nominal_tflops` uses the fixed
4 N M T per iteration instead.

The pruner (not part of the paper) combines a 13-64-64-1 network with a keep floor, a
redundancy rule and a Gaussian-subspace rule. The network is trained untimed, by the library's
own kernels, on restart trajectories the method records on workloads shaped like the small
N = 8 mixture, the EEG-like N = 64 and N = 128 cases, and N = 256 at reduced T and M (other
seeds than the timed data). Beside the headline the bench reports the unpruned fit (the
pruner's judge), the network's trained threshold, the FP8 form (stage iterations 1..3 on E4M3
operands), e2e through the public API with host buffers, and the plain FP32 matrix form.

Multi-GPU (torchrun): every rank fits its own data set (weak scaling, replicas: the fit has
no exchange step); value = all ranks' FLOPs / the slowest rank's time.

--impl reference: the FP64 CPU oracle (Algorithm 2 in numpy) timed on the host cores on a
bounded sample of the same workload (whitening + first component with a subset of the
restarts), same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-all-components & TFLOP/s, BF16 fused+pruned vs plain FP32, same GB300"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# restarts of the bounded oracle sample (whitening + component 1 at full T) per workload
ORACLE_RESTARTS = {"small": 64, "eeg64": 256, "eeg128": 64, "eeg256": 16, "eeg128_small": 64, "eeg256_small": 32}
# ncu DRAM bytes (read + write) of one persistent stage launch divided by its iterations x its
# X~ bytes (n_pad T 2, one pass per iteration), per workload, from the captures of the current
# kernel (profiles/stage_tc_kernel_eeg256_small.md: 19.32 GB / (30 x 204.8 MB) with the equal
# work shares, X~ larger than L2; profiles/stage_tc_kernel_eeg128_small.md: 3.78 GB /
# (30 x 102.4 MB), X~ within L2); absent where no capture of the current kernel exists
STAGE_TRAFFIC_RATIO = {"eeg256": 3.145, "eeg256_small": 3.145, "eeg128": 1.231, "eeg128_small": 1.231}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["small", "eeg64", "eeg128", "eeg256", "eeg128_small", "eeg256_small", "batch"],
                    default="eeg256",
                    help="workload (eeg128_small / eeg256_small: N = 128 / 256, T = 400,000, M = 4096 / 8192, for "
                         "ncu captures that must stay a few GB)")
    ap.add_argument("--components", type=int, default=0, metavar="K",
                    help="fit only the first K components (ncu captures of the widest stage launches)")
    ap.add_argument("--workers", type=int, default=8, help="concurrent fits of --config batch")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP32 comparator")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-prune", action="store_true", help="headline without the learned pruner")
    ap.add_argument("--precision", choices=["bf16", "fp8"], default="bf16",
                    help="precision of the headline fit (fp8: ICA_FP8, iterations 1..3 of each stage on E4M3 operands)")
    ap.add_argument("--fp8-iters", type=int, default=-1, metavar="K",
                    help="FP8 form: stage iterations 1..K on E4M3 operands (default: the library's)")
    ap.add_argument("--stage-streamk", type=int, default=-1, choices=[-1, 0, 1],
                    help="persistent stage's equal work shares: 1 on, 0 off (default: the library's)")
    ap.add_argument("--stage-lo-from", type=int, default=-1, metavar="T",
                    help="first stage iteration that adds the restart rows' low BF16 term (default: the library's)")
    ap.add_argument("--side-steps", type=int, default=1, help="timed steps of the unpruned, FP8 and e2e legs")
    ap.add_argument("--prune-recall", type=float, default=0.999,
                    help="recall of the training positives that sets the pruner's keep threshold")
    ap.add_argument("--prune-train", choices=["n256", "c1c3"], default="n256",
                    help="pruner training shapes: N = 8/64/128 plus a reduced N = 256 case, or N = 8/64/128 only")
    ap.add_argument("--prune-tau", type=float, default=0.0,
                    help="keep threshold of the headline's pruner network (0: the network keeps every restart, the "
                         "keep floor and the redundancy rule prune; <0: the trained threshold)")
    ap.add_argument("--no-network-leg", action="store_true",
                    help="skip the leg that times and judges the pruner with the network's trained threshold")
    ap.add_argument("--no-fp8-leg", action="store_true",
                    help="skip the leg that times and judges the FP8 form (iterations 1..3 of each stage on E4M3 "
                         "operands) with the headline's pruner")
    ap.add_argument("--prune-cos", type=float, default=0.99,
                    help="|cos| at iteration 5 above which a restart led by another one is redundant (0: off)")
    ap.add_argument("--plain-components", type=int, default=-1, metavar="K",
                    help="plain FP32 comparison on the first K components (0: the whole fit; default: 8 for "
                         "eeg256, whose whole plain fit takes about ten minutes, else 0)")
    ap.add_argument("--nvtx", action="store_true",
                    help="wrap each timed step of the headline in an NVTX range 'timed_step' (ncu launch lists)")
    ap.add_argument("--certify", type=int, default=0, metavar="K",
                    help="FP64 certification (oracle.certify_picks) of the first K components of one extra fit")
    ap.add_argument("--kernel-step", type=int, default=0, metavar="T",
                    help="instead of fits: time ica_fp_step (BF16) at the workload's N and M on T random "
                         "samples (used for ncu captures of the fused kernel on data larger than L2)")
    return ap.parse_args()


def workload(name: str, seed: int):
    import synth

    if name.endswith("_small"):  # the N = 256 / 128 cases at T = 400,000 (restarts as at full size)
        N = int(name[3:6])
        return synth.eeg_like(N, 400_000, 8192 if N == 256 else 4096, seed=seed)
    return {"small": synth.small_mixture, "eeg64": synth.eeg64, "eeg128": synth.eeg128, "eeg256": synth.eeg256}[name](seed)


def workload_desc(w) -> str:
    return (f"{w.name}: EEG-like mixture (3/4 non-Gaussian: Laplace, Student-t 4/6/10, uniform, binary, "
            f"sinusoid; 1/4 Gaussian; sigma 0.05 noise), N={w.N}, T={w.T}, M={w.M}, "
            f"{w.n_components} components, iters<={w.iters}, tol={w.tol}") if w.name.startswith("eeg") else \
        f"{w.name}: N={w.N}, T={w.T}, M={w.M}, {w.n_components} components, iters<={w.iters}, tol={w.tol}"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(w, n_restarts: int = 64):
    """Bounded oracle run: FP64 whitening + component 1 of Algorithm 2 on a subset of restarts.
    Returns (seconds, algorithmic FLOPs, description)."""
    import numpy as np

    import oracle
    import synth

    B0 = synth.restart_inits(n_restarts, w.N, 1, w.seed + 1000)
    t0 = time.perf_counter()
    Xw, V, mean = oracle.whiten(w.X)
    res = oracle.fast_ordering_ica(Xw, n_restarts, w.iters, w.tol, B0, n_components=1, record=True)
    dt = time.perf_counter() - t0
    n = w.N
    active = sum(len(a) for a, _ in res.traces[0].step_norms)
    flops = 4.0 * n * active * w.T + 2.0 * n * n_restarts * w.T
    return dt, flops, (f"FP64 whitening + component 1 of {w.n_components} with restarts 0..{n_restarts - 1} of "
                       f"{w.M}, full T={w.T} (Algorithm 2, numpy)")


def blas_threads() -> int:
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    try:
        from threadpoolctl import threadpool_info

        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.config, args.seed)
    R = ORACLE_RESTARTS.get(args.config, 64)
    for _ in range(args.warmup):
        oracle_sample(w, R)
    times, flops = [], 0.0
    desc = ""
    for _ in range(args.steps):
        dt, fl, desc = oracle_sample(w, R)
        times.append(dt)
        flops += fl
    tflops = flops / sum(times) / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators, synth/)",
            "config": {"workload": workload_desc(w), "sample": desc},
            "cpu_baseline": {"value": tflops, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate_over_ranks(total_ms, flops, nominal, world, device):
    """Whole-job figures of N replicas (one per rank, no exchange step): the time of the slowest
    rank, FLOPs summed over the ranks. Needs an initialised process group when world > 1."""
    if world <= 1:
        return total_ms, flops, nominal
    import torch
    import torch.distributed as dist

    t = torch.tensor([total_ms, flops, nominal], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1]), float(t[2])


_T0 = time.perf_counter()


def log(msg: str):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def train_pruner(ctx, dev, seed: int, recall: float = 0.999, with_n256: bool = True):
    """The learned restart pruner, trained untimed on the method's own restart trajectories from
    workloads shaped like the small N = 8 mixture and the EEG-like N = 64 and N = 128 cases, and
    (with_n256) an EEG-like N = 256 case at reduced T and M (seeds disjoint from the timed data).
    Returns (params, tau, report)."""
    import torch

    import synth
    from paper_2408_17118_gb300 import ica
    from paper_2408_17118_gb300 import pruner as pr

    t0 = time.perf_counter()
    shapes = [synth.small_mixture(seed + 101, iters=30, tol=1e-6), synth.eeg64(seed + 102), synth.eeg128(seed + 103)]
    if with_n256:  # the N = 256 shape at a fifth of the samples and a quarter of the restarts
        shapes.append(synth.eeg_like(256, 200_000, 2048, seed=seed + 104))
    sets = [(ica.ica_whiten(ctx, torch.from_numpy(w.X).to(dev))[0], w.M) for w in shapes]
    F, y = pr.collect_sets(ctx, sets, 30, 1e-6, seed=4321)
    t_col = time.perf_counter() - t0
    params, tau, report = pr.train(ctx, F, y, steps=400, recall=recall)
    report["collect_seconds"] = t_col
    report["collect_and_train_seconds"] = time.perf_counter() - t0
    report["trained_on"] = [f"N={w.N} T={w.T} M={w.M}" for w in shapes]
    return params, tau, report


def upsilon64(w, Xw_host):
    """Eq. 1 of the kurtosis (Eq. 2) of y = w Xw in FP64 (host, chunks of samples)."""
    import numpy as np

    T = Xw_host.shape[1]
    s4 = 0.0
    for t0 in range(0, T, 1 << 18):
        y = w @ Xw_host[:, t0:t0 + (1 << 18)].astype(np.float64)
        y2 = y * y
        s4 += float(np.sum(y2 * y2))
    a = s4 / T - 3.0
    return a - 2.0 * math.log(a / 2.0 + 1.0) if a > -2.0 else math.inf


def upsilon_tie_tol(alpha: float) -> float:
    """FP32 resolution of Upsilon (Eq. 1) at kurtosis alpha: the relative kurtosis error 1e-4 that
    FP32 parity allows, times |dUpsilon/dalpha| = |(alpha/2) / (alpha/2 + 1)| (steep next to
    binary-like sources, alpha -> -2)."""
    a = float(alpha)
    slope = abs((a / 2.0) / (a / 2.0 + 1.0)) if a > -2.0 else math.inf
    return 1e-4 * abs(a) * slope + 1e-6


def judge_same_components(Wu, st_u, Wp, Xw_host):
    """The pruner's judge: the pruned fit must pick the unpruned fit's components, in order.
    Compared: every component the Gaussianity test (Eq. 3) calls non-Gaussian in the unpruned fit
    (Upsilon above 2 (N - i + 2)(N - i + 1) / T; beyond them lies the Gaussian subspace, where no
    direction is unique, Theorem 1). Each such component must appear in the pruned fit; where it
    appears at another position, or the pruned fit has another direction in its place, the two
    objectives (FP64 Upsilon of the directions involved) must tie within the FP32 resolution of
    Upsilon (upsilon_tie_tol): an order FP32 cannot decide."""
    import numpy as np

    N, T = Xw_host.shape
    comps = st_u["components"]
    ng = 0
    for c in comps:
        if c["upsilon"] < 2.0 * (N - c["i"] + 2) * (N - c["i"] + 1) / T:
            break
        ng += 1
    Wp = np.asarray(Wp)
    cos = np.abs(np.asarray(Wu[:ng]) @ Wp.T) if len(Wp) else np.zeros((ng, 0))
    swapped, replaced, bad = [], [], []
    for i in range(ng):
        j = int(np.argmax(cos[i])) if cos.shape[1] else -1
        tol = upsilon_tie_tol(comps[i]["alpha"])
        if j >= 0 and cos[i, j] >= 1 - 1e-5:
            if j != i:  # found at another position: a swap with the unpruned pick at position j
                uj = comps[j]["upsilon"] if j < len(comps) else -math.inf
                (swapped if abs(uj - comps[i]["upsilon"]) <= tol + upsilon_tie_tol(comps[min(j, len(comps) - 1)]["alpha"])
                 else bad).append((i + 1, j + 1, comps[i]["upsilon"], uj))
            continue
        # not found: the pruned fit's direction at position i must tie with it in FP64
        if i >= len(Wp):
            bad.append((i + 1, None, None, None))
            continue
        uu, up = upsilon64(Wu[i], Xw_host), upsilon64(Wp[i], Xw_host)
        (replaced if up >= uu - tol else bad).append((i + 1, None, uu, up))
    return {"non_gaussian": ng, "same_position": ng - len(swapped) - len(replaced) - len(bad),
            "swapped_ties": swapped, "replaced_ties": replaced, "failed": bad, "ok": not bad}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2408_17118_gb300 import ica

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(args.config, args.seed + rank)
    N, T, M, K = w.N, w.T, w.M, w.n_components
    if args.components > 0:
        K = min(K, args.components)
    X_host = torch.from_numpy(w.X).pin_memory()
    X = X_host.to(dev)
    ctx = ica.Context(local)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    seed_fit = 1234 + rank

    prune = not args.no_prune
    params, tau, train_report = None, None, None
    log(f"workload {w.name} ready")
    if prune:
        params, tau, train_report = train_pruner(ctx, dev, args.seed, args.prune_recall, args.prune_train == "n256")
        log(f"pruner trained: {train_report}")
    # headline: BF16 (+ pruner); profile = 1 records CUDA events around each stage launch on the
    # library's stream inside the timed steps (the roofline's kernel time)
    head_prec = ica.ICA_FP8 if args.precision == "fp8" else ica.ICA_BF16
    opts_head = ica.ica_default_opts(precision=head_prec, profile=1)
    if args.stage_lo_from >= 0:
        opts_head.stage_lo_from = args.stage_lo_from
    if args.stage_streamk >= 0:
        opts_head.stage_streamk = args.stage_streamk
    if args.fp8_iters >= 0:
        opts_head.fp8_iters = args.fp8_iters
    tau_trained = tau
    if prune:
        if args.prune_tau >= 0:
            tau = args.prune_tau
        opts_head.prune_tau = tau
        opts_head.prune_cos = args.prune_cos

    def fit(o, pp, Xd=X):
        Xw, V, mean = ica.ica_whiten(ctx, Xd)
        W, kurt = ica.ica_order_fit(ctx, Xw, M, K, w.iters, w.tol, seed_fit, o, prune_params=pp)
        return W, kurt, Xw

    def fit_flops(st):
        return sum(v["flops"] for v in st["fused"].values())

    def fit_nominal(st):
        return sum(c["iterations"] for c in st["components"]) * 4.0 * N * M * T

    def timed_steps(o, pp, steps, sampler=None, nvtx=False):
        ms, sts, out = [], [], None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        for _ in range(steps):
            flush.zero_()  # L2 flushed between timed steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if nvtx:
                torch.cuda.nvtx.range_push("timed_step")
            e0.record(stream)
            out = fit(o, pp)
            e1.record(stream)
            if nvtx:
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            sts.append(json.loads(ica.ica_last_stats(ctx)))
        barrier()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        return ms, sts, out, clocks

    for _ in range(max(args.warmup, 3)):
        fit(opts_head, params)
    torch.cuda.synchronize()
    log("warm-up done")
    launches0 = json.loads(ica.ica_last_stats(ctx))["launches_total"]
    step_ms, stats, (W, kurt, Xw), clocks = timed_steps(opts_head, params, args.steps, ClockSampler(local), args.nvtx)
    launches = stats[-1]["launches_total"] - launches0
    total_ms = sum(step_ms)
    flops = sum(fit_flops(s) for s in stats)
    nominal = sum(fit_nominal(s) for s in stats)
    total_ms_max, flops_all, nominal_all = aggregate_over_ranks(total_ms, flops, nominal, world, dev)
    tflops = flops_all / (total_ms_max / 1e3) / 1e12

    # per-kernel device times of the timed steps (library events around each launch)
    kinds = {}
    for st in stats:
        for k, v in st["fused"].items():
            a = kinds.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0})
            for f in a:
                a[f] += v[f]
    phases = {k: v["ms"] / args.steps for k, v in kinds.items()}
    for st in stats:
        for k, v in st.get("phases", {}).items():
            phases[k] = phases.get(k, 0.0) + v["ms"] / args.steps

    def summary(sts, ms):
        last = sts[-1]["components"]
        return {"time_to_all_components_s": statistics.median(ms) / 1e3,
                "tflops": sum(fit_flops(x) for x in sts) / (sum(ms) / 1e3) / 1e12,
                "rows_updated": sum(c["rows_updated"] for c in last),
                "restarts_pruned": sum(c["pruned"] for c in last),
                "fallbacks": sum(c["fallback"] for c in last)}

    head = summary(stats, step_ms)
    log(f"headline {head}")
    if K <= 8:  # per-component iterations of the last timed step (profile captures need them)
        log("components " + str([(c["i"], c["iterations"], c["rows_updated"]) for c in stats[-1]["components"]]))
    # the same fits without the pruner (the pruner's fallback and judge)
    unpruned, judge = None, None
    if prune:
        opts_u = ica.ica_default_opts(precision=ica.ICA_BF16)
        fit(opts_u, None)
        u_ms, u_st, (Wu, ku, _), _ = timed_steps(opts_u, None, max(1, args.side_steps))
        unpruned = summary(u_st, u_ms)
        judge = judge_same_components(Wu.cpu().numpy(), u_st[-1], W.cpu().numpy(), Xw.cpu().numpy())
        log(f"unpruned {unpruned} judge {judge}")

    # the pruner with the network's trained threshold: timed once and judged like the headline
    network = None
    if prune and not args.no_network_leg and tau_trained is not None and tau_trained != tau:
        opts_n = ica.ica_default_opts(precision=ica.ICA_BF16)
        opts_n.prune_tau = tau_trained
        opts_n.prune_cos = args.prune_cos
        n_ms, n_st, (Wn, kn, _), _ = timed_steps(opts_n, params, 1)
        network = summary(n_st, n_ms)
        network["tau"] = tau_trained
        network["judge"] = judge_same_components(Wu.cpu().numpy(), u_st[-1], Wn.cpu().numpy(), Xw.cpu().numpy())
        log(f"network leg {network}")

    # the FP8 form with the headline's pruner: timed (side steps) and judged like the headline,
    # against the unpruned BF16 fit (or, without the pruner, against the headline's BF16 fit)
    fp8 = None
    if not args.no_fp8_leg:
        opts_8 = ica.ica_default_opts(precision=ica.ICA_FP8, profile=1)
        if args.fp8_iters >= 0:
            opts_8.fp8_iters = args.fp8_iters
        if prune:
            opts_8.prune_tau = tau
            opts_8.prune_cos = args.prune_cos
        fit(opts_8, params)
        f_ms, f_st, (W8, k8, _), _ = timed_steps(opts_8, params, max(1, args.side_steps))
        fp8 = summary(f_st, f_ms)
        fp8["stage_fp8_launches"] = f_st[-1].get("stage_fp8_launches")
        fp8["stage_ms"] = sum(x["fused"]["iteration"]["ms"] for x in f_st) / len(f_st)
        ref_W, ref_st = (Wu, u_st[-1]) if prune else (W, stats[-1])
        fp8["judge"] = judge_same_components(ref_W.cpu().numpy(), ref_st, W8.cpu().numpy(), Xw.cpu().numpy())
        fp8["judged_against"] = "unpruned BF16 fit" if prune else "headline BF16 fit"
        log(f"fp8 leg {fp8}")

    # e2e through the public API with host buffers: H2D of X (pinned), whiten + fit, D2H of W, kurt
    e2e_ms, e2e_flops = [], 0.0
    W_host = torch.empty((K, N), dtype=torch.float64).pin_memory()
    k_host = torch.empty(K, dtype=torch.float64).pin_memory()
    for _ in range(max(1, args.side_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd = X_host.to(dev, non_blocking=True)
        Wd, kd, _ = fit(opts_head, params, Xd)
        W_host[: Wd.shape[0]].copy_(Wd, non_blocking=True)
        k_host[: kd.shape[0]].copy_(kd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_flops += fit_flops(json.loads(ica.ica_last_stats(ctx)))
    e2e_tflops = e2e_flops / (sum(e2e_ms) / 1e3) / 1e12
    log(f"e2e {e2e_ms}")

    # plain FP32 matrix form on the same GPU (the comparator): one fit after a small untimed one
    # that creates the cuBLAS handle
    plain = None
    if not args.no_compare and world == 1:
        kp = args.plain_components if args.plain_components >= 0 else (8 if args.config == "eeg256" else 0)
        kp = K if kp == 0 or kp > K else kp
        popts = ica.ica_default_opts(precision=ica.ICA_PLAIN_FP32)
        Xw_s, _, _ = ica.ica_whiten(ctx, X[:8, :4096].contiguous())
        ica.ica_order_fit(ctx, Xw_s, 64, 2, 5, 1e-6, 1, popts)  # creates the cuBLAS handle

        def prefix_steps(o, pp, steps):
            ms, sts = [], []
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                Xw_p, _, _ = ica.ica_whiten(ctx, X)
                ica.ica_order_fit(ctx, Xw_p, M, kp, w.iters, w.tol, seed_fit, o, prune_params=pp)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                sts.append(json.loads(ica.ica_last_stats(ctx)))
            return ms, sts

        p_ms, p_st = prefix_steps(popts, None, 1)
        plain = summary(p_st, p_ms)
        plain.update({"dtype": "f32", "impl": "cuBLAS SGEMM (no TF32), Z materialised in device memory",
                      "components": kp})
        if kp < K:  # the headline configuration on the same components, for a like-for-like ratio
            b_ms, b_st = prefix_steps(opts_head, params, 2)
            plain["bf16_same_components"] = summary(b_st[1:], b_ms[1:])
            plain["speedup_same_components"] = (plain["time_to_all_components_s"] /
                                                plain["bf16_same_components"]["time_to_all_components_s"])
        log(f"plain {plain}")

    # parity spot check of the last timed result: orthonormal rows
    Wc = W.cpu().numpy()
    orth = float(np.abs(Wc @ Wc.T - np.eye(Wc.shape[0])).max())

    # roofline of the dominant kernel: the persistent BF16 stage (one launch per component runs
    # every iteration: update, row completion, removal of converged rows)
    peaks, peak_src = load_peaks()
    it = kinds.get("iteration", {"launches": 0, "ms": 0.0, "flops": 0.0})
    achieved = it["flops"] / (it["ms"] / 1e3) / 1e12 if it["ms"] > 0 else 0.0
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    # X~ bytes the stage reads per launch: one pass per iteration (X~ larger than L2 at N = 256)
    xt_iter_bytes = sum(c["iterations"] * ((N - c["i"] + 1 + 15) // 16 * 16) * T * 2.0
                        for c in stats[-1]["components"])
    ratio = STAGE_TRAFFIC_RATIO.get(args.config)
    traffic = ratio * xt_iter_bytes / max(1, it["launches"] / max(1, args.steps)) if ratio else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": ("ncu dram read+write of a captured stage launch / (its iterations x n_pad T 2 B), "
                                 "times the fit's iterations x X~ bytes per launch" if ratio else
                                 "no ncu capture of the current stage kernel at this workload"),
                "kernel": "stage_tc_kernel (persistent BF16 stage: tcgen05 update, row completion, removal of "
                          "converged rows)",
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "launches": it["launches"], "avg_launch_ms": it["ms"] / max(1, it["launches"]),
                "algorithmic_flops_per_launch": it["flops"] / max(1, it["launches"]),
                "share_of_step": it["ms"] / total_ms if total_ms else None,
                "timing": "CUDA events on the library stream around each launch, inside the timed steps"}

    cert = None
    if args.certify and rank == 0:
        import oracle

        opts_c = ica.ica_default_opts(precision=ica.ICA_BF16)
        cands = torch.zeros((K, opts_c.refine_topk, N), dtype=torch.float64, device=dev)
        Xw_c, _, _ = ica.ica_whiten(ctx, X)
        Wc2, kc2 = ica.ica_order_fit(ctx, Xw_c, M, K, w.iters, w.tol, seed_fit, opts_c, record_cands=cands)
        t0 = time.perf_counter()
        kk = min(args.certify, Wc2.shape[0])
        checks = oracle.certify_picks(Xw_c.cpu().numpy().astype(np.float64), Wc2.cpu().numpy(), cands.cpu().numpy(),
                                      K=30, eps=1e-9, components=range(kk))
        # components the Gaussianity test (Eq. 3) calls non-Gaussian; beyond them lies the Gaussian
        # subspace, where no direction is unique (Theorem 1) and no pick is a certified fixed point
        kc = kc2.cpu().numpy()
        ng = 0
        for i in range(len(kc)):
            a = float(kc[i])
            ups = a - 2.0 * math.log(a / 2.0 + 1.0) if a > -2.0 else math.inf
            if ups < 2.0 * (N - i + 1) * (N - i) / T:
                break
            ng += 1
        bad = [c.i + 1 for c in checks if c.pick_cos < 1 - 1e-5 or c.margin < -1e-4 * max(1, abs(c.ups_pick))]
        ngc = [c for c in checks if c.i < ng]
        cert = {"components": kk, "non_gaussian": min(ng, kk), "seconds": time.perf_counter() - t0,
                "min_pick_cos_non_gaussian": min((c.pick_cos for c in ngc), default=None),
                "min_margin_non_gaussian": min((c.margin for c in ngc), default=None),
                "failed_non_gaussian": [i for i in bad if i <= ng],
                "unmet_in_gaussian_subspace": [i for i in bad if i > ng]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, fl, desc = oracle_sample(w, ORACLE_RESTARTS.get(args.config, 64))
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle", "sample": desc,
               "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "e4m3+bf16",
            "data": "synthetic (seeded generators, synth/; stands in for the paper's EEG recordings)",
            "config": {"workload": workload_desc(w), "components_fitted": K,
                       "precision": ("bf16 tcgen05 + fp32 refinement" if args.precision == "bf16" else
                                     "e4m3 tcgen05 (stage iterations 1-3) + bf16 tcgen05 + fp32 refinement"),
                       "pruner": (f"on: keep floor {opts_head.prune_keep_frac:g} + redundancy |cos| >= "
                                  f"{args.prune_cos:g} + Gaussian-subspace rule (Eq. 3 at iteration 5), "
                                  f"network threshold {tau:g} (trained untimed; see "
                                  f"pruner_network_leg for its trained threshold)") if prune else "off",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "time_to_all_components_s": head["time_to_all_components_s"],
            "nominal_tflops": nominal_all / (total_ms_max / 1e3) / 1e12,
            "headline": head, "unpruned": unpruned, "pruner_judge": judge, "pruner_training": train_report,
            "pruner_network_leg": network,
            "fp8_leg": fp8,
            "plain_fp32": plain,
            "speedup_vs_plain_fp32": (plain["time_to_all_components_s"] / head["time_to_all_components_s"]
                                      if plain["components"] == K else plain["speedup_same_components"])
            if plain else None,
            "speedup_vs_unpruned": (unpruned["time_to_all_components_s"] / head["time_to_all_components_s"])
            if unpruned else None,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": int(X_host.numel() * 4),
                    "d2h_bytes_per_step": int(K * N * 8 + K * 8), "time_s": statistics.median(e2e_ms) / 1e3},
            "clocks": clocks, "gpu_launches": int(launches),
            "fused_kinds": kinds, "phase_ms_per_step": phases, "orthonormality": orth, "certify": cert,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    ctx.close()
    return 0

def run_kernel_step(args):
    """One fused BF16 update step (the iteration kernel plus the split combine), repeated."""
    import torch

    from paper_2408_17118_gb300 import ica

    w = workload(args.config, args.seed)
    n, M, T = w.X.shape[0], w.M, args.kernel_step
    dev = torch.device("cuda", 0)
    ctx = ica.Context(0)
    g = torch.Generator(device=dev).manual_seed(args.seed)
    n_pad = (n + 15) // 16 * 16
    ld = (T + 7) // 8 * 8
    Xt = torch.zeros((n_pad, ld), device=dev, dtype=torch.bfloat16)
    Xt[:n] = torch.randn((n, ld), device=dev, generator=g).to(torch.bfloat16)
    B = torch.zeros((M, n_pad), device=dev)
    B[:, :n] = torch.nn.functional.normalize(torch.randn((M, n), device=dev, generator=g), dim=1)
    for _ in range(max(args.warmup, 1)):
        ica.ica_fp_step(ctx, ica.ICA_BF16, B, n, Xt, T)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ica.ica_fp_step(ctx, ica.ICA_BF16, B, n, Xt, T)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"mode": "kernel_step", "n": n, "M": M, "T": T, "ms_per_call": ms,
                      "note": "ica_fp_step is synchronous: the time includes the call's host overhead"}), flush=True)
    ctx.close()
    return 0


def run_batch(args):
    """32 data sets of uneven N (16..128) and T (2e4..4e5, log-uniform), M = 512 restarts each,
    all components: whitening of every set plus one ica_order_fit_batched call per step, timed
    against the same sets fitted one after another (workers = 1)."""
    import numpy as np
    import torch

    import synth
    from paper_2408_17118_gb300 import ica

    dev = torch.device("cuda", 0)
    ws = synth.batch_of_datasets(count=32, seed=args.seed)
    M, iters, tol = ws[0].M, ws[0].iters, ws[0].tol
    Xs = [torch.from_numpy(w.X).to(dev) for w in ws]
    ctx = ica.Context(0)
    opts = ica.ica_default_opts(precision=ica.ICA_BF16)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(workers):
        Xws = [ica.ica_whiten(ctx, X)[0] for X in Xs]
        ica.ica_order_fit_batched(ctx, Xws, M, iters, tol, 1234, opts, workers=workers)
        return json.loads(ica.ica_last_stats(ctx))

    def flops_of(st):
        return sum(sum(v["flops"] for v in d["fused"].values()) for d in st["datasets"])

    res = {}
    for workers in (args.workers, 1):
        for _ in range(max(1, args.warmup)):
            step(workers)
        times, fl, last = [], 0.0, None
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            last = step(workers)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            fl += flops_of(last)
        res[workers] = {"ms_per_step": float(np.median(times)), "tflops": fl / (sum(times) / 1e3) / 1e12,
                        "cta_div": last["batched"]["cta_div"], "tune_ms": last["batched"]["tune_ms"]}
    main = res[args.workers]
    line = {"metric": METRIC, "value": main["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded generators, synth/)",
            "config": {"workload": "32 data sets, N in {16,32,48,64,96,128}, T log-uniform in [2e4, 4e5], M=512, "
                                   "all components, iters<=30, tol=1e-6", "workers": args.workers,
                       "l2": "flushed between timed steps (256 MB write)"},
            "time_to_all_components_s": main["ms_per_step"] / 1e3,
            "one_at_a_time": {"time_to_all_components_s": res[1]["ms_per_step"] / 1e3, "tflops": res[1]["tflops"]},
            "speedup_vs_one_at_a_time": res[1]["ms_per_step"] / main["ms_per_step"],
            "autotuned_cta_div": main["cta_div"], "tune_ms": main["tune_ms"]}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse_args()
    if args.config == "batch":
        return run_batch(args)
    if args.kernel_step:
        return run_kernel_step(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
