#!/usr/bin/env python3
"""Throughput benchmark of the GB300 portfolio solver.

Metric: solves/sec at 1e-6 relative KKT on one GB300 (batched mixed-precision
form, with the plain per-instance form beside it) and the fraction of the HBM
roofline reached by the solver kernel.

Default workload: the batched mixed-precision configuration, 512 single-period
instances (n ~ U{500..8000}, k in {40, 80}) and 64 multi-period instances
(T ~ U{5..40}, n ~ U{1000..4000}), BF16 F and A panels, FP32 matvecs, FP64
iterate state and FP64 KKT reductions, solved by one call of ff_solve_batch.
One step = one call: the batched repack of all inputs into the solver layout
(one launch) and the persistent solver launch over all 576 instances.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own batch (seeded by rank) with
no collective on the data path: weak scaling; rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle (interior point + polish) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2604_22625_gb300.replicas import dist_env, max_over_ranks, rank_seed, sum_over_ranks  # noqa: E402

METRIC = "solves/sec at 1e-6 rel. KKT on 1 GB300 (batched vs plain form); % HBM roofline"
UNIT = "solves/s"
TOL = 1e-6


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "single_large", "multi", "single_small", "batch_profile", "multi_profile",
                             "diff"])
    ap.add_argument("--max-iter", type=int, default=0, help="iteration cap (profiling runs only)")
    ap.add_argument("--tuned", action="store_true", help="take cta_work / check_every from the autotuner "
                    "(paper_2604_22625_gb300.tune; times candidates on a sample once, then cached)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="call ff_solve_batch directly instead of "
                    "replaying the captured CUDA graph")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-instance form")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the CPU baseline sample")
    ap.add_argument("--diff-multi", type=int, default=0, help="differentiation workload: also this many "
                    "multi-period instances (T=50, n=2000, k=60) through the multi-period adjoint")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def make_workload(name: str, rank: int, diff_multi: int = 0):
    """(problems, precision, description) of a named workload; rank seeds it."""
    from paper_2604_22625_gb300 import synthetic as S
    if name == "batch":
        probs = S.config_batch(seed=rank_seed(3, rank))
        desc = ("batched mixed precision: 512 single-period (n~U{500..8000}, k in {40,80}) + "
                "64 multi-period (T~U{5..40}, n~U{1000..4000}) instances")
        return probs, "bf16", desc
    if name == "batch_profile":
        probs = [p for p in S.config_batch(seed=rank_seed(3, rank), n_single=152, n_multi=0)]
        return probs, "bf16", "profiling case: 152 single-period instances of the batched workload"
    if name == "multi_profile":
        allp = S.config_batch(seed=rank_seed(3, rank))
        probs = sorted([p for p in allp if int(p.T) >= 2], key=lambda p: -p.n * p.T)[:8]
        return probs, "bf16", "profiling case: the 8 largest multi-period instances of the batched workload"
    if name == "diff":
        probs = S.config_diff(seed=rank_seed(4, rank), n_single=64, n_multi=diff_multi)
        extra = (f" + {diff_multi} multi-period instances T=50 n=2000 k=60 (vector-Jacobian products also for "
                 "w_T)") if diff_multi else ""
        return probs, "f32", ("differentiation: 64 single-period instances n=3000 k=60" + extra + ", forward to "
                              "1e-7 relative KKT then the batched adjoint (vector-Jacobian products for alpha, "
                              "F, D, s, q, w0)")
    if name == "single_large":
        return [S.config_single_large(seed=rank_seed(1, rank))], "f32", "single-period n=10000 k=100 m=160, FP32"
    if name == "multi":
        return [S.config_multi(seed=rank_seed(2, rank))], "f32", "multi-period T=20 n=5000 k=80, FP32"
    return [S.config_single_small(seed=rank_seed(0, rank))], "f64", "single-period n=500 k=20, FP64"


def storage_rounded(p, precision):
    if precision == "bf16":
        return p.with_F_rounded_bf16()
    if precision == "f32":
        return p.rounded(np.float32)
    return p


def algorithmic_bytes_per_iter(p, precision: str) -> float:
    """Bytes one iteration of the method must move for instance p:
    2 S(F) + 2 S(A) (each panel read in both matvec directions)
    + S(params) (alpha_t, D_t per period; spread and impact per trade; w0, w_T; L, U)
    + 2 S(z) + S(z0) (iterate read and written, Halpern anchor read),
    z = (x: P n, y_A: P m, y_D: R n).  Panels at the storage precision, state
    and parameters at the iterate precision of the mode (FP32 unless FP64)."""
    n, k = p.F.shape
    m = p.A.shape[0]
    multi = int(p.T) >= 2
    P = int(p.T) - 1 if multi else 1
    R = int(p.T) if multi else 1
    pe = {"bf16": 2, "f32": 4, "f64": 8}[precision]
    se = 8 if precision == "f64" else 4
    panels = 2 * (n * k + m * n) * pe
    params = ((2 * P + 2 * R + 2) * n + 2 * m) * se
    state = 3 * (P * n + P * m + R * n) * se
    return float(panels + params + state)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        sel = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", "GPU-" + uuid if not uuid.startswith("GPU-") else uuid]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    "-lms", "200"]

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons, nsamp = [], [], set(), 0
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            nsamp += 1
            for name, val in zip(self.REASONS, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        try:
            os.unlink(self.file.name)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": nsamp}


# ---------------------------------------------------------------------------
# distributed plumbing (timing only: no collective touches the data path)
# ---------------------------------------------------------------------------
def dist_init(backend: str):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample_rate(problems, precision, budget_s: float, start: int = 0):
    """Time the oracle on a stratified sample; return (solves/s estimate for
    the whole workload, sample description, seconds spent)."""
    import oracle
    singles = [p for p in problems if int(p.T) < 2]
    multis = [p for p in problems if int(p.T) >= 2]
    ts, tm = [], []
    t_begin = time.perf_counter()
    i = start
    while True:
        if singles:
            p = storage_rounded(singles[i % len(singles)], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            ts.append(time.perf_counter() - t0)
        if multis and (not tm or time.perf_counter() - t_begin < 0.6 * budget_s):
            p = storage_rounded(multis[i % len(multis)], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            tm.append(time.perf_counter() - t0)
        i += 1
        if time.perf_counter() - t_begin >= budget_s:
            break
    est = len(singles) * (statistics.mean(ts) if ts else 0.0) + len(multis) * (statistics.mean(tm) if tm else 0.0)
    rate = len(problems) / est if est > 0 else 0.0
    desc = (f"{len(ts)} of {len(singles)} single-period and {len(tm)} of {len(multis)} multi-period instances "
            f"solved by the FP64 oracle; rate = {len(problems)} / ({len(singles)} mean_single + "
            f"{len(multis)} mean_multi)")
    return rate, desc, time.perf_counter() - t_begin, ts, tm


def cpu_cores() -> int:
    n = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            n = min(n, int(os.environ[var]))
    return n


# ---------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    probs, precision, desc = make_workload(args.workload, 0, args.diff_multi)
    singles = [p for p in probs if int(p.T) < 2]
    multis = [p for p in probs if int(p.T) >= 2]

    import oracle

    def step(i, ts, tm):
        if singles:
            p = storage_rounded(singles[i % len(singles)], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            ts.append(time.perf_counter() - t0)
        if multis:
            p = storage_rounded(multis[i % len(multis)], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            tm.append(time.perf_counter() - t0)

    # warm-up: one single-period solve per step (loads the code and the BLAS
    # threads; a multi-period instance takes minutes on the host cores)
    smallest = min(probs, key=lambda p: p.F.shape[0] * max(1, int(p.T) - 1))
    for _ in range(args.warmup):
        oracle.solve(storage_rounded(smallest, precision))
    ts, tm = [], []
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i, ts, tm)
    wall = time.perf_counter() - t0
    est = len(singles) * (statistics.mean(ts) if ts else 0.0) + len(multis) * (statistics.mean(tm) if tm else 0.0)
    value = len(probs) / est if est > 0 else 0.0
    sample = (f"each timed step: one single-period and one multi-period instance of the workload (in "
              f"workload order from the first), solved by the FP64 oracle (interior point + active-set "
              f"polish); warm-up steps solve the smallest instance once each; value = {len(probs)} / "
              f"({len(singles)} mean_single + {len(multis)} mean_multi)")
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "instances": len(probs), "tol": TOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")

    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300.build import build
    build()

    probs, precision, desc = make_workload(args.workload, rank, args.diff_multi)
    opt_kw = {"time_limit": 600.0}
    if args.max_iter > 0:
        opt_kw["max_iter"] = args.max_iter
    diff = args.workload == "diff"
    if diff:
        opt_kw["tol"] = 1e-7
    tuned = None
    if args.tuned:
        from paper_2604_22625_gb300 import tune
        tuned = tune.tune(probs, precision=precision, tol=opt_kw.get("tol", TOL),
                          device=torch.cuda.get_device_name(dev))
        opt_kw.update(tuned.options())
    runner = api.BatchRunner(probs, precision=precision, device=str(dev), duals=diff, **opt_kw)
    tol_ok = 1e-7 if diff else TOL
    if diff:
        runner.prepare_backward()
        gen = torch.Generator(device="cpu").manual_seed(4)
        runner.g_dev.copy_(torch.randn(runner.g_dev.shape, generator=gen, dtype=runner.g_dev.dtype))
    stream = torch.cuda.current_stream(dev)
    bpi = [algorithmic_bytes_per_iter(p, precision) for p in probs]
    resident_in = runner.h2d_bytes

    use_graph = not args.no_graph and not diff
    if use_graph:
        runner.capture(stream)
    if diff:
        def step(s_):
            runner.run(s_)
            runner.backward(s_)
    else:
        step = runner.replay if use_graph else runner.run
    for _ in range(args.warmup):
        step(stream)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    solved_steps, iters_steps, kkt_max = [], [], 0.0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    t_wall = time.perf_counter()
    for s in range(args.steps):
        ev[s][0].record(stream)
        step(stream)
        ev[s][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    infos = runner.results()   # the last step's results (every step solves the same inputs)
    solved = sum(1 for i in infos if i["status"] == 0 and i["rel_kkt"] <= tol_ok)
    kkt_max = max(i["rel_kkt"] for i in infos)
    iters = [int(i["iterations"]) for i in infos]
    inst_s = [float(i["seconds"]) for i in infos]
    alg_bytes = float(sum(b * it for b, it in zip(bpi, iters)))

    launches_per_step = 1 + runner.solver_launches() + (runner.backward_launches() if diff else 0)
    t_max = max_over_ranks(dist, dev_s, dev)
    solved_all = sum_over_ranks(dist, float(solved * args.steps), dev)
    value = solved_all / t_max if t_max > 0 else 0.0
    mean_step_s = dev_s / max(args.steps, 1)
    achieved = alg_bytes / mean_step_s / 1e9 if mean_step_s > 0 else 0.0

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        peaks = {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # end to end through the public API: pinned host inputs -> solve -> host results
    e2e = None
    if not args.no_e2e and not diff:
        k_e2e = 1
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            runner.run_from_host(stream)
            stream.synchronize()
        e2e_s = (time.perf_counter() - t0)
        rec = runner.res_host.numpy().view(api.L.RESULT_DTYPE)
        e2e_solved = int(sum(1 for r in rec if r["status"] == 0 and r["rel_kkt"] <= TOL))
        e2e_t = max_over_ranks(dist, e2e_s, dev)
        e2e_solved_all = sum_over_ranks(dist, float(e2e_solved * k_e2e), dev)
        e2e = {"value": e2e_solved_all / e2e_t if e2e_t > 0 else 0.0, "unit": UNIT,
               "h2d_bytes_per_step": int(runner.h2d_bytes), "d2h_bytes_per_step": int(runner.d2h_bytes),
               "steps": k_e2e}

    # plain per-instance form (FP32 panels and matvecs, one solve call per instance), sampled
    plain = None
    if not args.no_plain and args.workload == "batch" and rank == 0:
        singles = [p for p in probs if int(p.T) < 2][:3]
        multis = [p for p in probs if int(p.T) >= 2][:1]
        ts, tm, ok = [], [], 0
        for grp, acc in ((singles, ts), (multis, tm)):
            for p in grp:
                sol = api.solve(p.rounded(np.float32), precision="f32", device=str(dev), time_limit=600.0)
                acc.append(sol.info["seconds"])
                ok += int(sol.info["status"] == 0 and sol.info["rel_kkt"] <= TOL)
        ns = sum(1 for p in probs if int(p.T) < 2)
        nm = len(probs) - ns
        est = ns * statistics.mean(ts) + nm * statistics.mean(tm)
        plain = {"value": len(probs) / est, "unit": UNIT, "converged": f"{ok}/{len(ts) + len(tm)}",
                 "sample": f"{len(ts)} single + {len(tm)} multi instances of the batch solved one call each "
                           f"(FP32 panels, automatic cluster size); rate = {len(probs)} / "
                           f"({ns} mean_single + {nm} mean_multi) of device seconds"}

    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1 and not diff:
        rate, sample, spent, ts, tm = oracle_sample_rate(probs, precision, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample}

    if rank == 0:
        l2_mb = torch.cuda.get_device_properties(dev).L2_cache_size / 2 ** 20
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "f32": "f32", "f64": "f64"}[precision],
            "data": "synthetic",
            "config": {"workload": desc, "instances": len(probs), "tol": tol_ok,
                       "precision": {"bf16": "BF16 F/A panels, FP32 matvecs, FP64 iterate state and KKT",
                                     "f32": "FP32 panels and matvecs, FP64 iterate state and KKT",
                                     "f64": "FP64 throughout"}[precision],
                       "l2": f"inputs larger than L2 ({resident_in / 2**20:.0f} MiB packed inputs, "
                             f"{runner.ws_bytes / 2**20:.0f} MiB workspace vs {l2_mb:.0f} MiB L2)",
                       "parallelism": f"replicas x{ws} (one batch per GPU)" if ws > 1 else "1 GPU",
                       "max_iter_cap": args.max_iter or None,
                       "schedule": tuned.options() if tuned is not None else "default (cta_work 8192, check_every 64)",
                       "graph": use_graph},
            "solved": solved, "max_rel_kkt": kkt_max,
            "iterations_mean": float(statistics.mean(iters)),
            "instance_seconds": {"sum": float(sum(inst_s)), "max": float(max(inst_s))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "team_kernel (+ the one repack launch in the same call)",
                         "peak_source": peak_src},
            "cpu_baseline": cpu,
            "plain_form": plain,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "step_ms": step_ms,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
