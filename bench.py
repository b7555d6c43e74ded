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
(one launch) and the persistent solver launches over all 576 instances (one
per cluster-size group, concurrent), plus the FP64 re-solve of instances that
stop at the FP32 rounding floor.  The batch runs at cta_work 16384 and
check_every 128, the fastest point of the autotuner's grid for this batch
(--cta-work / --check-every, or --tuned to run the autotuner).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other workloads (--workload): diff (forward and batched adjoint), risk (the
risk model of Sec. 3.2 over 21 windows), joint (the joint primal prox
variant against the plain split), paper_grid (the lambda grid of Sec. 4.1 on
paper-shaped synthetic instances), single_small, single_large, multi (one
instance each).

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
                             "diff", "risk", "paper_grid", "joint"])
    ap.add_argument("--grid-n", type=int, default=2000, help="paper_grid: assets per instance")
    ap.add_argument("--joint-count", type=int, default=64, help="joint: single-period instances compared")
    ap.add_argument("--grid-dates", type=int, default=21, help="paper_grid: instances (dates) per setting")
    ap.add_argument("--grid-kinds", default="single,multi", help="paper_grid: comma-separated kinds to run")
    ap.add_argument("--eta", default="literal", choices=["literal", "inverted"], help="paper_grid: reading "
                    "of the intraday cost profile")
    ap.add_argument("--primal-weight", type=int, default=-1, help="1/0: adaptive primal weight on/off "
                    "(-1: the library default)")
    ap.add_argument("--max-iter", type=int, default=0, help="iteration cap (profiling runs only)")
    ap.add_argument("--cta-work", type=float, default=16384.0,
                    help="batch workload: asset-periods per CTA (the fastest point of the autotuner's grid "
                         "on this batch in a sweep on GB300; 0 = the library default)")
    ap.add_argument("--check-every", type=int, default=128,
                    help="batch workload: iterations between KKT checks (as --cta-work; 0 = library default)")
    ap.add_argument("--tuned", action="store_true", help="take cta_work / check_every from the autotuner "
                    "(paper_2604_22625_gb300.tune; times candidates on a sample once, then cached)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="call ff_solve_batch directly instead of "
                    "replaying the captured CUDA graph")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-instance form")
    ap.add_argument("--tol", type=float, default=TOL, help="relative KKT tolerance of the timed solves")
    ap.add_argument("--no-oracle-check", action="store_true", help="skip the oracle check of the timed outputs")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration solves")
    ap.add_argument("--check-singles", type=int, default=8)
    ap.add_argument("--check-multis", type=int, default=3)
    ap.add_argument("--check-workers", type=int, default=4)
    ap.add_argument("--plain-singles", type=int, default=16)
    ap.add_argument("--plain-multis", type=int, default=8)
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
# stratified samples of a workload (shared by the oracle check, the plain
# per-instance form and both CPU baselines)
# ---------------------------------------------------------------------------
def strata(problems, kind: str, count: int):
    """Indices of ``count`` instances of one kind ("single" / "multi") at the
    centres of ``count`` equal-count strata of the size order (asset-periods
    times rows), so that each stratum's instance stands for it."""
    idx = [i for i, p in enumerate(problems) if (int(p.T) >= 2) == (kind == "multi")]
    if not idx or count <= 0:
        return []
    key = lambda i: (problems[i].F.shape[0] * max(1, int(problems[i].T) - 1) *  # noqa: E731
                     (problems[i].F.shape[1] + problems[i].A.shape[0]), i)
    idx.sort(key=key)
    count = min(count, len(idx))
    return [idx[min(len(idx) - 1, int((2 * j + 1) * len(idx) / (2 * count)))] for j in range(count)]


def extremes(problems, kind: str, count: int):
    """``count`` instances of one kind spread over the size order, both ends included."""
    idx = [i for i, p in enumerate(problems) if (int(p.T) >= 2) == (kind == "multi")]
    if not idx or count <= 0:
        return []
    idx.sort(key=lambda i: (problems[i].F.shape[0] * max(1, int(problems[i].T) - 1), i))
    pos = np.unique(np.round(np.linspace(0, len(idx) - 1, min(count, len(idx)))).astype(int))
    return [idx[j] for j in pos]


# ---------------------------------------------------------------------------
# the oracle against the GPU's outputs (a spawned process pool: the oracle is
# CPU work and must not be forked from a process that holds a CUDA context)
# ---------------------------------------------------------------------------
def _oracle_check_one(task):
    """Worker: (tag, problem, precision, x, yA, yD) -> comparison with the oracle."""
    import oracle
    from oracle import Scaled
    from oracle.kkt import evaluate
    tag, prob, precision, x, yA, yD = task
    pr = storage_rounded(prob, precision)
    sc = Scaled(pr)
    t0 = time.perf_counter()
    ref = oracle.solve(pr, polish_max_vars=10 ** 7)
    x = np.asarray(x, dtype=np.float64).reshape(sc.P, sc.n)
    out = {"tag": tag, "err_inf": float(np.max(np.abs(x - ref.x))),
           "obj_gap": abs(sc.objective(x) - ref.obj) / abs(ref.obj),
           "oracle_certified": bool(ref.polished), "oracle_rel_kkt": float(ref.kkt.rel_kkt),
           "oracle_s": time.perf_counter() - t0}
    if yA is not None and yD is not None:
        k = evaluate(sc, x, yA, yD)
        out["rel_kkt"] = float(k.rel_kkt)
    return out


def _oracle_time_one(task):
    """Worker: seconds of one oracle solve."""
    import oracle
    prob, precision = task
    t0 = time.perf_counter()
    oracle.solve(storage_rounded(prob, precision))
    return time.perf_counter() - t0


def spawn_pool(workers: int):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(processes=workers)


def summarize_check(rows, bars=(1e-5, 1e-6)):
    """oracle_check block of the bench line."""
    if not rows:
        return None
    return {"n": len(rows), "max_err_inf": max(r["err_inf"] for r in rows),
            "max_obj_gap_strict": max(r["obj_gap"] for r in rows),
            "max_rel_kkt_strict": max((r.get("rel_kkt", float("nan")) for r in rows), default=None),
            "within_bars": all(r["err_inf"] <= bars[0] and r["obj_gap"] <= bars[1] for r in rows),
            "oracle_certified": sum(1 for r in rows if r["oracle_certified"]),
            "instances": rows}


# ---------------------------------------------------------------------------
# CPU oracle timing (stratified sample; the same sample in both arms)
# ---------------------------------------------------------------------------
CPU_SINGLES = 4
CPU_MULTIS = 4


def cpu_sample(problems):
    """The instances the CPU baselines time: CPU_SINGLES single-period and
    CPU_MULTIS multi-period instances at the centres of equal-count size strata."""
    return strata(problems, "single", CPU_SINGLES), strata(problems, "multi", CPU_MULTIS)


def cpu_rate(problems, ts, tm):
    """Whole-workload rate from the stratum means: N / (N_s mean_s + N_m mean_m)."""
    ns = sum(1 for p in problems if int(p.T) < 2)
    nm = len(problems) - ns
    est = ns * (statistics.mean(ts) if ts else 0.0) + nm * (statistics.mean(tm) if tm else 0.0)
    return len(problems) / est if est > 0 else 0.0


def cpu_sample_desc(problems, si, mi, reps: str):
    ns = sum(1 for p in problems if int(p.T) < 2)
    nm = len(problems) - ns
    sz = ", ".join(f"T={int(problems[i].T)} n={problems[i].F.shape[0]}" for i in mi)
    return (f"{len(si)} single-period and {len(mi)} multi-period instances of the workload at the centres of "
            f"equal-count size strata (multi: {sz}), solved by the FP64 oracle (interior point + active-set "
            f"polish) {reps}; value = {len(problems)} / ({ns} mean_single + {nm} mean_multi)")


def oracle_sample_rate(problems, precision):
    """Time the oracle once on every instance of the stratified CPU sample."""
    import oracle
    si, mi = cpu_sample(problems)
    ts, tm = [], []
    t_begin = time.perf_counter()
    for grp, acc in ((si, ts), (mi, tm)):
        for i in grp:
            p = storage_rounded(problems[i], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            acc.append(time.perf_counter() - t0)
    return (cpu_rate(problems, ts, tm), cpu_sample_desc(problems, si, mi, "once each"),
            time.perf_counter() - t_begin, ts, tm)


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
    si, mi = cpu_sample(probs)

    import oracle

    def step(i, ts, tm):
        # one single-period instance per step, cycling through the stratified
        # sample; the multi-period sample (minutes each on the host cores) is
        # spread over the steps, each instance once: step i takes those with
        # index = i mod K, so the whole run stays within a few minutes
        if si:
            p = storage_rounded(probs[si[i % len(si)]], precision)
            t0 = time.perf_counter()
            oracle.solve(p)
            ts.append(time.perf_counter() - t0)
        for j in range(i, len(mi), max(args.steps, 1)):
            p = storage_rounded(probs[mi[j]], precision)
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
    value = cpu_rate(probs, ts, tm)
    sample = cpu_sample_desc(probs, si, mi, "one single-period instance per timed step cycling through the "
                             "sample, and each multi-period instance of the sample once, spread over the steps; "
                             "warm-up steps solve the smallest instance once each")
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
def _outputs(runner, i):
    """(x, yA, yD) of instance i as host arrays (duals None when not kept)."""
    P, n = runner.P[i], runner.n[i]
    x = runner.w_dev[int(runner.w_off[i]):int(runner.w_off[i]) + P * n].double().cpu().numpy()
    if runner.yD_ptrs is None:
        return x, None, None
    p = runner.problems[i]
    m = int(np.asarray(p.A).shape[0])
    R = int(p.T) if int(p.T) >= 2 else 1
    yA = runner.yA_dev[int(runner.yA_off[i]):int(runner.yA_off[i]) + P * m].double().cpu().numpy()
    yD = runner.yD_dev[int(runner.yD_off[i]):int(runner.yD_off[i]) + R * n].double().cpu().numpy()
    return x, yA, yD


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")

    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300 import synthetic as S
    from paper_2604_22625_gb300.build import build
    build()

    probs, precision, desc = make_workload(args.workload, rank, args.diff_multi)
    opt_kw = {"time_limit": 600.0, "tol": args.tol}
    if args.max_iter > 0:
        opt_kw["max_iter"] = args.max_iter
    diff = args.workload == "diff"
    if diff:
        opt_kw["tol"] = 1e-7
    tuned = None
    schedule = "library default (cta_work 8192, check_every 64)"
    if args.tuned:
        from paper_2604_22625_gb300 import tune
        tuned = tune.tune(probs, precision=precision, tol=opt_kw["tol"], device=torch.cuda.get_device_name(dev))
        opt_kw.update(tuned.options())
        schedule = f"autotuned now: {tuned.options()}"
    elif args.workload == "batch" and (args.cta_work > 0 or args.check_every > 0):
        if args.cta_work > 0:
            opt_kw["cta_work"] = args.cta_work
        if args.check_every > 0:
            opt_kw["check_every"] = args.check_every
        schedule = (f"cta_work {opt_kw.get('cta_work', 8192.0):g}, check_every {opt_kw.get('check_every', 64)}: "
                    "the fastest point of the autotuner's grid (cta_work 4096/8192/16384, check_every 32/64/128) "
                    "for this batch in a sweep on GB300")
    # duals are kept so that the oracle can evaluate the relative KKT of the timed outputs
    runner = api.BatchRunner(probs, precision=precision, device=str(dev), duals=True, **opt_kw)
    tol_ok = opt_kw["tol"]
    if diff:
        runner.prepare_backward()
        gen = torch.Generator(device="cpu").manual_seed(4)
        runner.g_dev.copy_(torch.randn(runner.g_dev.shape, generator=gen, dtype=runner.g_dev.dtype))
    stream = torch.cuda.current_stream(dev)
    bpi = [algorithmic_bytes_per_iter(p, precision) for p in probs]
    resident_in = runner.h2d_bytes
    check_oracle = (not args.no_oracle_check) and rank == 0 and args.workload == "batch"

    use_graph = not args.no_graph and not diff
    if use_graph:
        runner.capture(stream)
    escalated_steps = []

    bw_ev = []   # (start, end) events of the backward pass of each step (diff workload)

    def step(s_):
        if use_graph:
            runner.replay(s_)
        else:
            runner.run(s_)
        escalated_steps.append(runner.finish(s_))
        if diff:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s_)
            runner.backward(s_)
            e1.record(s_)
            bw_ev.append((e0, e1))

    for _ in range(args.warmup):
        step(stream)
    torch.cuda.synchronize(dev)
    escalated_steps.clear()
    bw_ev.clear()

    # the oracle check starts on the warm-up outputs (the timed steps solve the
    # same inputs; their outputs are compared bit for bit below) and runs in
    # spawned processes while the GPU is timed
    pool, pending, picks, snap = None, None, [], {}
    if check_oracle:
        picks = extremes(probs, "single", args.check_singles) + extremes(probs, "multi", args.check_multis)
        snap = {i: _outputs(runner, i) for i in picks}
        workers = max(1, min(len(picks), args.check_workers))
        threads = max(1, cpu_cores() // workers)
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = str(threads)
        pool = spawn_pool(workers)
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
        tasks = [(probs[i].tag, probs[i], precision, *snap[i]) for i in picks]
        # largest first, so that the longest oracle solve starts first
        order = sorted(range(len(tasks)), key=lambda j: -probs[picks[j]].F.shape[0] * max(1, int(probs[picks[j]].T)))
        pending = [(j, pool.apply_async(_oracle_check_one, (tasks[j],))) for j in order]

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
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
    same_outputs = all(all((a is None and b is None) or np.array_equal(a, b) for a, b in zip(snap[i], _outputs(runner, i)))
                       for i in picks)

    esc_launches = 2 * max(escalated_steps, default=0)   # repack + solver launch(es) of the FP64 re-solve (bound)
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
        e2e_solved = int(sum(1 for r in rec if r["status"] == 0 and r["rel_kkt"] <= tol_ok))
        e2e_t = max_over_ranks(dist, e2e_s, dev)
        e2e_solved_all = sum_over_ranks(dist, float(e2e_solved * k_e2e), dev)
        e2e = {"value": e2e_solved_all / e2e_t if e2e_t > 0 else 0.0, "unit": UNIT,
               "h2d_bytes_per_step": int(runner.h2d_bytes), "d2h_bytes_per_step": int(runner.d2h_bytes),
               "steps": k_e2e}

    # plain per-instance form (FP32 panels and matvecs, one solve call per
    # instance), on a sample spread over the size order of each kind
    plain = None
    if not args.no_plain and args.workload == "batch" and rank == 0:
        si = extremes(probs, "single", args.plain_singles)
        mi = extremes(probs, "multi", args.plain_multis)
        ts, tm, ok = [], [], 0
        for grp, acc in ((si, ts), (mi, tm)):
            for i in grp:
                sol = api.solve(probs[i].rounded(np.float32), precision="f32", device=str(dev), time_limit=600.0,
                                tol=tol_ok)
                acc.append(sol.info["seconds"])
                ok += int(sol.info["status"] == 0 and sol.info["rel_kkt"] <= tol_ok)
        ns = sum(1 for p in probs if int(p.T) < 2)
        nm = len(probs) - ns
        est = ns * statistics.mean(ts) + nm * statistics.mean(tm)
        Ts = sorted({int(probs[i].T) for i in mi})
        plain = {"value": len(probs) / est, "unit": UNIT, "converged": f"{ok}/{len(ts) + len(tm)}",
                 "sample": f"{len(ts)} single + {len(tm)} multi instances spread over the size order of each kind "
                           f"(both ends included; multi T in {Ts}), solved one call each (FP32 panels, automatic "
                           f"cluster size); rate = {len(probs)} / ({ns} mean_single + {nm} mean_multi) of device "
                           f"seconds"}

    # the other configurations, one solve each, with the oracle check
    per_config = None
    cfg_pending = []
    if args.workload == "batch" and rank == 0 and not args.no_configs:
        per_config = {}
        for name, prob, prec in (("single n=500 k=20 FP64", S.config_single_small(), "f64"),
                                 ("single n=10000 k=100 m=160 FP32", S.config_single_large(), "f32"),
                                 ("multi T=20 n=5000 k=80 FP32", S.config_multi(), "f32")):
            pr = prob if prec == "f64" else prob.rounded(np.float32)
            sol = api.solve(pr, precision=prec, device=str(dev), return_duals=True, tol=tol_ok, time_limit=600.0)
            per_config[name] = {"status": sol.info["status_name"], "iterations": int(sol.info["iterations"]),
                                "device_s": float(sol.info["seconds"]), "rel_kkt": float(sol.info["rel_kkt"]),
                                "escalated": bool(sol.info["escalated"])}
            if pool is not None:
                cfg_pending.append((name, pool.apply_async(_oracle_check_one,
                                                           ((name, pr, prec, sol.x, sol.yA, sol.yD),))))

    oracle_check = None
    if pool is not None:
        rows = [None] * len(pending)
        for j, fut in pending:
            rows[j] = fut.get()
        oracle_check = summarize_check(rows)
        oracle_check["outputs"] = ("the timed steps' outputs" if same_outputs else
                                   "the warm-up outputs (the timed outputs differed)")
        oracle_check["sample"] = (f"{args.check_singles} single-period and {args.check_multis} multi-period "
                                  f"instances spread over the size order, both ends included")
        for name, fut in cfg_pending:
            r = fut.get()
            per_config[name].update({"err_inf": r["err_inf"], "obj_gap": r["obj_gap"],
                                     "oracle_rel_kkt_at_gpu_point": r.get("rel_kkt"),
                                     "oracle_certified": r["oracle_certified"]})
        pool.close()
        pool.join()

    # the CPU baseline is timed after the pool has finished: alone on the cores
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1 and not diff:
        rate, sample, spent, ts, tm = oracle_sample_rate(probs, precision)
        cpu = {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample,
               "seconds": spent}

    if rank == 0:
        l2_mb = torch.cuda.get_device_properties(dev).L2_cache_size / 2 ** 20
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "f32": "f32", "f64": "f64"}[precision],
            "data": "synthetic",
            "config": {"workload": desc, "instances": len(probs), "tol": tol_ok,
                       "kkt": "relative KKT max(r_primal, r_dual, r_gap), r_gap = |P - D| / (|P| + |D|)",
                       "precision": {"bf16": "BF16 F/A panels, FP32 matvecs, FP64 iterate state and KKT; an "
                                             "instance that ends at the FP32 rounding floor is solved again in "
                                             "FP64 on the same BF16-rounded data inside the step",
                                     "f32": "FP32 panels and matvecs, FP64 iterate state and KKT",
                                     "f64": "FP64 throughout"}[precision],
                       "l2": f"inputs larger than L2 ({resident_in / 2**20:.0f} MiB packed inputs, "
                             f"{runner.ws_bytes / 2**20:.0f} MiB workspace vs {l2_mb:.0f} MiB L2)",
                       "parallelism": f"replicas x{ws} (one batch per GPU)" if ws > 1 else "1 GPU",
                       "max_iter_cap": args.max_iter or None,
                       "schedule": schedule,
                       "graph": use_graph},
            "solved": solved, "max_rel_kkt": kkt_max,
            "escalated_fp64": max(escalated_steps, default=0),
            "iterations_mean": float(statistics.mean(iters)),
            "backward_ms": [a.elapsed_time(b) for a, b in bw_ev] if diff else None,
            "backward_status": ([int(v) for v in runner.bstatus.cpu().tolist()] if diff else None),
            "instance_seconds": {"sum": float(sum(inst_s)), "max": float(max(inst_s))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "team_kernel (+ the one repack launch in the same call)",
                         "peak_source": peak_src},
            "oracle_check": oracle_check,
            "per_config": per_config,
            "cpu_baseline": cpu,
            "plain_form": plain,
            "e2e": e2e,
            "gpu_launches": (launches_per_step + esc_launches) * args.steps,
            "clocks": clocks,
            "step_ms": step_ms,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# risk-model estimation (Sec. 3.2): its own line
# ---------------------------------------------------------------------------
RISK_WINDOWS, RISK_T, RISK_N, RISK_P = 21, 504, 5000, 6


def risk_workload(rank: int):
    from paper_2604_22625_gb300 import synthetic as S
    return [S.make_returns(RISK_T, RISK_N, rank_seed(5, rank) * 1000 + d, p=RISK_P, late_frac=0.1,
                           irregular_frac=0.01) for d in range(RISK_WINDOWS)]


def risk_bytes_per_window(T, n, p) -> float:
    """Algorithmic bytes of one window: R and F read once (float32), beta, D
    (float64), the history counts (int32) and Sigma_f written once."""
    return float(T * n * 4 + T * p * 4 + n * p * 8 + n * 8 + n * 4 + p * p * 8)


def run_risk(args):
    import torch
    ws, rank, local = dist_env()
    desc = (f"risk-model estimation: {RISK_WINDOWS} windows of T={RISK_T} days, n={RISK_N} stocks, p={RISK_P} "
            f"factors (10 % listed inside the window, 1 % with a gap)")
    metric, unit = "estimation windows/sec (Sec. 3.2 factor model, batched)", "windows/s"
    wins = risk_workload(rank)
    if args.impl == "reference":
        if rank != 0:
            return 0
        from oracle import risk
        for _ in range(args.warmup):
            risk.estimate(wins[0].F, wins[0].R[:, :200])
        t0 = time.perf_counter()
        for s_ in range(args.steps):
            w = wins[s_ % len(wins)]
            risk.estimate(w.F, w.R)
        wall = time.perf_counter() - t0
        value = args.steps / wall
        sample = "one window per timed step (all its stocks), oracle least squares per stock"
        print(json.dumps({"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": ws,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": desc},
                          "cpu_baseline": {"value": value, "unit": unit, "cores": cpu_cores(), "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "gpu_launches": 0}), flush=True)
        return 0
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")
    from paper_2604_22625_gb300 import _lib as L
    from paper_2604_22625_gb300.build import build
    build()
    Fh = torch.tensor(np.stack([w.F for w in wins]), dtype=torch.float32).pin_memory()
    Rh = torch.tensor(np.stack([w.R for w in wins]), dtype=torch.float32).pin_memory()
    count, T, p = Fh.shape
    n = Rh.shape[2]
    F = Fh.to(dev)
    R = Rh.to(dev)
    nb = L.ff_risk_workspace_size(count, T, n, p)
    wsb = torch.empty(nb, dtype=torch.uint8, device=dev)
    beta = torch.empty(count, n, p, dtype=torch.float64, device=dev)
    sig = torch.empty(count, p, p, dtype=torch.float64, device=dev)
    D = torch.empty(count, n, dtype=torch.float64, device=dev)
    nobs = torch.empty(count, n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(s_):
        rc = L.ff_risk_estimate(count, T, n, p, F.data_ptr(), R.data_ptr(), 42, beta.data_ptr(), sig.data_ptr(),
                                D.data_ptr(), nobs.data_ptr(), wsb.data_ptr(), nb, s_.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(L.ff_risk_last_error())

    for _ in range(max(3, args.warmup)):
        step(stream)
    torch.cuda.synchronize(dev)
    # inputs (212 MB) exceed the L2; the L2 is also flushed between steps by a 256 MiB write
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    steps = max(args.steps, 10)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(local)
    sampler.start()
    for k in range(steps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        step(stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    mean_s = statistics.mean(ms) / 1e3
    value = count / mean_s
    alg = count * risk_bytes_per_window(T, n, p)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    # end to end: pinned host returns in, estimates out
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    F.copy_(Fh, non_blocking=True)
    R.copy_(Rh, non_blocking=True)
    step(stream)
    out_b = beta.cpu()
    out_d = D.cpu()
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    # oracle check on sampled windows and stocks
    from oracle import risk
    check = []
    bh, dh, nh = out_b.numpy(), out_d.numpy(), nobs.cpu().numpy()
    for d in (0, count - 1):
        ref = risk.estimate(wins[d].F, wins[d].R)
        ok = ref.valid
        check.append({"window": d, "max_abs_beta_err": float(np.max(np.abs(bh[d][ok] - ref.beta[ok]))),
                      "max_rel_D_err": float(np.max(np.abs(dh[d][ok] / ref.D[ok] - 1.0))),
                      "valid_match": bool(np.array_equal(~np.isnan(dh[d]), ok))})
    t0 = time.perf_counter()
    risk.estimate(wins[0].F, wins[0].R)
    cpu_s = time.perf_counter() - t0
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": ws, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * mean_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "l2": "inputs larger than L2 and a 256 MiB L2 flush between steps",
                       "precision": "float32 returns; FP32 chunk sums folded into double-float; FP64 solves"},
            "roofline": {"bound": "hbm", "achieved": alg / mean_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / mean_s / 1e9 / peak, "traffic": None,
                         "kernel": "risk_prep_kernel + risk_ginv_kernel + risk_stream_kernel + "
                                   "risk_finish_kernel (one ff_risk_estimate call, timed as a whole)",
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
            "oracle_check": check,
            "cpu_baseline": {"value": 1.0 / cpu_s, "unit": unit, "cores": cpu_cores(), "kind": "oracle",
                             "sample": "one window (all 5000 stocks) solved by the oracle"},
            "e2e": {"value": count / e2e_s, "unit": unit, "h2d_bytes_per_step": int(Fh.numel() * 4 + Rh.numel() * 4),
                    "d2h_bytes_per_step": int(out_b.numel() * 8 + out_d.numel() * 8)},
            "gpu_launches": 4 * steps, "clocks": clocks, "step_ms": ms}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the paper's experiment shape (Sec. 4.1, Table 1) on synthetic data
# ---------------------------------------------------------------------------
def sgm1(times) -> float:
    """Shifted geometric mean with shift 1 s (Sec. 4.1)."""
    t = np.asarray(times, dtype=np.float64)
    return float(np.exp(np.mean(np.log(t + 1.0))) - 1.0)


def run_paper_grid(args):
    """Every (lambda1, lambda2 = lambda3) setting of the paper's grid, single-
    and multi-period (T = 10, eta profile), grid_dates instances each, solved
    one call each as in the paper's protocol (360 s limit, started at w0),
    with SGM1 and solved counts; the first date of every setting is checked
    against the oracle (spawned processes, concurrent with the GPU)."""
    import torch
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300 import synthetic as S
    from paper_2604_22625_gb300.build import build
    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    workers = max(1, min(8, cpu_cores() // 2))
    threads = max(1, cpu_cores() // workers)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(threads)
    pool = spawn_pool(workers)
    rows, pend = [], []
    grid_kw = {} if args.primal_weight < 0 else {"primal_weight": args.primal_weight}
    t_all = time.perf_counter()
    kinds = [k for k in ("single", "multi") if k in args.grid_kinds.split(",")]
    for kind in kinds:
        for lam23 in S.PAPER_LAMBDA23:
            for lam1 in S.PAPER_LAMBDA1:
                times, its, solved, esc = [], [], 0, 0
                for date in range(args.grid_dates):
                    prob = S.make_paper_instance(date, lam1, lam23, kind, n=args.grid_n, eta_reading=args.eta)
                    pr = prob.rounded(np.float32)
                    sol = api.solve(pr, precision="f32", device=str(dev), return_duals=True, tol=args.tol,
                                    time_limit=360.0, **grid_kw)
                    ok = sol.info["status"] == 0 and sol.info["rel_kkt"] <= args.tol
                    solved += int(ok)
                    esc += int(sol.info["escalated"])
                    # an escalated solve's time includes the FP32 attempt
                    times.append(float(sol.info["seconds"]) + float(sol.info.get("first_seconds", 0.0)))
                    its.append(int(sol.info["iterations"]))
                    if date == 0:
                        pend.append((len(rows), pool.apply_async(
                            _oracle_check_one, ((prob.tag, pr, "f64", sol.x, sol.yA, sol.yD),))))
                rows.append({"kind": kind, "lambda1": lam1, "lambda23": lam23, "solved": solved,
                             "count": args.grid_dates, "sgm1_s": sgm1(times), "max_s": max(times),
                             "iterations_mean": float(np.mean(its)), "escalated_fp64": esc})
    wall = time.perf_counter() - t_all
    for j, fut in pend:
        r = fut.get()
        rows[j].update({"oracle_err_inf": r["err_inf"], "oracle_obj_gap": r["obj_gap"],
                        "oracle_certified": r["oracle_certified"]})
    pool.close()
    pool.join()
    line = {"metric": "paper lambda grid: solved count and SGM1 (s) per setting", "unit": "s",
            "config": {"workload": f"synthetic paper-shaped instances ({'+'.join(kinds)}): n={args.grid_n}, p=6 "
                                   f"factors with a full factor covariance, T=10 (multi, eta {args.eta}), "
                                   f"{args.grid_dates} per setting, FP32, tol {args.tol}, 360 s limit, one solve "
                                   "call each"},
            "wall_s": wall, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_joint(args):
    """The joint primal prox variant (ff_solve_joint_batch) against the plain
    split (ff_solve_batch) on the same single-period instances of the batch
    workload, both in FP64 and to the same tolerance: iterations per instance,
    device time per call (CUDA events on the launching stream), agreement of
    the two solutions, and the oracle on a sample."""
    import torch
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300 import _lib as L
    from paper_2604_22625_gb300 import synthetic as S
    from paper_2604_22625_gb300.build import build
    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    singles = [p for p in S.config_batch(seed=rank_seed(3, 0)) if int(p.T) < 2]
    step = max(1, len(singles) // args.joint_count)
    probs = singles[::step][:args.joint_count]
    count = len(probs)
    stream = torch.cuda.current_stream(dev)
    # joint arm: device problems, workspace and outputs set up once
    dps = [api.to_device(p, dtype=torch.float64, device=str(dev)) for p in probs]
    structs = (L.ff_problem * count)(*[d.struct for d in dps])
    opts = api.options("f64", tol=args.tol, time_limit=360.0)
    nb = L.ff_joint_workspace_size(structs, count)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    res = torch.zeros(count * L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    wj = [torch.empty(d.n, dtype=torch.float64, device=dev) for d in dps]
    yaj = [torch.empty(max(d.m, 1), dtype=torch.float64, device=dev) for d in dps]
    ydj = [torch.empty(d.n, dtype=torch.float64, device=dev) for d in dps]

    def joint_call():
        rc = L.ff_solve_joint_batch(structs, count, opts, ws.data_ptr(), nb, res.data_ptr(),
                                    [t.data_ptr() for t in wj], stream.cuda_stream,
                                    [t.data_ptr() for t in yaj], [t.data_ptr() for t in ydj])
        if rc != L.FF_OK:
            raise RuntimeError(f"ff_solve_joint_batch: {L.ff_status_string(rc)} {L.ff_last_error()}")

    plain = api.BatchRunner(probs, precision="f64", device=str(dev), duals=True, tol=args.tol, time_limit=360.0)

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(max(1, args.warmup)):
        joint_call()
        plain.run(stream)
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    ms_joint = timed(joint_call, steps)
    ms_plain = timed(lambda: plain.run(stream), steps)
    jinfo = [api._info(r) for r in res.cpu().numpy().view(L.RESULT_DTYPE)]
    pinfo = plain.results()
    it_j = np.array([i["iterations"] for i in jinfo], dtype=np.float64)
    it_p = np.array([i["iterations"] for i in pinfo], dtype=np.float64)
    ok_j = sum(1 for i in jinfo if i["status"] == 0 and i["rel_kkt"] <= args.tol)
    ok_p = sum(1 for i in pinfo if i["status"] == 0 and i["rel_kkt"] <= args.tol)
    wp = plain.portfolios()
    diff = max(float(np.max(np.abs(wj[t].cpu().numpy() - np.asarray(wp[t]).ravel()))) for t in range(count))
    # the oracle on the smallest, the median and the largest instances
    order = sorted(range(count), key=lambda t: probs[t].F.shape[0])
    picks = sorted(set([order[0], order[count // 2], order[-1]]))
    pool = spawn_pool(len(picks))
    tasks = [(probs[t].tag, probs[t], "f64", wj[t].cpu().numpy(), yaj[t][:dps[t].m].cpu().numpy(),
              ydj[t].cpu().numpy()) for t in picks]
    checks = pool.map(_oracle_check_one, tasks)
    pool.close()
    pool.join()
    mj, mp = statistics.mean(ms_joint), statistics.mean(ms_plain)
    line = {"metric": "joint primal prox vs plain split (single-period, FP64): solves/s", "unit": "solves/s",
            "value": ok_j / (mj / 1e3), "plain_value": ok_p / (mp / 1e3), "higher_is_better": True,
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{count} single-period instances of the batch workload (every {step}th, "
                                   f"n {min(int(p.F.shape[0]) for p in probs)}-{max(int(p.F.shape[0]) for p in probs)}), "
                                   f"tol {args.tol}, joint: one CTA per instance; plain: ff_solve_batch, "
                                   "default schedule"},
            "joint": {"solved": ok_j, "ms_per_call": mj, "iterations_mean": float(it_j.mean()),
                      "iterations_median": float(np.median(it_j)),
                      "mu_rounds_per_iteration": float(np.mean([i["threshold_rounds"] / max(1, i["iterations"])
                                                                for i in jinfo])),
                      "instance_seconds_mean": float(np.mean([i["seconds"] for i in jinfo]))},
            "plain": {"solved": ok_p, "ms_per_call": mp, "iterations_mean": float(it_p.mean()),
                      "iterations_median": float(np.median(it_p)),
                      "instance_seconds_mean": float(np.mean([i["seconds"] for i in pinfo]))},
            "iterations_ratio_median": float(np.median(it_j / np.maximum(it_p, 1))),
            "max_abs_w_joint_minus_plain": diff, "oracle_check": checks,
            "gpu_launches": steps * (1 + plain.solver_launches())}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.workload == "risk":
        return run_risk(args)
    if args.workload == "joint":
        return run_joint(args)
    if args.workload == "paper_grid":
        return run_paper_grid(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
