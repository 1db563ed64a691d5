#!/usr/bin/env python
"""Benchmark: randomized PSD projections per second at n = 20000.

Workload (one "step"): one Algorithm 1 projection (the paper's Alg. 2 with the
range finder of Alg. 1) and one Algorithm 2 projection (the paper's Alg. 3
with alpha from Alg. 5, N = 10) of the same synthetic FP32 symmetric matrix,
n = 20000, k = 100, p = 10 (sketch width 110), q = 1, full P = W W^T written.
A step therefore runs every step of the path: Omega, the sketch and power
passes, CholeskyQR2, the core pass, the l x l eigensolve, the factor, the
reconstruction and the alpha estimate.

Matrix recipe: A = U diag(lam) U^T, U = 4 Householder reflectors, 200
eigenvalues decaying geometrically 100 -> 0.1, 300 uniform in [-5, -0.1], the
rest N(0, 0.01^2), formed in FP64 and rounded to FP32 (synth_inputs.py).
A (1.6 GB) is larger than L2, so no flush is needed between steps.

`value` = projections / s over all ranks (N > 1: independent replicas, one
per GPU, no collective on the data path), with the 2K projections of the K
steps spread over S = 4 independent contexts and CUDA streams (every stream
gets both algorithms; timed until all streams finish; --streams sets S).
`sequential` gives the same steps on one stream, and latency, stage times and
rooflines come from it.  Extra keys: roofline of the
dominant kernel, cpu_baseline (the FP64 oracle on host cores), e2e (the
host-buffer C-ABI call with copies inside the timed region), clocks, kernel
launches, per-algorithm latency p50/p99, per-stage times and accuracy against
the oracle and the exact projection.

`--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, K_DEFAULT, P_DEFAULT, Q_DEFAULT, SEED = 20000, 100, 10, 1, 1
STAGES = ["apass", "gemv", "orth", "core", "eig", "factor", "syrk", "other", "pack"]
PREC_NAMES = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x3": 3}
DTYPE_NAMES = {"fp32": "f32", "tf32": "tf32", "bf16": "bf16", "bf16x3": "bf16x3"}


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time from each rank's own: the largest x over all ranks
    (rank-local x when there is one rank).  Backend-agnostic: NCCL with a CUDA
    device on the GPUs, gloo with the CPU in the multi-process tests."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput with every rank doing the same units (weak
    scaling, independent replicas): all ranks' units over the slowest rank."""
    return units_per_rank * world / max_seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--p", type=int, default=P_DEFAULT)
    ap.add_argument("--q", type=int, default=Q_DEFAULT)
    ap.add_argument("--prec", default="auto", choices=["auto", *PREC_NAMES])
    ap.add_argument("--syrk-prec", default="auto", choices=["auto", "fp32", "bf16x3"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-FP32 comparison")
    ap.add_argument("--no-forms", action="store_true", help="skip the TF32 / split-BF16 comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload in the headline run")
    ap.add_argument("--no-serve", action="store_true", help="skip the served workload in the headline run")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "batched", "serve", "profile", "batched-profile"],
                    help="batched: 512 matrices, sides log-uniform in [64, 2048], through psdproj_batched; "
                         "serve: Poisson arrivals through psdproj_server; profile: the small case the ncu "
                         "summaries under profiles/ are captured on (three Alg. 2 projections, BF16 form, "
                         "split-BF16 SYRK, side --n)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="offered requests per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=48, help="distinct matrices the requests draw from")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--streams", type=int, default=4,
                    help="independent contexts / CUDA streams the projections of the headline run on")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# the oracle baseline (host cores)
# --------------------------------------------------------------------------
def oracle_sample(A64_or_none, n, k, p, q, Vr=None, lam=None):
    """One FP64 oracle Algorithm 1 projection; returns (seconds, W)."""
    import numpy as np
    import oracle
    import synth_inputs as si
    if A64_or_none is None:
        A64_or_none = si.form_A_numpy(Vr, lam).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    out = oracle.alg1(A64_or_none, k, p, q, SEED)
    return time.perf_counter() - t0, out["W"]


def oracle_step(A64, k, p, q):
    """One step of the headline workload in the FP64 oracle: an Algorithm 1
    and an Algorithm 2 projection (N = 10) of A64.  Returns (seconds, W of
    Algorithm 1, W of Algorithm 2)."""
    import oracle
    t0 = time.perf_counter()
    o1 = oracle.alg1(A64, k, p, q, SEED)
    o2 = oracle.alg2(A64, k, p, q, SEED, N=10)
    return time.perf_counter() - t0, o1["W"], o2["W_red"]


def oracle_single_core(n, k, p, q):
    """The oracle on ONE host core: one Algorithm 1 projection of the decay
    recipe at side n, in a child process started with OMP_NUM_THREADS=1 (the
    oracle's OpenMP regions then run on one thread).  Returns seconds or None."""
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "import numpy as np, oracle, synth_inputs as si\n"
            "Vr, lam = si.make_problem('decay', %d)\n"
            "A = si.form_A_numpy(Vr, lam).astype(np.float32).astype(np.float64)\n"
            "oracle.build(); t0 = time.perf_counter(); oracle.alg1(A, %d, %d, %d, %d)\n"
            "print(time.perf_counter() - t0)\n") % (ROOT, n, k, p, q, SEED)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return float(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, rank 0 only, at
    the headline configuration itself (n, k, p, q of the run, both
    algorithms, no scaling).  One step (one Algorithm 1 and one Algorithm 2
    projection, about 15-25 s on 16 cores at n = 20000) is timed whatever
    --steps asks for, so that the arm ends within a minute; no warm-up (the
    oracle keeps no state between calls)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import synth_inputs as si
    Vr, lam = si.make_problem("decay", args.n)
    A64 = si.form_A_numpy(Vr, lam).astype(np.float32).astype(np.float64)
    t_step, _, _ = oracle_step(A64, args.k, args.p, args.q)
    value = 2.0 / t_step
    sample = (f"one step of the headline workload in the FP64 oracle: an Algorithm 1 and an Algorithm 2 "
              f"(N = 10) projection at n={args.n}, k={args.k}, p={args.p}, q={args.q}, {t_step:.1f} s; "
              f"one step timed (requested {args.steps}), no warm-up")
    line = {
        "metric": f"PSD projections/s at n={args.n}", "value": value, "unit": "projections/s",
        "n_gpus": args.gpus, "steps": 1, "warmup": 0, "steps_requested": args.steps,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": workload_config(args, "fp64-oracle", "n/a"),
        "cpu_baseline": {"value": value, "unit": "projections/s", "cores": cores_used(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "projections/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, prec, syrk_prec):
    return {"workload": (f"randomized PSD projection, Alg. 1 + Alg. 2 per step, n={args.n}, "
                         f"k={args.k}, p={args.p}, q={args.q}, N=10, full P"),
            "n": args.n, "k": args.k, "p": args.p, "q": args.q, "N": 10,
            "prec": prec, "syrk_prec": syrk_prec,
            "l2": "inputs larger than L2 (A = %.2f GB)" % (4.0 * args.n * args.n / 1e9),
            "parallelism": f"replicas{args.gpus}"}


def source_sha(paths):
    h = hashlib.sha256()
    for pth in paths:
        with open(os.path.join(ROOT, pth), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_file: str, n: int, kernel: str):
    """DRAM traffic per launch (bytes) recorded in profiles/traffic.txt for
    `kernel` at size n, if it was taken on the current source of the kernel's
    file (else None).  Lines: file sha16 n kernel bytes; '#' starts a comment."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = source_sha([kernel_file])
    for ln in open(path):
        parts = ln.split("#")[0].split()
        if (len(parts) >= 5 and parts[0] == kernel_file and parts[1] == sha and int(parts[2]) == n
                and parts[3] == kernel):
            return float(parts[4])
    return None


def run_batched(args, emit=True):
    """The many-small-matrices workload: a batch of independent projections
    (batch recipe: sides log-uniform in [64, 2048], k = min(n/8, 64), p = 8,
    q = 1, the two algorithms alternating) through one psdproj_batched call per
    step, timed with CUDA events on the context's stream; the same batch with
    1, 4, 8 and 16 helper streams, replayed from a CUDA graph, and grouped
    (psdproj_batched_grouped)."""
    import numpy as np
    import torch
    import paper_2410_19208_gb300 as ps
    import synth_inputs as si
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = args.prec if args.prec != "auto" else "bf16"
    syrk_prec = args.syrk_prec if args.syrk_prec != "auto" else ("fp32" if prec == "fp32" else "bf16x3")
    opts = ps.make_opts(prec=PREC_NAMES[prec], syrk_prec=PREC_NAMES[syrk_prec])
    sizes = [int(x) for x in si.log_uniform_sizes(args.batch_count, 64, 2048, seed=7)]
    probs, nbytes = [], 0
    for i, n in enumerate(sizes):
        Vr, lam = si.make_problem("batch", n, seed_u=1000 + i, seed_lam=5000 + i)
        A = si.form_A_torch(Vr, lam, dev)
        P = torch.empty(n, n, device=dev)
        probs.append(dict(A=A, k=max(2, min(n // 8, 64)), p=8, q=1, seed=SEED + i, algorithm=1 + (i % 2), P=P))
        nbytes += 4 * n * n
    stream = torch.cuda.current_stream(dev)
    ctx = ps.Context(0, stream)
    per = {}
    for S in (1, 4, 8, 16):
        ctx.set_batch_streams(S)
        for _ in range(max(args.warmup, 3)):
            ctx.batched(probs, opts=opts)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the batched warm-up")
        steps = max(1, args.steps // 4)
        sampler = ClockSampler(0)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ps.lib().psdproj_kernel_launches()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ctx.batched(probs, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = int(ps.lib().psdproj_kernel_launches() - l0)
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the batched run")
        per[S] = {"value": len(probs) * steps / (ms / 1e3), "ms_per_step": ms / steps,
                  "gpu_launches": launches, "clocks": clocks}
    # the same batch recorded once into a CUDA graph and replayed
    # (psdproj_batched_graph), with the stream counts that pay most
    for S in (16, 32):
        ctx.set_batch_streams(S)
        for _ in range(max(args.warmup, 3)):
            ctx.batched(probs, opts=opts, graph=True)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the graph batched warm-up")
        steps = max(2, args.steps // 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ps.lib().psdproj_kernel_launches()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ctx.batched(probs, opts=opts, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the graph batched run")
        per[f"graph{S}"] = {"value": len(probs) * steps / (ms / 1e3), "ms_per_step": ms / steps,
                            "gpu_launches": int(ps.lib().psdproj_kernel_launches() - l0), "clocks": None}
    # the grouped batch (psdproj_batched_grouped): the small steps of all
    # problems as one launch per step, the streaming steps on the lanes, the
    # whole batch recorded once into a CUDA graph and replayed
    for S in (16, 32, 64):
        ctx.set_batch_streams(S)
        for _ in range(max(args.warmup, 3)):
            ctx.batched(probs, opts=opts, grouped=True)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the grouped batched warm-up")
        steps = max(2, args.steps // 4)
        sampler = ClockSampler(0)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ps.lib().psdproj_kernel_launches()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ctx.batched(probs, opts=opts, grouped=True)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        if ctx.sync_status() != 0:
            raise SystemExit("device status set during the grouped batched run")
        per[f"grouped{S}"] = {"value": len(probs) * steps / (ms / 1e3), "ms_per_step": ms / steps,
                              "gpu_launches": int(ps.lib().psdproj_kernel_launches() - l0), "clocks": clocks}
    # the autotuner (psdproj_tune_batch) picks a lane count for this batch's
    # bucket from graph replays; the choice and its time are reported beside
    # the fixed counts
    tuned_S, tuned_ms = ctx.tune_batch(probs, opts=opts, reps=3)
    if ctx.sync_status() != 0:
        raise SystemExit("device status set during the batch autotuning")
    best = max(per, key=lambda S: per[S]["value"])
    # HBM roofline of the batch: the algorithmic bytes of every projection
    # (BF16 form: the pack reads A's upper triangle and writes the image, 6 B
    # per entry; 2q + 2 passes over the image, 2 B per entry; P written,
    # 4 n^2; Alg. 3 adds 2(N + 1) power-iteration products over the image)
    peaks, peak_kind = measured_peaks()
    per_entry = {"bf16": (6.0, 2.0, 2.0), "bf16x3": (8.0, 4.0, 4.0), "tf32": (8.0, 4.0, 4.0),
                 "fp32": (0.0, 4.0, 4.0)}[prec]
    batch_bytes = 0.0
    for d in probs:
        nn = d["A"].shape[0]
        up = nn * (nn + 1) / 2.0
        batch_bytes += (per_entry[0] + (2 * d["q"] + 2) * per_entry[1]) * up + 4.0 * nn * nn
        if d["algorithm"] == 2:
            batch_bytes += 2 * (10 + 1) * per_entry[2] * up
    ach = batch_bytes / (per[best]["ms_per_step"] / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_batch": batch_bytes,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    line = {"metric": "batched PSD projections/s (512 matrices, sides log-uniform 64..2048)",
            "value": per[best]["value"], "unit": "projections/s", "n_gpus": 1, "steps": max(1, args.steps // 4),
            "warmup": max(args.warmup, 3), "ms_per_step": per[best]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[prec], "data": "synthetic",
            "config": {"workload": f"psdproj_batched (graph: psdproj_batched_graph; grouped: "
                                   f"psdproj_batched_grouped), {len(probs)} problems per "
                                   "step, batch recipe, k = min(n/8, 64), p = 8, q = 1, Alg. 1 / Alg. 2 alternating",
                       "helper_streams": best, "batch_bytes_A": nbytes,
                       "autotuned": {"helper_streams": tuned_S, "ms_per_batch": tuned_ms,
                                     "value": len(probs) / (tuned_ms / 1e3) if tuned_ms > 0 else None},
                       "l2": "inputs larger than L2 (the batch's A is %.2f GB)" % (nbytes / 1e9)},
            "by_streams": {str(S): per[S] for S in per}, "roofline": roof,
            "gpu_launches": per[best]["gpu_launches"], "clocks": per[best]["clocks"] or per[1]["clocks"]}
    if emit:
        print(json.dumps(line))
    ctx.close()
    return line


def run_serve(args, emit=True):
    """The served workload: requests arrive as a Poisson process (rate
    --serve-rate, --serve-seconds long), each a matrix of side log-uniform in
    [256, 8192] (batch recipe; drawn from a pool of --serve-pool matrices
    generated on the device beforehand), k in {16, 32, 64, 128}, p = 8,
    q in {0, 1} and a random algorithm, submitted to a psdproj_server with a
    120 GB admission budget.  Latency runs from submit to completion (the
    server's clock); throughput = completed requests / (last completion -
    first submit)."""
    import numpy as np
    import torch
    import paper_2410_19208_gb300 as ps
    import synth_inputs as si
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = args.prec if args.prec != "auto" else "bf16"
    syrk_prec = args.syrk_prec if args.syrk_prec != "auto" else ("fp32" if prec == "fp32" else "bf16x3")
    opts = ps.make_opts(prec=PREC_NAMES[prec], syrk_prec=PREC_NAMES[syrk_prec])
    rng = np.random.default_rng(SEED)
    sizes = [int(x) for x in si.log_uniform_sizes(args.serve_pool, 256, 8192, seed=13)]
    pool = []
    for i, n in enumerate(sizes):
        Vr, lam = si.make_problem("batch", n, seed_u=3000 + i, seed_lam=7000 + i)
        pool.append(si.form_A_torch(Vr, lam, dev))
    free_P = [[] for _ in sizes]
    torch.cuda.synchronize()
    srv = ps.Server(0, workers=args.serve_workers, admit_bytes=120 * 10 ** 9, opts=opts)

    def draw(i):
        n = sizes[i]
        k = int(rng.choice([16, 32, 64, 128]))
        return dict(k=min(k, n - 8), q=int(rng.integers(0, 2)), alg=int(rng.integers(1, 3)),
                    seed=int(rng.integers(1, 1 << 62)))

    # warm-up: one request per pool matrix (workspaces and images sized)
    t_w = []
    for i in range(len(sizes)):
        P = torch.empty(sizes[i], sizes[i], device=dev)
        d = draw(i)
        t_w.append((srv.submit(pool[i], d["k"], 8, d["q"], d["seed"], algorithm=d["alg"], P=P), i, P))
    for t, i, P in t_w:
        st_ = srv.wait(t, 600.0)
        if st_ is None or st_[0] != 0:
            raise SystemExit(f"warm-up request failed: {st_}")
        free_P[i].append(P)

    l0 = ps.lib().psdproj_kernel_launches()
    inflight, params, failures = {}, {}, []
    lat, statuses = [], []
    n_req = int(args.serve_rate * args.serve_seconds)
    gaps = rng.exponential(1.0 / args.serve_rate, n_req)
    arrivals = np.cumsum(gaps)
    pick = rng.integers(0, len(sizes), n_req)
    late = 0

    def reap(block=False):
        for t in list(inflight):
            r = srv.wait(t, 600.0 if block else 0.0)
            if r is None:
                continue
            i, P = inflight.pop(t)
            free_P[i].append(P)
            statuses.append(r[0])
            lat.append(r[1])
            if r[0] != 0 and len(failures) < 8:
                failures.append({"status": ps.STATUS.get(r[0], r[0]), "n,pool,k,q,alg,seed": params[t]})
            params.pop(t, None)

    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    for j in range(n_req):
        target = t0 + arrivals[j]
        while time.perf_counter() < target:
            pass
        if time.perf_counter() - target > 0.005:
            late += 1
        i = int(pick[j])
        if not free_P[i]:
            reap()
        P = free_P[i].pop() if free_P[i] else torch.empty(sizes[i], sizes[i], device=dev)
        d = draw(i)
        t = srv.submit(pool[i], d["k"], 8, d["q"], d["seed"], algorithm=d["alg"], P=P)
        inflight[t] = (i, P)
        params[t] = (sizes[i], i, d["k"], d["q"], d["alg"], d["seed"])
        if j % 16 == 0:
            reap()
    reap(block=True)
    t1 = time.perf_counter()
    clocks = sampler.stop()
    st = srv.stats()
    launches = int(ps.lib().psdproj_kernel_launches() - l0)
    srv.close()
    lat_s = sorted(lat)

    def pq(q_):
        return lat_s[min(len(lat_s) - 1, int(round(q_ * (len(lat_s) - 1))))]

    line = {"metric": "served PSD projections/s (Poisson arrivals, sides log-uniform 256..8192)",
            "value": len(lat) / (t1 - t0), "unit": "requests/s", "n_gpus": 1, "steps": n_req, "warmup": len(sizes),
            "ms_per_step": 1e3 * (t1 - t0) / max(1, len(lat)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAMES[prec], "data": "synthetic",
            "config": {"workload": f"psdproj_server, {args.serve_workers} workers, offered {args.serve_rate:g} req/s "
                                   f"for {args.serve_seconds:g} s, k in {{16,32,64,128}}, p = 8, q in {{0,1}}, "
                                   "random algorithm, 120 GB admission budget",
                       "pool_matrices": len(sizes), "mean_n2": float(np.mean(np.square(sizes)))},
            "offered_rate": args.serve_rate, "requests": n_req, "completed": len(lat),
            "failed": int(sum(1 for x in statuses if x != 0)), "failures": failures,
            "arrivals_late_over_5ms": late,
            "latency_ms": {"p50": pq(0.5), "p90": pq(0.9), "p99": pq(0.99), "max": lat_s[-1]},
            "server": st, "gpu_launches": launches, "clocks": clocks}
    if emit:
        print(json.dumps(line))
    return line


def run_profile_case(args):
    """The ncu capture workload: three Algorithm 2 projections (BF16 form,
    split-BF16 SYRK) of the decay recipe at side args.n, each launching
    pack_upper_bf16_kernel once, sym_pass_bf16_kernel four times,
    sym_gemv_tiles_kernel 22 times and syrk_bf16x3_kernel once."""
    import torch
    import paper_2410_19208_gb300 as ps
    import synth_inputs as si
    n, k, p, q = args.n, args.k, args.p, args.q
    Vr, lam = si.make_problem("decay", n)
    A = si.form_A_torch(Vr, lam, "cuda")
    ctx = ps.Context(0)
    P = torch.empty(n, n, device="cuda")
    W = ps.tall_empty(n, k + p)
    opts = ps.make_opts(prec=ps.PREC_BF16, syrk_prec=ps.PREC_BF16X3)
    for _ in range(3):
        ctx.alg2(A, k, p, q, SEED, P=P, W=W, opts=opts)
    st = ctx.sync_status()
    if st != 0:
        raise SystemExit(f"device status {ps.STATUS.get(st)}")
    print(json.dumps({"workload": "profile", "n": n, "status": "ok"}))
    ctx.close()


def run_batched_profile_case(args):
    """A case for ncu: the 512-matrix batch recipe (BF16 form, split-BF16
    SYRK) through psdproj_batched_grouped, recorded and run once, then
    replayed once; no timing."""
    import torch
    import paper_2410_19208_gb300 as ps
    import synth_inputs as si
    dev = torch.device("cuda", 0)
    sizes = [int(x) for x in si.log_uniform_sizes(args.batch_count, 64, 2048, seed=7)]
    probs = []
    for i, n in enumerate(sizes):
        Vr, lam = si.make_problem("batch", n, seed_u=1000 + i, seed_lam=5000 + i)
        probs.append(dict(A=si.form_A_torch(Vr, lam, dev), k=max(2, min(n // 8, 64)), p=8, q=1, seed=SEED + i,
                          algorithm=1 + (i % 2), P=torch.empty(n, n, device=dev)))
    opts = ps.make_opts(prec=ps.PREC_BF16, syrk_prec=ps.PREC_BF16X3)
    ctx = ps.Context(0, torch.cuda.current_stream(dev))
    ctx.set_batch_streams(32)
    for _ in range(2):
        ctx.batched(probs, opts=opts, grouped=True)
    st = ctx.sync_status()
    if st != 0:
        raise SystemExit(f"device status {ps.STATUS.get(st)}")
    print(json.dumps({"workload": "batched-profile", "problems": len(probs), "status": "ok"}))
    ctx.close()


def main():
    args = parse()
    if args.workload == "profile":
        run_profile_case(args)
        return
    if args.workload == "batched-profile":
        run_batched_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2410_19208_gb300 as ps
    import synth_inputs as si

    prec = args.prec if args.prec != "auto" else "bf16"
    syrk_prec = args.syrk_prec if args.syrk_prec != "auto" else ("fp32" if prec == "fp32" else "bf16x3")
    n, k, p, q = args.n, args.k, args.p, args.q
    m = k + p
    Vr, lam = si.make_problem("decay", n)
    A = si.form_A_torch(Vr, lam, dev)
    stream = torch.cuda.current_stream(dev)
    ctx = ps.Context(local, stream)
    P = torch.empty(n, n, device=dev)
    W = ps.tall_empty(n, m, dev)
    rank_t = torch.zeros(1, dtype=torch.int32, device=dev)
    alpha_t = torch.zeros(1, dtype=torch.float64, device=dev)
    # further independent contexts, each on its own stream: the headline
    # spreads the projections of the K steps over all of them
    S = max(1, args.streams)
    lanes = [(ctx, stream, P, W, rank_t, alpha_t)]
    for _ in range(S - 1):
        st_ = torch.cuda.Stream(dev)
        lanes.append((ps.Context(local, st_), st_, torch.empty(n, n, device=dev), ps.tall_empty(n, m, dev),
                      torch.zeros(1, dtype=torch.int32, device=dev),
                      torch.zeros(1, dtype=torch.float64, device=dev)))
    ctx2 = lanes[1][0] if S > 1 else ctx
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    def set_reserve(r):
        # SMs that every context's persistent grids leave to the other
        # contexts' single-block steps while the contexts run at once
        # (psdproj_set_reserved_sms; 1, the library default, for one stream)
        for ln in lanes:
            ln[0].set_reserved_sms(max(0, min(r, sm_count - 1)))
    import ctypes

    def pct(v, q_):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q_ * (len(v) - 1))))]

    def measure(prec_, syrk_, steps, sample_clocks, alpha_mode=0):
        opts = ps.make_opts(prec=PREC_NAMES[prec_], syrk_prec=PREC_NAMES[syrk_], alpha_mode=alpha_mode)

        def step(lat=None):
            if lat is not None:
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
            ctx.alg1(A, k, p, q, SEED, P=P, W=W, rank=rank_t, opts=opts)
            if lat is not None:
                e1.record(stream)
            ctx.alg2(A, k, p, q, SEED, alpha_out=alpha_t, P=P, W=W, rank=rank_t, opts=opts)
            if lat is not None:
                e2.record(stream)
                lat.append((e0, e1, e2))

        for _ in range(max(args.warmup, 3)):
            step()
        st = ctx.sync_status()
        if st != 0:
            raise SystemExit(f"device status {ps.STATUS.get(st)} during warm-up ({prec_})")
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.4)
        l0 = ps.lib().psdproj_kernel_launches()
        ps.lib().psdproj_timing_enable(ctx.h, 1)
        lat = []
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(steps):
            step(lat)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        launches = int(ps.lib().psdproj_kernel_launches() - l0)
        ms_k = (ctypes.c_double * len(STAGES))()
        cnt_k = (ctypes.c_int * len(STAGES))()
        ps.lib().psdproj_timing_read(ctx.h, ms_k, cnt_k, len(STAGES))
        ps.lib().psdproj_timing_enable(ctx.h, 0)
        st = ctx.sync_status()
        if st != 0:
            raise SystemExit(f"device status {ps.STATUS.get(st)} in the timed region ({prec_})")
        elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
        a1 = [x[0].elapsed_time(x[1]) for x in lat]
        a2 = [x[1].elapsed_time(x[2]) for x in lat]
        stages = {STAGES[i]: {"ms_total": ms_k[i], "launches": cnt_k[i],
                              "ms_avg": (ms_k[i] / cnt_k[i]) if cnt_k[i] else None} for i in range(len(STAGES))}
        # accuracy of this form against the exact projection (closed form)
        ctx.alg1(A, k, p, q, SEED, P=None, W=W, rank=rank_t,
                 opts=ps.make_opts(prec=PREC_NAMES[prec_], syrk_prec=PREC_NAMES[syrk_],
                                   out_mode=ps.OUT_FACTOR))
        W1 = W.cpu().numpy().astype(np.float64)
        ctx.alg2(A, k, p, q, SEED, alpha_out=alpha_t, P=None, W=W, rank=rank_t,
                 opts=ps.make_opts(prec=PREC_NAMES[prec_], syrk_prec=PREC_NAMES[syrk_],
                                   out_mode=ps.OUT_FACTOR, alpha_mode=alpha_mode))
        W2 = W.cpu().numpy().astype(np.float64)
        return dict(elapsed_ms=elapsed_ms, lat1=a1, lat2=a2, stages=stages, launches=launches,
                    clocks=clocks, W1=W1, W2=W2, opts=opts)

    def measure_concurrent(prec_, syrk_, steps, sample_clocks):
        """K steps (one Alg. 1 and one Alg. 2 projection each) spread over the S
        contexts: projection j (step j // 2) goes to stream (j + j // 2) mod S,
        so every stream gets both algorithms; timed from an event on the first
        stream before the first projection to the first stream after every
        stream's last one."""
        opts = ps.make_opts(prec=PREC_NAMES[prec_], syrk_prec=PREC_NAMES[syrk_])
        set_reserve(2 * S if S > 1 else 1)

        def run(count):
            ev = torch.cuda.Event()
            ev.record(stream)
            for ln in lanes[1:]:
                ln[1].wait_event(ev)
            for j in range(2 * count):
                c_, _, P_, W_, r_, a_ = lanes[(j + j // 2) % S]
                if j % 2 == 0:
                    c_.alg1(A, k, p, q, SEED, P=P_, W=W_, rank=r_, opts=opts)
                else:
                    c_.alg2(A, k, p, q, SEED, alpha_out=a_, P=P_, W=W_, rank=r_, opts=opts)
            for ln in lanes[1:]:
                ev2 = torch.cuda.Event()
                ev2.record(ln[1])
                stream.wait_event(ev2)

        run(max(args.warmup, 3))
        torch.cuda.synchronize(dev)
        for c_ in [ln[0] for ln in lanes]:
            st = c_.sync_status()
            if st != 0:
                raise SystemExit(f"device status {ps.STATUS.get(st)} during warm-up (concurrent)")
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.4)
        l0 = ps.lib().psdproj_kernel_launches()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        run(steps)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        launches = int(ps.lib().psdproj_kernel_launches() - l0)
        for c_ in [ln[0] for ln in lanes]:
            st = c_.sync_status()
            if st != 0:
                raise SystemExit(f"device status {ps.STATUS.get(st)} in the timed region (concurrent)")
        elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
        set_reserve(1)
        return dict(elapsed_ms=elapsed_ms, launches=launches, clocks=clocks)

    # relative Frobenius error against the exact projection X+ = U diag(lam+) U^T,
    # in Gram form through the reflectors (no n x n matrix):
    #   ||X+ - W W^T||^2 = sum lam+^2 - 2 sum_i lam+_i ||(U^T W)_i||^2 + ||W^T W||^2
    lam_p = np.maximum(lam, 0.0)
    xp = float(np.sqrt(np.sum(lam_p ** 2)))

    def err_exact(Wf):
        X = Wf.copy()
        for t in range(Vr.shape[0]):          # U^T = H_r ... H_1: apply H_1 first
            v = Vr[t]
            X -= np.outer(v, (2.0 / float(v @ v)) * (v @ X))
        G = Wf.T @ Wf
        d2 = float(np.sum(lam_p ** 2) - 2.0 * np.sum(lam_p * np.sum(X * X, axis=1)) + np.sum(G * G))
        return float(np.sqrt(max(d2, 0.0)) / xp)

    # sequential, one stream: per-projection latency, stage times, rooflines
    head = measure(prec, syrk_prec, args.steps, False)
    elapsed_ms = head["elapsed_ms"]
    stages = head["stages"]
    opts = head["opts"]
    seq_value = job_rate(2 * args.steps, world, elapsed_ms / 1e3)
    # headline: the same K steps with the two projections of a step on two streams
    conc = measure_concurrent(prec, syrk_prec, args.steps, True)
    value = job_rate(2 * args.steps, world, conc["elapsed_ms"] / 1e3)

    # ---- rooflines: the dominant kernel and the other HBM-bound ones -------
    # algorithmic bytes per launch: U(n) = n(n+1)/2
    # upper-triangle entries; the BF16 form reads 2 bytes per entry from its
    # image, the FP32 form 4 bytes from A.  Per-launch times come from the
    # context's CUDA-event stage timing over the timed region (events on the
    # launching stream), divided by the launches a stage holds.
    peaks, peak_kind = measured_peaks()
    upper_elems = n * (n + 1) // 2
    N_PI = 10
    steps_ = args.steps

    def per_launch(stage, launches_per_stage):
        st_ = stages[stage]
        if not st_["launches"]:
            return None
        return st_["ms_total"] / (st_["launches"] * launches_per_stage)

    def hbm_entry(name, kfile, kname, stage, lps, nbytes, flops=None):
        ms = per_launch(stage, lps)
        if ms is None:
            return None
        gbs = nbytes / (ms / 1e3) / 1e9
        e = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "frac": gbs / peaks["hbm_gbs"], "per_launch_ms": ms, "algorithmic_bytes_per_launch": nbytes,
             "launches_per_step": stages[stage]["launches"] * lps / steps_,
             "ms_per_step": stages[stage]["ms_total"] / steps_,
             "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
             "traffic": traffic_from_profile(kfile, n, kname)}
        if flops is not None:
            e["algorithmic_flops_per_launch"] = flops
            e["tensor_tflops"] = flops / (ms / 1e3) / 1e12
        return e

    if prec == "fp32":
        # FP32 FMA on the CUDA cores: 2 n^2 m algorithmic FLOPs per pass,
        # peak = 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock
        apass_ms = stages["apass"]["ms_avg"]
        flops = 2.0 * n * n * m
        achieved = flops / (apass_ms / 1e3) / 1e12
        peak = sm_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "kernel": "sym_pass_simt",
                "peak_source": f"derived: {sm_count} SMs x 128 FP32 FMA lanes x 2 x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz",
                "hbm_frac_of_" + peak_kind: (upper_elems * 4 / (apass_ms / 1e3) / 1e9) / peaks["hbm_gbs"],
                "per_launch_ms": apass_ms, "algorithmic_bytes_per_launch": upper_elems * 4.0,
                "algorithmic_flops_per_launch": flops,
                "traffic": traffic_from_profile("paper_2410_19208_gb300/csrc/sympass_simt.cu", n,
                                                "sym_pass_simt_kernel")}
        path = None
    else:
        GEMV_FP32 = ("sym_gemv (power iteration, FP32 A)", "paper_2410_19208_gb300/csrc/gemv.cu",
                     "sym_gemv_kernel", "gemv", 2 * (N_PI + 1), upper_elems * 4.0)
        SYRK = ("syrk_bf16x3 (tcgen05, P written)", "paper_2410_19208_gb300/csrc/syrk_tc.cu",
                "syrk_bf16x3_kernel", "syrk", 1, n * n * 4.0)
        TC = "paper_2410_19208_gb300/csrc/sympass_tc.cu"
        if prec == "bf16":
            rows = [("sym_gemv_tiles (power iteration on the BF16 image)", "paper_2410_19208_gb300/csrc/gemv.cu",
                     "sym_gemv_tiles_kernel", "gemv", 2 * (N_PI + 1), upper_elems * 2.0),
                    ("sym_pass_bf16 (tcgen05, BF16 image)", TC, "sym_pass_bf16_kernel", "apass", 1,
                     upper_elems * 2.0, 2.0 * n * n * m),
                    SYRK,
                    ("pack_upper_bf16 (A read, image written)", TC, "pack_upper_bf16_kernel", "pack", 1,
                     upper_elems * 6.0)]
        elif prec == "bf16x3":
            # three tensor-core passes per product (A_hi X_hi, A_hi X_lo, A_lo X_hi)
            rows = [GEMV_FP32,
                    ("sym_pass_bf16 x3 (split BF16: hi and lo images)", TC, "sym_pass_bf16_kernel", "apass", 3,
                     upper_elems * 2.0, 2.0 * n * n * m),
                    SYRK,
                    ("pack_upper_bf16 x2 (hi and lo images)", TC, "pack_upper_bf16_kernel", "pack", 2,
                     upper_elems * 6.0)]
        else:
            # TF32: the pass streams the full image (n^2 x 4 bytes); its
            # algorithmic bytes are the FP32 upper triangle's, U(n) x 4
            TF = "paper_2410_19208_gb300/csrc/sympass_tf32.cu"
            rows = [GEMV_FP32,
                    ("sym_pass_tf32 (tcgen05 kind::tf32, full TF32 image)", TF, "sym_pass_tf32_kernel", "apass", 1,
                     upper_elems * 4.0, 2.0 * n * n * m),
                    SYRK,
                    ("pack_full_tf32 (A upper read, full image written)", TF, "pack_full_tf32_kernel", "pack", 1,
                     upper_elems * 4.0 + n * n * 4.0)]
        cand = [hbm_entry(*r) for r in rows]
        cand = [c for c in cand if c is not None]
        dom = max(cand, key=lambda c: c["ms_per_step"])
        roof = dict(dom)
        roof["others"] = [c for c in cand if c is not dom]
        # whole step: every algorithmic HBM byte of both projections
        passes = 2 * q + 2
        # algorithmic bytes per upper-triangle entry of the form: (pack, pass, power product)
        per_entry = {"bf16": (6.0, 2.0, 2.0), "bf16x3": (8.0, 4.0, 4.0), "tf32": (8.0, 4.0, 4.0)}[prec]
        path_bytes = 2 * (per_entry[0] * upper_elems + passes * per_entry[1] * upper_elems + 4.0 * n * n) \
            + 2 * (N_PI + 1) * per_entry[2] * upper_elems
        step_ms = elapsed_ms / args.steps
        path = {"bytes_per_step": path_bytes, "achieved": path_bytes / (step_ms / 1e3) / 1e9,
                "unit": "GB/s", "peak": peaks["hbm_gbs"],
                "frac": path_bytes / (step_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                "note": "per projection: pack + (2q+2) passes over the image of A + the P write; "
                        "plus 2(N+1) power-iteration products for Alg. 3; the small steps "
                        "(orthonormalisation, eigensolver) move almost no HBM bytes"}

    line = {
        "metric": f"PSD projections/s at n={n}", "value": value, "unit": "projections/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": conc["elapsed_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAMES[prec], "data": "synthetic",
        "config": workload_config(args, prec, syrk_prec),
        "roofline": roof,
        "path_roofline": path,
        "latency_ms": {"alg1_p50": pct(head["lat1"], 0.5), "alg1_p99": pct(head["lat1"], 0.99),
                       "alg2_p50": pct(head["lat2"], 0.5), "alg2_p99": pct(head["lat2"], 0.99)},
        "sequential": {"value": seq_value, "unit": "projections/s", "ms_per_step": elapsed_ms / args.steps,
                       "note": "the same steps on one context and one stream, Alg. 1 then Alg. 2; "
                               "latency, stages and rooflines are from this run"},
        "concurrency": f"{S} contexts on {S} CUDA streams; the 2K projections of the K steps are spread "
                       "over them, every stream getting both algorithms; each context's persistent grids "
                       f"leave {min(2 * S, sm_count - 1) if S > 1 else 1} SMs free "
                       "(psdproj_set_reserved_sms)",
        "stages": stages, "gpu_launches": conc["launches"], "clocks": conc["clocks"],
        "error_vs_exact": {"alg1": err_exact(head["W1"]), "alg2": err_exact(head["W2"])},
    }
    if prec != "fp32" and not args.no_plain:
        # the plain FP32 form at the same (k, p, q, seed), timed both ways the
        # headline is: on one stream, and spread over the same S contexts
        ks = max(2, min(args.steps, 5))
        plain = measure("fp32", "fp32", ks, False)
        pv1 = 2 * ks * world / (plain["elapsed_ms"] / 1e3)
        pconc = measure_concurrent("fp32", "fp32", ks, False)
        pvS = 2 * ks * world / (pconc["elapsed_ms"] / 1e3)
        line["plain_fp32"] = {"value": pvS, "unit": "projections/s", "streams": S,
                              "ms_per_step": pconc["elapsed_ms"] / ks,
                              "one_stream": {"value": pv1, "ms_per_step": plain["elapsed_ms"] / ks},
                              "speedup_of_headline": value / pvS,
                              "speedup_one_stream": seq_value / pv1,
                              "note": f"speedup_of_headline: the headline form over plain FP32, both on {S} "
                                      "streams; speedup_one_stream: both on one stream",
                              "error_vs_exact": {"alg1": err_exact(plain["W1"]),
                                                 "alg2": err_exact(plain["W2"])}}
        Wg = plain["W1"]
    else:
        Wg = head["W1"]
    if prec == "bf16" and not args.no_forms:
        # the other tensor-core forms of the A-passes at the same (k, p, q,
        # seed): one-stream time per step and error against the exact projection
        forms = {}
        for fp in ("tf32", "bf16x3"):
            ks = max(2, min(args.steps, 3))
            r = measure(fp, syrk_prec, ks, False)
            forms[fp] = {"value": 2 * ks * world / (r["elapsed_ms"] / 1e3), "unit": "projections/s",
                         "ms_per_step": r["elapsed_ms"] / ks, "streams": 1,
                         "error_vs_exact": {"alg1": err_exact(r["W1"]), "alg2": err_exact(r["W2"])}}
        line["forms"] = forms
        # variant: Alg. 3 with alpha from the Ritz values of the unshifted
        # sketch (one extra pass over A instead of the 2(N+1) power-iteration
        # products), same form as the headline
        ks = max(2, min(args.steps, 3))
        r = measure(prec, syrk_prec, ks, False, alpha_mode=1)
        line["variant_alpha_ritz"] = {
            "value": 2 * ks * world / (r["elapsed_ms"] / 1e3), "unit": "projections/s",
            "ms_per_step": r["elapsed_ms"] / ks, "streams": 1,
            "alg2_ms_p50": pct(r["lat2"], 0.5), "alg2_ms_p50_min_eig": pct(head["lat2"], 0.5),
            "error_vs_exact": {"alg1": err_exact(r["W1"]), "alg2": err_exact(r["W2"])}}

    # ---- the batched and the served workloads (their own recipes) ----------
    if world == 1 and not args.no_batched:
        b = run_batched(args, emit=False)
        line["batched"] = {"value": b["value"], "unit": b["unit"], "ms_per_step": b["ms_per_step"],
                           "workload": b["config"]["workload"], "helper_streams": b["config"]["helper_streams"],
                           "by_streams": {k_: v_["value"] for k_, v_ in b["by_streams"].items()},
                           "roofline": b["roofline"], "gpu_launches": b["gpu_launches"], "clocks": b["clocks"]}
        torch.cuda.empty_cache()
    if world == 1 and not args.no_serve:
        v = run_serve(args, emit=False)
        line["served"] = {"value": v["value"], "unit": v["unit"], "workload": v["config"]["workload"],
                          "seconds": args.serve_seconds, "offered_rate": v["offered_rate"],
                          "requests": v["requests"], "completed": v["completed"], "failed": v["failed"],
                          "latency_ms": v["latency_ms"], "arrivals_late_over_5ms": v["arrivals_late_over_5ms"],
                          "clocks": v["clocks"]}
        torch.cuda.empty_cache()

    # ---- end to end through the host-buffer C-ABI call --------------------
    if not args.no_e2e:
        Ah = A.cpu().pin_memory()
        T = len(lanes)                      # one host thread per context
        Phs = [torch.empty(n, n, dtype=torch.float32).pin_memory() for _ in range(T)]
        for j in range(T):
            lanes[j][0].alg1_host(Ah, k, p, q, SEED, P=Phs[j], opts=opts)
        if dist:
            dist.barrier()
        steps_e2e = max(args.e2e_steps, 1)
        # 2 * steps_e2e projections (one Alg. 2 and one Alg. 3 per step), as
        # many per thread as divide evenly; thread j alternates the algorithms
        per = [0] * T
        for i in range(2 * steps_e2e):
            per[i % T] += 1

        def host_loop(j):
            c_ = lanes[j][0]
            for i in range(per[j]):
                if (i + j) % 2 == 0:
                    c_.alg1_host(Ah, k, p, q, SEED, P=Phs[j], opts=opts)
                else:
                    c_.alg2_host(Ah, k, p, q, SEED, P=Phs[j], opts=opts)

        # host threads (the C calls release the GIL), each on its own context
        # and stream, so that copies in both directions and the computation
        # of different projections overlap
        ths = [threading.Thread(target=host_loop, args=(j,)) for j in range(T)]
        set_reserve(2 * T if T > 1 else 1)
        t0 = time.perf_counter()
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        dt = time.perf_counter() - t0
        set_reserve(1)
        dt = max_over_ranks(dt, dist, dev)
        upper_bytes = 4 * (n * (n + 1) // 2)          # read over the host link from the pinned A
        line["e2e"] = {"value": job_rate(2 * steps_e2e, world, dt), "unit": "projections/s",
                       "h2d_bytes_per_step": 2 * upper_bytes, "d2h_bytes_per_step": 2 * (4 * n * n + 4 + 8),
                       "api": f"psdproj_alg1_host + psdproj_alg2_host from {T} host threads (one context "
                              "each), pinned host buffers; A's upper triangle in, the full P out",
                       "link": "NVLink-C2C measured at about 211 GB/s host-to-device and 193 GB/s "
                               "device-to-host: P's 1.6 GB out alone bounds it near 120 projections/s; "
                               "measured, the two directions overlap little (about 8.3 + 3.8 ms each)"}
        del Ah, Phs

    # ---- accuracy and the oracle baseline (rank 0, N = 1 only) -------------
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        A64 = A.cpu().numpy().astype(np.float64)
        del P, lanes
        torch.cuda.empty_cache()
        t_or, Wo, Wo2 = oracle_step(A64, k, p, q)
        del A64
        rel = lambda Wx, Wr: float(np.sqrt(max(oracle.factor_dist2(Wx, Wr), 0.0) / oracle.factor_norm2(Wr)))
        err_o, err_o2 = err_exact(Wo), err_exact(Wo2)
        line["accuracy_alg1"] = {
            "headline_rel_fro_vs_oracle": rel(head["W1"], Wo),
            "plain_fp32_rel_fro_vs_oracle": rel(Wg, Wo),
            "headline_rel_fro_vs_exact": err_exact(head["W1"]),
            "oracle_rel_fro_vs_exact": err_o,
            "headline_ratio_to_oracle_error": err_exact(head["W1"]) / err_o}
        line["accuracy_alg2"] = {
            "headline_rel_fro_vs_oracle": rel(head["W2"], Wo2),
            "headline_rel_fro_vs_exact": err_exact(head["W2"]),
            "oracle_rel_fro_vs_exact": err_o2,
            "headline_ratio_to_oracle_error": err_exact(head["W2"]) / err_o2}
        line["cpu_baseline"] = {"value": 2.0 / t_or, "unit": "projections/s", "cores": cores_used(),
                                "kind": "oracle",
                                "sample": f"one step of the workload in the FP64 oracle (an Algorithm 1 and an "
                                          f"Algorithm 2 projection at n={n}, k={k}, p={p}, q={q}), {t_or:.1f} s"}
        n1 = min(n, 4096)
        t1 = oracle_single_core(n1, k, p, q)
        if t1 is not None:
            line["cpu_baseline_single_core"] = {
                "value": 1.0 / t1, "unit": "projections/s", "cores": 1, "kind": "oracle",
                "sample": f"one FP64 oracle Algorithm 1 projection at n={n1} (k={k}, p={p}, q={q}) on one "
                          f"core (OMP_NUM_THREADS=1), {t1:.1f} s; a smaller side than the headline's so that "
                          "the sample stays bounded"}
    print(json.dumps(line), flush=True)
    ctx.close()
    for ln in (lanes[1:] if 'lanes' in locals() else []):
        ln[0].close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
