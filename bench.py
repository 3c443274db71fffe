#!/usr/bin/env python
"""Benchmark of the one-sided Jacobi hyperbolic SVD on GB300.

One step = one complete HSVD (all sweeps until the Eq. 2.3 test passes for
every pair, then the finalisation), inputs already in HBM.

Default (the metric: HSVD time and effective TFLOP/s at sigma rel-err <= 1e-12,
the new forms against plain FP64, one GB300): the split-precision form (BF16
slices on the tensor cores, FP64 rotations) on the 4096 x 4096 factor
G = Q1 diag(sigma) Q2 (Haar Q, sigma log-uniform on [1e-6, 1], 2048 random +1
in J, seed 3) is timed as ``value``; in the same run ``forms_vs_plain`` times
the plain FP64 method on the same factor, the batched form on 10,000 factors
against a loop of single solves, and the learned form on the graded 8192
factor (condition 1e8) against the plain FP64 method, each with its sigma
error against the stored oracle values.  Effective TFLOP/s =
S * 2 n^2 (4m + 2n) / time, S the plain run's sweeps on the same factor (the
same flop count for every form).  ``--workload``/``--form`` select a single
other configuration.

``--impl reference`` times the CPU oracle (plain FP64 C code, the disjoint
pairs of each modulus step on OpenMP threads) on the host cores instead, each
step a bounded sample of the same workload (stated in ``config.sample``).

Multi-GPU: independent factors per rank (replicas, weak scaling), no
collective on the data path; a barrier and max-over-ranks timing only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MAX_SWEEPS = 40
U64 = 2.0 ** -53
METRIC = "HSVD time & eff. TFLOP/s at sigma rel-err <= 1e-12: new forms vs plain FP64, 1 GB300"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel, from one ncu capture of this workload; an entry is removed when the
# kernel changes
PROFILED_TRAFFIC = {
    ("graded1024", "fp64", "k_update<64>"): (17.317e6, "profiles/kernels_graded1024_fp64.md"),
    ("graded1024", "fp64", "k_gram<32>"): (8.396e6, "profiles/kernels_graded1024_fp64.md"),
    ("haar4096", "bf16x8", "k_update_x"): (498.15e6, "profiles/kernels_haar4096_bf16x8.md"),
    ("haar4096", "bf16x8", "k_gram_x"): (151.58e6, "profiles/kernels_haar4096_bf16x8.md"),
    ("haar4096", "bf16x8", "k_solve_cross<128,8>"): (18.97e6, "profiles/kernels_haar4096_bf16x8.md"),
}
# FP64 DFMA peak derived from the unit counts and the maximum clock (no FP64
# figure in the measured peaks): 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz
FP64_PEAK = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_PEAK_SOURCE = "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived from units and clock)"
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
GOLDEN = os.path.join(GOLDEN_DIR, "graded1024_sigma.txt")

# name -> (n, generator description, default block width)
WORKLOADS = {
    "graded1024": (1024, "graded 1024x1024 G=B diag(10^(-6i/n)), J=diag(+1x512,-1x512)", 32),
    "haar4096": (4096, "4096x4096 G=Q1 diag(sigma) Q2, Haar Q, sigma log-uniform [1e-6,1], 2048 random +1 in J", 64),
    "haar1024": (1024, "1024x1024 G=Q1 diag(sigma) Q2, Haar Q, sigma log-uniform [1e-6,1], 512 random +1 in J", 64),
    "graded2048": (2048, "graded 2048x2048 G=B diag(10^(-6i/n)), J=diag(+1x1024,-1x1024)", 32),
    "graded8192": (8192, "graded 8192x8192 G=B diag(10^(-8i/n)) (condition 1e8), J=diag(+1x4096,-1x4096)", 64),
    "batch10k": (256, "10000 independent square N(0,1) factors, n uniform on [16,256], m=n, random p in [0,n] "
                      "+1 signs at random positions (seed 4)", 1),
}
DEFAULT_WORKLOAD, DEFAULT_FORM = "haar4096", "bf16x8"
BATCH_COUNT = 10000
# columns of the factor the reference arm's oracle sweeps per step
REFERENCE_COLUMNS = 2048


def make_input(name, seed_offset=0):
    from paper_1008_1371_gb300 import workloads

    n = WORKLOADS[name][0]
    if name == "graded8192":
        return workloads.graded(n, decades=8.0, seed=5 + seed_offset)
    if name.startswith("graded"):
        return workloads.graded(n, decades=6.0, seed=2 + seed_offset)
    return workloads.haar(n, seed=3 + seed_offset)


def flops_per_sweep(m, n):
    """Blocked-method work of one quasi-sweep: Gram 4mn^2, G update 4mn^2, V update 4n^3."""
    return 2.0 * n * n * (4.0 * m + 2.0 * n)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sweeps", type=int, default=0,
                    help="oracle sweeps timed for cpu_baseline (0: a complete solve within about 10 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--form", default=DEFAULT_FORM, choices=["fp64", "bf16x8", "learned", "learned-bf16x8"],
                    help="Gram/update arithmetic (FP64 FMA or BF16 slices on the tensor cores), optionally "
                         "with the learned skip network")
    ap.add_argument("--no-forms", action="store_true",
                    help="default configuration only: skip forms_vs_plain (the plain FP64, batched and learned "
                         "comparisons)")
    ap.add_argument("--loop-count", type=int, default=1000,
                    help="forms_vs_plain / batch10k: factors in the measured loop of single solves (an evenly "
                         "spread sample; 0 = the whole batch)")
    ap.add_argument("--tau", type=float, default=0.5, help="learned form: skip threshold on P(rotation)")
    ap.add_argument("--check", action="store_true",
                    help="split precision: also solve with FP64 products (untimed) and report the sigma "
                         "agreement and the invariants of Eq. 1.1")
    ap.add_argument("--count", type=int, default=BATCH_COUNT, help="batch10k: number of factors")
    ap.add_argument("--group-width", type=int, default=0, help="batch10k: 0 autotunes, else 256/512/1024")
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 512, 1024],
                    help="batch10k: threads a CTA of the persistent kernel (0: 1024)")
    ap.add_argument("--block", type=int, default=0, help="block width (0: the workload's)")
    ap.add_argument("--tstop", type=float, default=0.0,
                    help="tangent-threshold early stop (Sec. 2): 0 off, negative = the paper's T_eps = 2^-27; "
                         "the effective flop count then uses the plain run's sweeps")
    ap.add_argument("--schedule", default="auto", choices=["auto", "steps", "pairs"],
                    help="sweep schedule of the blocked method (auto: the library's choice, the pair schedule)")
    ap.add_argument("--tol", type=float, default=0.0,
                    help="eps of Eq. 2.3 (0: n 2^-53; the paper's own is 2^-52)")
    ap.add_argument("--probe-rates", action="store_true",
                    help="print the library GEMM rates of this GPU (cuBLAS FP64 and BF16, cuBLASLt INT8) and exit: "
                         "the evidence for the slice type of the split-precision form")
    return ap.parse_args()


def probe_rates(n=8192, reps=10):
    """Dense GEMM rates of the vendor libraries on this GPU (CUDA events, best
    of `reps` after warm-up): FP64 (torch.matmul, cuBLAS), BF16 (cuBLAS) and
    INT8 -> INT32 (torch._int_mm, cuBLASLt).  The split-precision form needs
    the fastest exact tensor-core product of small integers; these rates pick
    the slice type."""
    import torch

    dev = torch.device("cuda:0")

    def rate(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12, best

    out = {"n": n, "reps": reps}
    a = torch.randn(n, n, device=dev, dtype=torch.float64)
    b = torch.randn(n, n, device=dev, dtype=torch.float64)
    out["fp64_tflops"], out["fp64_ms"] = rate(lambda: a @ b)
    a = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    b = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    out["bf16_tflops"], out["bf16_ms"] = rate(lambda: a @ b)
    a = torch.randint(-64, 64, (n, n), device=dev, dtype=torch.int8)
    b = torch.randint(-64, 64, (n, n), device=dev, dtype=torch.int8).t().contiguous().t()
    out["int8_tops"], out["int8_ms"] = rate(lambda: torch._int_mm(a, b))
    print(json.dumps(out))
    return 0


def max_over_ranks(value, world, device=None):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile

        try:
            fd, self.path = tempfile.mkstemp(prefix="hsvd_clocks_%d_" % self.gpu, suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
            if getattr(self, "f", None) is not None:
                self.f.close()
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if os.path.basename(self.path).startswith("hsvd_clocks_"):
            os.remove(self.path)  # the temporary file of __enter__
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def golden_path(workload):
    return os.path.join(GOLDEN_DIR, "%s_sigma.txt" % workload)


def accuracy_vs_golden(G, J, sigma, path=GOLDEN):
    """sigma against the stored oracle values (tests/golden/make_golden.py),
    per sign group after sorting, when G has the bytes they were computed for.

    Gate (the metric's sigma rel-err <= 1e-12, with the per-value noise floor
    u kappa_j = u || |G| |v_j| ||_2 / sigma_j of FP64 itself): |d sigma_j| /
    sigma_j <= max(1e-12, 2 u kappa_j) -- the run and the oracle are two FP64
    computations, each within about its floor of the exact value; where twice
    the floor is below 1e-12 the metric's 1e-12 applies.  ``gate`` is "pass"
    or "fail"."""
    import hashlib

    if not os.path.exists(path):
        return {"note": "no stored oracle values (%s)" % os.path.basename(path)}
    with open(path) as f:
        head = [ln for ln in f.read().splitlines() if ln.startswith("#")]
    want = next((ln.split("sha256(G)=")[1].strip() for ln in head if "sha256(G)=" in ln), None)
    have = hashlib.sha256(np.ascontiguousarray(G, dtype="<f8").tobytes(order="F")).hexdigest()
    if want != have:
        return {"note": "stored oracle values belong to other bytes of G (libm/LAPACK rounding); not compared"}
    ref = np.loadtxt(path)
    worst, worst_tight, worst_ratio, n_loose = 0.0, 0.0, 0.0, 0
    for sg in (1, -1):
        idx = np.where(J == sg)[0]
        if idx.size == 0:
            continue
        o = np.argsort(ref[idx, 0])
        y, k = ref[idx, 0][o], ref[idx, 1][o]
        e = np.abs(np.sort(sigma[idx]) - y) / y
        worst = max(worst, float(e.max()))
        tight = 2.0 * k <= 1e-12
        n_loose += int((~tight).sum())
        if tight.any():
            worst_tight = max(worst_tight, float(e[tight].max()))
        worst_ratio = max(worst_ratio, float((e / np.maximum(1e-12, 2.0 * k)).max()))
    return {"sigma_max_rel_err": worst, "sigma_max_rel_err_where_2floor_below_1e-12": worst_tight,
            "values_held_to_2floor": n_loose, "worst_err_over_tolerance": worst_ratio,
            "oracle": head[0].lstrip("# ").split(",")[0] if head else "",
            "gate": "pass" if worst_ratio <= 1.0 else "fail",
            "gate_rule": "|d sigma_j|/sigma_j <= max(1e-12, 2 u kappa_j) per value, u kappa_j the stored floor"}


def check_against_fp64(api, G, J, sigma, U, V, tol, J_np):
    """sigma of a split-precision run against a plain FP64 run on the same GPU
    (per sign group, sorted), gated per value by max(1e-12, u kappa_j), and the
    invariants of Eq. 1.1 of the split-precision result."""
    import torch

    n = G.shape[1]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    r64 = api.hsvd_solve_ex(G, J, api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS, method=api.HSVD_METHOD_BLOCKED,
                                                block_w=64, sort=False))
    ev1.record()
    ev1.synchronize()
    plain_ms = ev0.elapsed_time(ev1)  # one run, graphs built inside: an upper bound
    kap = (2.0 ** -53 * torch.linalg.vector_norm(G.abs() @ r64.V.abs(), dim=0) / r64.sigma).cpu().numpy()
    sx, s64 = sigma.cpu().numpy(), r64.sigma.cpu().numpy()
    worst, worst_gate = 0.0, 0.0
    for sg in (1, -1):
        idx = np.where(J_np == sg)[0]
        o = np.argsort(s64[idx])
        e = np.abs(np.sort(sx[idx]) - s64[idx][o]) / s64[idx][o]
        worst = max(worst, float(e.max()))
        worst_gate = max(worst_gate, float((e / np.maximum(1e-12, kap[idx][o])).max()))
    eye = torch.eye(n, dtype=torch.float64, device=G.device)
    Jd = torch.diag(J.to(torch.float64))
    e1 = float((U.T @ U - eye).abs().max())
    e2 = float((V.T @ Jd @ V - Jd).abs().max()) / max(1.0, float(V.abs().max()) ** 2)
    res = torch.linalg.vector_norm(G @ V - U * sigma[None, :], dim=0) / (
        torch.linalg.matrix_norm(G) * torch.linalg.vector_norm(V, dim=0))
    return {"vs_plain_fp64_max_rel_sigma_diff": worst, "vs_plain_fp64_worst_over_floor_gate": worst_gate,
            "plain_fp64_sweeps": r64.sweeps, "plain_fp64_ms": plain_ms,
            "max_abs_UtU_minus_I": e1, "max_VtJV_minus_J_scaled": e2,
            "max_residual_GV_minus_U_sigma": float(res.max()),
            "gate": "two runs, each within its floor of the exact value: |d sigma|/sigma <= 2 max(1e-12, "
                    "u kappa_j) per value (worst_over_floor_gate <= 2); invariants <= 1e-12 n"}


def host_info():
    """The host the CPU baseline ran on: CPU model, logical cores, and the
    oracle's compiler flags."""
    import platform

    import oracle

    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" not in line:
                    continue
                key, val = line.split(":", 1)
                if key.strip().lower() in ("model name", "cpu part", "hardware"):
                    model = val.strip()
                    break
    except (OSError, UnicodeDecodeError):
        pass
    flags = " ".join(getattr(getattr(oracle, "oracle", None), "CFLAGS", []))
    return {"cpu": model, "machine": platform.machine(), "nproc": os.cpu_count(),
            "oracle_cflags": flags + " -fopenmp (if available)"}


def cpu_baseline(G, J, tol, sweeps, budget_s=10.0):
    """The oracle as it stands on the host's cores: its modulus-parallel mode
    (the disjoint pairs of each step on OpenMP threads) on the same factor.
    `sweeps` > 0 times that many sweeps; 0 times a complete solve when one
    sweep is cheap enough, else as many sweeps as fit in about `budget_s`
    seconds (one timed sweep decides)."""
    import oracle

    oracle.build()
    cores = oracle.set_threads(0)
    m, n = G.shape

    def run(k):
        t0 = time.perf_counter()
        r = oracle.hsvd(G, J, tol, k, order="modulus", want_u=False, want_v=False)
        return r, time.perf_counter() - t0

    if sweeps <= 0:
        r, dt = run(1)
        k = max(1, min(MAX_SWEEPS, int(budget_s / max(dt, 1e-9))))
        if k > 1:
            r, dt = run(k)
    else:
        r, dt = run(sweeps)
    per_sweep = dt / max(r["sweeps"], 1)
    what = "a complete solve (%d sweeps)" % r["sweeps"] if r["status"] == 0 else "%d sweep(s)" % r["sweeps"]
    return {"value": flops_per_sweep(m, n) / per_sweep / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "host": host_info(),
            "sample": "%s of the modulus-parallel FP64 oracle (%d OpenMP threads) on the same %dx%d factor, %.2f s "
                      "per sweep; effective rate per sweep with the blocked flop count 2n^2(4m+2n)"
                      % (what, cores, m, n, per_sweep)}


def pointwise_flops_per_sweep(m, n):
    """Pointwise work of one sweep (n^2/2 pairs): three dot products and the
    updates of two G columns and two W columns, (n^2/2)(12m + 6n)."""
    return 0.5 * n * n * (12.0 * m + 6.0 * n)


def oracle_batch_sample(oracle, facs, per_core=8):
    """A bounded, evenly spread sample of the batch solved completely by the
    row-cyclic oracle, the factors split across the host's cores (the oracle
    is reentrant and ctypes releases the interpreter lock during each call).
    Returns (effective flops, seconds, factors solved, threads, sample note)."""
    from concurrent.futures import ThreadPoolExecutor

    cores = os.cpu_count() or 1
    count = len(facs)
    nsample = min(count, per_core * cores)
    stride = max(1, count // nsample)
    idx = list(range(0, count, stride))[:nsample]

    def one(k):
        G, J = facs[k]
        r = oracle.hsvd(G, J, G.shape[1] * 2.0 ** -53, 30, want_u=False, want_v=False)
        return r["sweeps"] * pointwise_flops_per_sweep(*G.shape)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        f = sum(ex.map(one, idx))
    dt = time.perf_counter() - t0
    note = ("%d of %d factors (every %dth) solved completely by the row-cyclic FP64 oracle, split across %d host "
            "threads, %.1f s" % (len(idx), count, stride, cores, dt))
    return f, dt, len(idx), cores, note


def batched_setup(api, dev, count, seed):
    """The batch workload on the device: one buffer per array kind, the
    factors as column-major views into it."""
    import torch
    from paper_1008_1371_gb300 import workloads

    facs = workloads.batch(count, seed=seed)
    ms_ = [G.shape[0] for G, _ in facs]
    ns_ = [G.shape[1] for G, _ in facs]

    def packed(sizes, dtype):
        buf = torch.empty(sum(sizes), dtype=dtype, device=dev)
        out, o = [], 0
        for z in sizes:
            out.append(buf[o:o + z])
            o += z
        return buf, out

    gbuf, gv = packed([m * n for m, n in zip(ms_, ns_)], torch.float64)
    jbuf, jv = packed(ns_, torch.int8)
    gcat = np.concatenate([G.ravel(order="F") for G, _ in facs])
    gbuf.copy_(torch.from_numpy(gcat))
    jbuf.copy_(torch.from_numpy(np.concatenate([J for _, J in facs])))
    Gs = [g.view(n, m).t() for g, m, n in zip(gv, ms_, ns_)]
    sbuf, sig = packed(ns_, torch.float64)
    ubuf, uv = packed([m * n for m, n in zip(ms_, ns_)], torch.float64)
    vbuf, vv = packed([n * n for n in ns_], torch.float64)
    Us = [u.view(n, m).t() for u, m, n in zip(uv, ms_, ns_)]
    Vs = [v.view(n, n).t() for v, n in zip(vv, ns_)]
    keep = (gbuf, jbuf, sbuf, ubuf, vbuf)
    return dict(facs=facs, ms=ms_, ns=ns_, G=Gs, J=jv, sigma=sig, U=Us, V=Vs, keep=keep)


def measure_batched(api, dev, count, steps, warmup, group_width, loop_count, rank=0, world=1, with_e2e=True,
                    with_cpu=True, clocks=False, cta_threads=0):
    """The batched form on `count` factors: `warmup` + `steps` timed
    persistent launches (CUDA events, L2 flushed between steps), a measured
    loop of single hsvd_solve calls on an evenly spread sample of
    `loop_count` factors (0: all), sampled factors against the CPU oracle,
    and optionally the end-to-end time with host arrays and the oracle's
    rate on the host cores."""
    import torch

    B = batched_setup(api, dev, count, 4 + rank)
    facs, ms_, ns_ = B["facs"], B["ms"], B["ns"]
    opts = api.make_batch_opts(max_sweeps=30, group_width=group_width, cta_threads=cta_threads)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve():
        return api.hsvd_solve_batched(B["G"], B["J"], opts, out=(B["sigma"], B["U"], B["V"]), stream=stream)

    for _ in range(warmup):
        r = solve()
    torch.cuda.synchronize()
    step_ms, infos = [], []
    clk = ClockSampler(dev.index or 0) if clocks else None
    if clk:
        clk.__enter__()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(r.info)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if clk:
        clk.__exit__()
    assert r.rc == api.HSVD_OK, r.rc
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    eff = sum(sw * pointwise_flops_per_sweep(m, n) for sw, m, n in zip(r.sweeps, ms_, ns_))
    kern_ms = sum(i.ms_kernel for i in infos) / len(infos)
    out = {"ms": ms, "ms_median": statistics.median(step_ms), "eff_flops": eff, "kernel_ms": kern_ms,
           "launches": int(sum(i.kernel_launches for i in infos)), "info": r.info,
           "max_sweeps_run": int(r.info.max_sweeps_run), "clocks": clk.summary() if clk else None}

    # a loop of single solves (the library's default method per factor),
    # measured on the stated sample of the batch
    if rank == 0:
        nloop = count if loop_count <= 0 else min(count, loop_count)
        stride = max(1, count // nloop)
        idx = list(range(0, count, stride))[:nloop]
        one = api.hsvd_solve_ex(B["G"][idx[0]], B["J"][idx[0]], api.make_opts(max_sweeps=30),
                                out=(B["sigma"][idx[0]], B["U"][idx[0]], B["V"][idx[0]]), stream=stream)
        torch.cuda.synchronize()
        f_loop = 0.0
        t0 = time.perf_counter()
        for k in idx:
            one = api.hsvd_solve_ex(B["G"][k], B["J"][k], api.make_opts(max_sweeps=30),
                                    out=(B["sigma"][k], B["U"][k], B["V"][k]), stream=stream)
            f_loop += one.sweeps * pointwise_flops_per_sweep(ms_[k], ns_[k])
        torch.cuda.synchronize()
        t_loop = time.perf_counter() - t0
        scaled = t_loop * 1e3 * (count / len(idx))
        out["loop"] = {
            "factors": len(idx), "of": count, "ms_measured": t_loop * 1e3,
            "ms_whole_batch": t_loop * 1e3 if len(idx) == count else scaled,
            "whole_batch": "measured" if len(idx) == count else "measured sample x %d/%d" % (count, len(idx)),
            "tflops": f_loop / t_loop / 1e12, "speedup_of_batched": scaled / ms,
            "sample": "%d of %d factors (every %dth), one hsvd_solve call each (default method per factor), "
                      "timed back to back on the host clock" % (len(idx), count, stride)}
        # sampled factors against the CPU oracle (per sign group, sorted)
        import oracle

        oracle.build()
        rng = np.random.default_rng(0)
        worst, worst_ratio = 0.0, 0.0
        solve()  # the batched results again (the loop overwrote some)
        torch.cuda.synchronize()
        for k in sorted(rng.choice(count, min(6, count), replace=False).tolist()):
            G, J = facs[k]
            ref = oracle.hsvd(G, J, G.shape[1] * U64, 30, order="modulus", want_u=False, want_v=True)
            floor = U64 * np.linalg.norm(np.abs(G) @ np.abs(ref["V"]), axis=0) / ref["sigma"]
            s_k = B["sigma"][k].cpu().numpy()
            for sg in (1, -1):
                sel = np.where(J == sg)[0]
                if sel.size:
                    o = np.argsort(ref["sigma"][sel])
                    a, b, fl = np.sort(s_k[sel]), ref["sigma"][sel][o], floor[sel][o]
                    e = np.abs(a - b) / b
                    worst = max(worst, float(e.max()))
                    worst_ratio = max(worst_ratio, float(np.max(e / np.maximum(1e-12, 2.0 * fl))))
        out["accuracy"] = {"sampled_factors": min(6, count), "max_rel_sigma_err_vs_oracle": worst,
                           "worst_err_over_tolerance": worst_ratio,
                           "gate_rule": "|d sigma_j|/sigma_j <= max(1e-12, 2 u kappa_j), u kappa_j from the oracle's V",
                           "gate": "pass" if worst_ratio <= 1.0 else "fail"}

    if with_e2e:
        Gh = [torch.from_numpy(G).pin_memory() for G, _ in facs]
        Jh = [torch.from_numpy(J).pin_memory() for _, J in facs]
        api.hsvd_solve_batched(Gh, Jh, opts)
        ts = []
        for _ in range(max(3, steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.hsvd_solve_batched(Gh, Jh, opts)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(ts) / len(ts), world, dev)
        out["e2e"] = {"value": world * eff / e2e_s / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_s * 1e3,
                      "h2d_bytes_per_step": sum(m * n * 8 + n for m, n in zip(ms_, ns_)),
                      "d2h_bytes_per_step": sum(n * 8 + m * n * 8 + n * n * 8 for m, n in zip(ms_, ns_)),
                      "note": "host arrays (pinned), one copy per matrix and direction inside the call"}
    if with_cpu and rank == 0 and world == 1:
        import oracle

        oracle.build()
        f, dt, _, cores, note = oracle_batch_sample(oracle, facs)
        out["cpu"] = {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                      "host": host_info(), "sample": note}
    return out


def batched_roofline(res):
    fp64_peak = FP64_PEAK
    achieved = res["eff_flops"] / (res["kernel_ms"] * 1e-3) / 1e12
    info = res["info"]
    return {"kernel": "k_batched", "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": None, "peak_source": FP64_PEAK_SOURCE,
            "ms_kernel": res["kernel_ms"], "group_width_per_bucket": list(info.bucket_width),
            "resident_G_W_shared__G_shared__neither": list(info.resident)}


def run_batched(args):
    """The batched form on the 10,000-factor workload, against a measured loop
    of single solves."""
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1008_1371_gb300 import api, build_lib

    if local == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    count = args.count
    res = measure_batched(api, dev, count, args.steps, args.warmup, args.group_width, args.loop_count, rank, world,
                          with_e2e=not args.no_e2e, with_cpu=not args.no_cpu_baseline, clocks=True,
                          cta_threads=args.cta_threads)
    value = world * res["eff_flops"] / (res["ms"] * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": "HSVD effective TFLOP/s (batched form, sigma rel-err <= 1e-12)", "value": value,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch10k"][1].replace("10000", str(count)), "count": count,
                       "form": "batched", "group_width": args.group_width or "autotuned",
                       "cta_threads": args.cta_threads or 1024,
                       "method": "pointwise per factor, diagonal sorting", "tol": "n 2^-53 per factor",
                       "max_sweeps_run": res["max_sweeps_run"],
                       "l2": "flushed (256 MB write) between steps; inputs 2.6 GB > L2",
                       "parallelism": "replicas" if world > 1 else "single"},
            "ms_per_step_median": res["ms_median"], "accuracy": res.get("accuracy"),
            "gpu_launches": res["launches"], "roofline": batched_roofline(res),
            "loop_of_single_solves": res.get("loop"), "e2e": res.get("e2e"), "cpu_baseline": res.get("cpu"),
            "clocks": res["clocks"],
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def metric_name(form, workload=None):
    if workload == DEFAULT_WORKLOAD and form == DEFAULT_FORM:
        return METRIC
    names = {"fp64": "plain FP64", "bf16x8": "split-precision BF16x8 products",
             "learned": "learned skip network, FP64 products",
             "learned-bf16x8": "learned skip network, BF16x8 products"}
    return "HSVD effective TFLOP/s (%s, sigma rel-err <= 1e-12)" % names[form]


def train_skip_model(block, prec, log):
    """The learned form's network, trained on traces of the plain method on
    graded factors of other seeds (1024 x 1024, decades 4, 6, 8), by the
    library's own kernels; seeded, outside every timed region."""
    from paper_1008_1371_gb300 import learn, workloads

    t0 = time.perf_counter()
    train_set = [workloads.graded(1024, decades=d, seed=s) for d, s in ((6.0, 100), (4.0, 101), (8.0, 102),
                                                                         (6.0, 103))]
    X, y = learn.collect(train_set, block_w=block, precision=prec)
    params, losses = learn.train(X, y, steps=600, lr=3e-3, batch=4096, seed=0)
    log.update({"train_rows": int(X.shape[0]), "train_positive_fraction": float(y.mean()),
                "train_loss_first_last": [losses[0], losses[-1]], "train_s": time.perf_counter() - t0,
                "train_set": "graded 1024x1024, decades 6/4/8/6, seeds 100-103, plain blocked traces"})
    return params


def run_reference_batched(args, oracle):
    """The oracle on the batch workload: each step solves a bounded sample of
    the factors completely, split across the host's cores; rate in effective
    flops."""
    from paper_1008_1371_gb300 import workloads

    count = args.count
    facs = workloads.batch(count, seed=4)
    times, flops = [], []
    note, cores = "", 1
    for i in range(args.warmup + args.steps):
        f, dt, _, cores, note = oracle_batch_sample(oracle, facs)
        if i >= args.warmup:
            times.append(dt)
            flops.append(f)
    value = sum(flops) / sum(times) / 1e12
    per = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": "HSVD effective TFLOP/s (batched form, sigma rel-err <= 1e-12)",
        "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS["batch10k"][1].replace("10000", str(count)), "count": count,
                                        "method": "CPU oracle, pointwise per factor, row-cyclic order",
                                        "sample": note},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "host": host_info(),
                         "sample": note},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    if args.workload == "batch10k":
        return run_reference_batched(args, oracle)
    G, J = make_input(args.workload)
    m, n = G.shape
    tol = args.tol if args.tol > 0 else n * U64
    # a bounded sample per step: one oracle sweep over the whole factor up to
    # n = 2048 (about a second on 16 host cores), over its first 2048 columns
    # (all rows) beyond
    nc = min(n, REFERENCE_COLUMNS)
    Gs, Js = np.asfortranarray(G[:, :nc]), J[:nc]
    cores = oracle.set_threads(0)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.hsvd(Gs, Js, tol, 1, order="modulus", want_u=False, want_v=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    value = flops_per_sweep(m, nc) / per / 1e12
    sample = ("one sweep of the modulus-parallel CPU oracle per step over %s of the %dx%d factor (%dx%d), rate "
              "with the blocked flop count 2n^2(4m+2n) of that shape"
              % ("all columns" if nc == n else "the first %d columns" % nc, m, n, m, nc))
    line = {
        "impl": "reference", "metric": metric_name(args.form, args.workload),
        "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][1],
                                        "method": "CPU oracle, pointwise, modulus order on OpenMP threads",
                                        "m": m, "n": n, "tol": tol, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "host": host_info(),
                         "sample": sample + " (%d OpenMP threads)" % cores},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_status": r["status"],
    }
    print(json.dumps(line))
    return 0


def executed_fp64_flops(info, m, n, b):
    """FP64 flops the blocked method executes: every visit forms its Gram
    (three distinct b x b blocks of length-m dot products, 6 m b^2) and every
    rotated pair updates an m x 2b and an n x 2b panel (2 (m + n) (2b)^2);
    the O(b^2) inner solve per visit is left out."""
    nb = -(-n // (2 * b)) * 2
    visits = info.pair_visits if info.pair_visits else info.sweeps * nb * (nb // 2)
    return visits * 6.0 * m * b * b + info.pair_updates * 2.0 * (m + n) * (2 * b) ** 2


def time_solve(api, G, J, opts, out, stream):
    """One solve bracketed by CUDA events on its stream: (result, ms)."""
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = api.hsvd_solve_ex(G, J, opts, out=out, stream=stream)
    e1.record(stream)
    e1.synchronize()
    return r, e0.elapsed_time(e1)


def measure_plain_fp64(api, G, J, G_np, J_np, workload, tol, block, out, stream, sort=None):
    """The plain FP64 blocked method on the same factor (one timed solve): its
    time, sweeps, effective and executed FP64 rates, and its sigma against the
    stored oracle values.  ``sort``: diagonal sorting on/off (None: the
    library's choice, off for this form)."""
    m, n = G_np.shape
    opts = api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS, method=api.HSVD_METHOD_BLOCKED, block_w=block,
                         precision=api.HSVD_PRECISION_FP64, sort=sort)
    r, ms = time_solve(api, G, J, opts, out, stream)
    ex = executed_fp64_flops(r, m, n, block)
    return r, {"ms": ms, "sweeps": r.sweeps, "status": api.hsvd_status_string(r.status), "block_w": block,
               "sort": bool(sort),
               "eff_tflops": r.sweeps * flops_per_sweep(m, n) / (ms * 1e-3) / 1e12,
               "executed_fp64_tflops": ex / (ms * 1e-3) / 1e12,
               "executed_frac_of_fp64_peak": ex / (ms * 1e-3) / 1e12 / FP64_PEAK,
               "executed_note": "Gram 6 m b^2 per visit + update 2 (m+n) (2b)^2 per rotated pair, over the whole "
                                "solve's time (inner solves and sweep overheads included), against the derived "
                                "FP64 peak %.3f TFLOP/s" % FP64_PEAK,
               "accuracy": accuracy_vs_golden(G_np, J_np, out[0].cpu().numpy(), golden_path(workload))}


def measure_learned(api, dev, stream, tau, log):
    """The learned form on the graded 8192 factor (condition 1e8, b = 64,
    FP64 products) against the plain FP64 method on the same factor, one timed
    solve each; the network is trained first (outside the timed solves)."""
    import torch

    n, block = 8192, 64
    params = train_skip_model(block, api.HSVD_PRECISION_FP64, log)
    G_np, J_np = make_input("graded8192")
    G = torch.from_numpy(G_np).to(dev).t().contiguous().t()
    J = torch.from_numpy(J_np).to(dev)
    sigma = torch.empty(n, dtype=torch.float64, device=dev)
    U = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    V = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    tol = n * U64
    kw = dict(tol=tol, method=api.HSVD_METHOD_BLOCKED, block_w=block, precision=api.HSVD_PRECISION_FP64, sort=False)
    pr, plain_ms = time_solve(api, G, J, api.make_opts(max_sweeps=MAX_SWEEPS, **kw), (sigma, U, V), stream)
    s_plain = sigma.clone()
    acc_plain = accuracy_vs_golden(G_np, J_np, s_plain.cpu().numpy(), golden_path("graded8192"))
    lr, learned_ms = time_solve(api, G, J, api.make_opts(max_sweeps=2 * MAX_SWEEPS, skip_model=params,
                                                         skip_tau=tau, **kw), (sigma, U, V), stream)
    f = pr.sweeps * flops_per_sweep(n, n)
    return {"workload": WORKLOADS["graded8192"][1] + ", b=64, FP64 products, no sorting",
            "plain_ms": plain_ms, "learned_ms": learned_ms, "speedup_vs_plain": plain_ms / learned_ms,
            "plain_eff_tflops": f / (plain_ms * 1e-3) / 1e12, "learned_eff_tflops": f / (learned_ms * 1e-3) / 1e12,
            "plain_sweeps": pr.sweeps, "learned_sweeps": lr.sweeps, "masked_sweeps": lr.masked_sweeps,
            "judge_sweeps": lr.judge_sweeps, "plain_pair_visits": pr.pair_visits,
            "learned_pair_visits": lr.pair_visits,
            "status": [api.hsvd_status_string(pr.status), api.hsvd_status_string(lr.status)],
            "max_rel_sigma_diff_vs_plain": float(((sigma - s_plain).abs() / s_plain).max()),
            "accuracy_plain": acc_plain,
            "accuracy_learned": accuracy_vs_golden(G_np, J_np, sigma.cpu().numpy(), golden_path("graded8192")),
            "tau": tau, "training": log}


def run_blocked(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1008_1371_gb300 import api, build_lib

    if local == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    n, wdesc, wblock = WORKLOADS[args.workload]
    block = args.block or wblock
    prec = api.HSVD_PRECISION_BF16X8 if args.form in ("bf16x8", "learned-bf16x8") else api.HSVD_PRECISION_FP64
    if prec == api.HSVD_PRECISION_BF16X8:
        block = 64
    learned = args.form.startswith("learned")
    forms = (not args.no_forms and world == 1 and args.workload == DEFAULT_WORKLOAD and args.form == DEFAULT_FORM
             and args.tstop == 0.0 and args.tol == 0.0)
    learn_log = {}
    skip_model = train_skip_model(block, prec, learn_log) if learned else None
    G_np, J_np = make_input(args.workload, seed_offset=rank)
    m = G_np.shape[0]
    tol = args.tol if args.tol > 0 else n * U64
    G = torch.from_numpy(G_np).to(dev).t().contiguous().t()
    J = torch.from_numpy(J_np).to(dev)
    sigma = torch.empty(n, dtype=torch.float64, device=dev)
    U = torch.empty((n, m), dtype=torch.float64, device=dev).t()
    V = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    schedule = {"auto": api.HSVD_SCHEDULE_AUTO, "steps": api.HSVD_SCHEDULE_STEPS,
                "pairs": api.HSVD_SCHEDULE_PAIRS}[args.schedule]
    # diagonal sorting: the library's choice (on for split precision, off for
    # FP64); the learned form follows visits across sweeps and needs it off
    sort = False if learned else None
    opts = api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS * (2 if learned else 1), method=api.HSVD_METHOD_BLOCKED,
                         block_w=block, precision=prec, sort=sort, skip_model=skip_model,
                         skip_tau=args.tau, tstop=args.tstop, schedule=schedule)
    # kernel timing: the same solve with every kernel bracketed by CUDA events,
    # under the step schedule (each kernel alone on the GPU, back to back)
    opts_prof = api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS * (2 if learned else 1), method=api.HSVD_METHOD_BLOCKED,
                              block_w=block, profile=True, precision=prec, sort=sort, skip_model=skip_model,
                              skip_tau=args.tau, tstop=args.tstop, schedule=api.HSVD_SCHEDULE_STEPS)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def solve():
        return api.hsvd_solve_ex(G, J, opts, out=(sigma, U, V), stream=stream)

    # the learned form and the early stop are measured against the plain method
    # on the same factor: one plain solve (after one warm-up), untimed in the
    # step loop; its sweep count is the S of the effective flop count
    plain = None
    if learned or args.tstop != 0.0:
        popts = api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS, method=api.HSVD_METHOD_BLOCKED, block_w=block,
                              precision=prec, sort=sort)
        api.hsvd_solve_ex(G, J, popts, out=(sigma, U, V), stream=stream)
        pr, pms = time_solve(api, G, J, popts, (sigma, U, V), stream)
        plain = {"ms": pms, "sweeps": pr.sweeps, "pair_visits": pr.pair_visits, "sigma": sigma.clone(),
                 "status": pr.status}

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    infos, step_ms = [], []
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = solve()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, world, dev)
    ms_median = statistics.median(step_ms)
    info = infos[-1]
    assert info.status == api.HSVD_OK, api.hsvd_status_string(info.status)
    sigma_run = sigma.cpu().numpy()
    # second timed region: per-kernel CUDA-event times (step schedule)
    infos_k = []
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        infos_k.append(api.hsvd_solve_ex(G, J, opts_prof, out=(sigma, U, V), stream=stream))
    torch.cuda.synchronize()
    ms_steps = sum(i.ms_gram + i.ms_solve + i.ms_update + i.ms_other for i in infos_k) / len(infos_k)
    sweeps = info.sweeps

    # accuracy against the stored oracle values (tests/golden/make_golden.py, on
    # a machine whose G has the same bytes as this one's)
    accuracy = None
    if rank == 0 and os.path.exists(golden_path(args.workload)):
        accuracy = accuracy_vs_golden(G_np, J_np, sigma_run, golden_path(args.workload))
    if rank == 0 and args.check and prec == api.HSVD_PRECISION_BF16X8:
        accuracy = dict(accuracy or {}, vs_plain_fp64=check_against_fp64(api, G, J, sigma, U, V, tol, J_np))

    # the plain FP64 method on the same factor (the metric's comparison)
    plain64 = None
    if forms:
        # the comparison is at the metric's accuracy: on this factor the plain
        # form meets the sigma gate with diagonal sorting (and is faster with
        # it); the library's default for the form (unsorted) is timed beside it
        pr64, plain64 = measure_plain_fp64(api, G, J, G_np, J_np, args.workload, tol, 64, (sigma, U, V), stream,
                                           sort=True)
        _, uns = measure_plain_fp64(api, G, J, G_np, J_np, args.workload, tol, 64, (sigma, U, V), stream,
                                    sort=False)
        plain64["unsorted_default"] = {k: uns[k] for k in ("ms", "sweeps", "status", "executed_frac_of_fp64_peak")}
        plain64["unsorted_default"]["accuracy_gate"] = uns["accuracy"].get("gate")
        plain64["unsorted_default"]["worst_err_over_tolerance"] = uns["accuracy"].get("worst_err_over_tolerance")
        plain = {"sweeps": pr64.sweeps, "status": pr64.status}
    # S of the effective flop count: the plain run's sweeps (the learned form's
    # own count includes its masked and judge sweeps)
    s_eff = plain["sweeps"] if plain and plain["status"] == api.HSVD_OK else sweeps
    eff_flops = s_eff * flops_per_sweep(m, n)
    vs_plain, tstop_vs_plain = None, None
    if plain and args.tstop != 0.0:
        tstop_vs_plain = {"plain_ms": plain["ms"], "tstop_ms": ms, "plain_sweeps": plain["sweeps"],
                          "tstop_sweeps": sweeps, "plain_status": api.hsvd_status_string(plain["status"]),
                          "stop_rule": {1: "orthogonality", 2: "tangent"}.get(info.stop_rule, "none"),
                          "max_rel_sigma_diff_vs_plain":
                              float(np.max(np.abs(sigma_run - plain["sigma"].cpu().numpy())
                                           / plain["sigma"].cpu().numpy()))}
    if plain and learned:
        vs_plain = {"plain_ms": plain["ms"], "learned_ms": ms, "speedup_vs_plain": plain["ms"] / ms,
                    "plain_sweeps": plain["sweeps"], "learned_sweeps": sweeps, "masked_sweeps": info.masked_sweeps,
                    "judge_sweeps": info.judge_sweeps, "plain_pair_visits": plain["pair_visits"],
                    "learned_pair_visits": info.pair_visits,
                    "max_rel_sigma_diff_vs_plain": float(np.max(np.abs(sigma_run - plain["sigma"].cpu().numpy())
                                                                / plain["sigma"].cpu().numpy())),
                    "tau": args.tau, "training": learn_log}
    value = world * eff_flops / (ms * 1e-3) / 1e12

    # dominant kernel class by CUDA-event time over the kernel-timing region
    tot = {k: sum(getattr(i, "ms_" + k) for i in infos_k) for k in ("gram", "solve", "update", "other")}
    upd_pairs = sum(i.pair_updates for i in infos_k)
    nb = -(-n // (2 * block)) * 2
    visits = sum(i.pair_visits for i in infos_k) or sum(i.sweeps for i in infos_k) * nb * (nb // 2)
    alg = {
        "update": upd_pairs * 2.0 * (m + n) * (2 * block) ** 2,
        "gram": visits * (6.0 if prec == api.HSVD_PRECISION_FP64 else 8.0) * m * block * block,
        # an inner rotation mixes two rows and two columns of A_P and two
        # columns of W_P: 3 vector pairs of length 2b, 6 flops per index
        "solve": sum(i.rotations for i in infos_k) * 18.0 * (2 * block),
    }
    dom = max(("gram", "update", "solve"), key=lambda k: tot[k])
    achieved = alg[dom] / (tot[dom] * 1e-3) / 1e12 if tot[dom] > 0 else None
    # the inner solve's main kernel: the cross pass (every step but the first of a sweep)
    kname = {"gram": "k_gram<%d>" % block, "update": "k_update<%d>" % (2 * block),
             "solve": "k_solve_cross<%d,%d>" % (2 * block, 4 if block == 16 else 8)}
    if prec == api.HSVD_PRECISION_BF16X8:
        kname = {"gram": "k_gram_x", "update": "k_update_x", "solve": "k_solve_cross<128,8>"}
    if dom == "solve" or prec == api.HSVD_PRECISION_FP64:
        roofline = {"kernel": kname[dom], "bound": "alu", "achieved": achieved, "peak": FP64_PEAK,
                    "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK) if achieved else None, "traffic": None,
                    "peak_source": FP64_PEAK_SOURCE}
        if dom == "solve":
            roofline["note"] = ("the inner solve is a chain of dependent rotation steps (sqrt/div latency and "
                                "cluster barriers per step): latency bound, far below the FP64 unit's rate")
    else:
        # the tensor work of a split product: 36 BF16 slice products per FP64 product
        bf16_peak = 1897.8
        ach_t = 36.0 * achieved if achieved else None
        roofline = {"kernel": kname[dom], "bound": "tensor", "achieved": ach_t, "peak": bf16_peak,
                    "unit": "TFLOP/s", "frac": (ach_t / bf16_peak) if ach_t else None, "traffic": None,
                    "peak_source": "bf16 dense, measured burst (MEASURED_PEAKS.json bf16_tflops)",
                    "fp64_equivalent_tflops": achieved}
    roofline["ms_by_kernel"] = {k: v / len(infos_k) for k, v in tot.items()}
    roofline["timing"] = ("kernels bracketed by CUDA events in a second timed region of %d solves under the step "
                          "schedule (each kernel alone on the GPU); the step schedule's own time per solve there: "
                          "%.2f ms" % (len(infos_k), ms_steps))
    roofline["alg_fp64_tflops_by_kernel"] = {k: alg[k] / (tot[k] * 1e-3) / 1e12 for k in alg if tot[k] > 0}
    traffic = PROFILED_TRAFFIC.get((args.workload, args.form, roofline["kernel"]))
    if traffic:
        roofline["traffic"] = traffic[0]
        roofline["traffic_source"] = traffic[1]

    # end to end through the C ABI with pinned host arrays, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Gh = torch.from_numpy(G_np).t().contiguous().t().pin_memory()
        Jh = torch.from_numpy(J_np).pin_memory()
        sh = torch.empty(n, dtype=torch.float64).pin_memory()
        Uh = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
        Vh = torch.empty((n, n), dtype=torch.float64).pin_memory().t()
        opts_e2e = api.make_opts(tol=tol, max_sweeps=MAX_SWEEPS * (2 if learned else 1),
                                 method=api.HSVD_METHOD_BLOCKED, block_w=block, precision=prec, sort=sort,
                                 skip_model=skip_model, skip_tau=args.tau, tstop=args.tstop, schedule=schedule)
        api.hsvd_solve_ex(Gh, Jh, opts_e2e, out=(sh, Uh, Vh))
        e2e_t = []
        for _ in range(max(3, args.steps // 4)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.hsvd_solve_ex(Gh, Jh, opts_e2e, out=(sh, Uh, Vh))
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = sum(e2e_t) / len(e2e_t)
        e2e_s = max_over_ranks(e2e_s, world, dev)
        e2e = {"value": world * eff_flops / e2e_s / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": m * n * 8 + n, "d2h_bytes_per_step": n * 8 + m * n * 8 + n * n * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(G_np, J_np, tol, args.cpu_sweeps)

    forms_vs_plain = None
    if forms:
        forms_vs_plain = {"precision": {
            "workload": wdesc, "form": "BF16x8 split-precision Gram/update on the tensor cores, FP64 rotations",
            "form_ms": ms, "form_sweeps": sweeps, "plain_fp64": plain64, "speedup_vs_plain": plain64["ms"] / ms,
            "form_accuracy": accuracy}}
        del G, U, V, sigma  # room for the next workloads
        torch.cuda.empty_cache()
        b = measure_batched(api, dev, BATCH_COUNT, 3, 1, 0, args.loop_count, with_e2e=False, with_cpu=False)
        forms_vs_plain["batched"] = {
            "workload": WORKLOADS["batch10k"][1], "batched_ms": b["ms"],
            "batched_eff_tflops": b["eff_flops"] / (b["ms"] * 1e-3) / 1e12, "steps": 3, "warmup": 1,
            "loop_of_single_solves": b["loop"], "speedup_vs_loop": b["loop"]["ms_whole_batch"] / b["ms"],
            "roofline": batched_roofline(b), "accuracy": b["accuracy"], "gpu_launches": b["launches"]}
        del b
        torch.cuda.empty_cache()
        forms_vs_plain["learned"] = measure_learned(api, dev, stream, args.tau, {})

    if rank == 0:
        line = {
            "metric": metric_name(args.form, args.workload), "value": value,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_step_median": ms_median,
            "config": {"workload": wdesc, "method": "blocked, b=%d, %s" % (block, args.form), "m": m, "n": n,
                       "block_w": block, "form": args.form, "tol": tol, "tstop": args.tstop,
                       "schedule": args.schedule,
                       "sweeps": sweeps, "sweeps_in_flop_count": s_eff,
                       "inner": "block-oriented",
                       "sort": bool(sort is None and prec == api.HSVD_PRECISION_BF16X8),
                       "l2": "flushed (256 MB write) between steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy": accuracy, "forms_vs_plain": forms_vs_plain,
            "learned_vs_plain": vs_plain, "tstop_vs_plain": tstop_vs_plain,
            "gpu_launches": int(sum(i.kernel_launches for i in infos)),
            # host wall time inside each timed solve spent capturing and
            # instantiating its sweep graph (part of ms_per_step)
            "host_graph_ms_per_step": sum(getattr(i, "ms_host_graph", 0.0) for i in infos) / len(infos),
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
        }
        # the timed form's own sigma decides the exit status; the comparison
        # runs report their gates in their own entries
        gates = [x.get("gate") for x in (accuracy, (accuracy or {}).get("vs_plain_fp64")) if isinstance(x, dict)]
        line["accuracy_gate"] = "fail" if "fail" in gates else ("pass" if gates else "not compared")
        print(json.dumps(line))
        if line["accuracy_gate"] == "fail":
            sys.stderr.write("accuracy gate failed: sigma beyond the stated tolerance against the oracle\n")
            return 3
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.probe_rates:
        return probe_rates()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch10k":
        return run_batched(args)
    return run_blocked(args)


if __name__ == "__main__":
    sys.exit(main())
