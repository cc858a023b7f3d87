#!/usr/bin/env python
"""Benchmark of the HOOI hot path on the 3-mode Zipf workload.

Workload: 2,000,000 x 1,000,000 x 50,000 COO tensor with 100M distinct
nonzeros, Zipf(1.1) coordinates per mode (seeded permutation of the index
space), lognormal(0,1) values, core 10x10x10, seeded random orthonormal
initial factors.  A step is one HOOI invocation (Fig. 1: TTM-chain + factor
update for every mode, then core and fit) with the tensor resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "zipf1.1-2Mx1Mx50K-nnz100M-k10"
METRIC = "HOOI s/iter & TTM-chain GB/s (% HBM peak), mixed vs FP64 GPU at fixed fit"
CPU_SAMPLE = 500_000  # elements of the oracle's bounded sample (first elements of the stream)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--nnz", type=int, default=None, help="fewer nonzeros, same recipe (smoke runs only)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE)
    ap.add_argument("--adjoint", action="store_true",
                    help="a step also runs the adjoint of every mode's TTM-chain (dL/dF_m and dL/dvals for a fixed "
                         "cotangent dZ_n), the differentiable use of the path")
    ap.add_argument("--schemes", type=int, default=0, metavar="P",
                    help="instead of timing: print the Section 4.1 metrics (E_max, R_sum, R_max) of Lite, CoarseG "
                         "and MediumG with P processors for every mode of the workload (the paper's comparison of "
                         "distribution schemes, Section 7), with seeded random orders")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3"],
                    help="FP32 context with the Gram in split TF32 (fp32) or split BF16 (bf16x3)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    sm_max_mhz=float(d.get("sm_max_mhz", 2070)), source="measured")
    return dict(hbm_gbs=6800.0, bf16=1900.0, bf16_sustained=1700.0, sm_max_mhz=2070.0, source="fallback")


# dense TF32 / BF16 tensor rates of the part (nominal 1.1 and 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def ttm_roofline(kernel, bytes_per_launch, flops_per_launch, s_per_launch, pk, fp32_peak_tflops, traffic):
    """Roofline object of the TTM-chain launches.  The CUDA-core chain is
    reported against the measured HBM copy bandwidth (algorithmic bytes per
    launch over its time).  A chain that runs on the tensor cores in every mode
    is a contraction: its algorithmic FLOPs (2 nnz Khat per launch) against the
    TF32 rate, i.e. the measured sustained BF16 rate (the chain is timed inside
    a long step) times the nominal TF32 / BF16 ratio; its HBM figures stay
    alongside."""
    gbs = bytes_per_launch / s_per_launch / 1e9
    tflops = flops_per_launch / s_per_launch / 1e12
    common = dict(kernel=kernel, bytes_per_launch=int(bytes_per_launch), ms_per_launch=round(s_per_launch * 1e3, 4),
                  alu_tflops=round(tflops, 2), alu_frac_fp32=round(tflops / fp32_peak_tflops, 4))
    if kernel == "k_ttmc_tc":
        peak = pk["bf16_sustained"] * TF32_PER_BF16
        return dict(bound="tensor", achieved=round(tflops, 2), peak=round(peak, 1), unit="TFLOP/s",
                    frac=round(tflops / peak, 4), traffic=None,
                    peak_source=pk["source"] + " (bf16_tflops_sustained x 1.1/2.25, the nominal TF32/BF16 ratio)",
                    hbm_gbs=round(gbs, 1), hbm_frac=round(gbs / pk["hbm_gbs"], 4), **common)
    return dict(bound="hbm", achieved=round(gbs, 1), peak=pk["hbm_gbs"], unit="GB/s", frac=round(gbs / pk["hbm_gbs"], 4),
                traffic=traffic, peak_source=pk["source"] + " (hbm_gbs)", **common)


# ----------------------------------------------------------------- clocks
class Clocks:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------- helpers
def job_time(t_loc, world, device):
    """The job's timed region: the maximum over ranks of the local one (the job
    ends when its slowest rank does)."""
    if world == 1:
        return t_loc
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t_loc], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def per_invocation(t_all, steps, world):
    """Whole-job seconds per invocation: world ranks each ran `steps`
    invocations (replicas) within t_all."""
    return t_all / (steps * world)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def ttm_bytes_flops(w, R, n):
    """Algorithmic bytes and FLOPs of one TTM-chain launch along mode n:
    the element stream (N-1 coordinates + row code + value, 4 B each), every
    other factor read once, the compact Z written once; one FMA per Z entry
    per element."""
    L, K, nnz = w["L"], w["K"], len(w["vals"])
    N = len(L)
    khat = int(np.prod([K[m] for m in range(N) if m != n]))
    stream = nnz * 4 * (N + 1)
    fac = sum(L[m] * K[m] * 4 for m in range(N) if m != n)
    z = R[n] * khat * 4
    return stream + fac + z, 2.0 * nnz * khat


def core_mode(w, R):
    """The mode whose TTM-chain forms the core (the library's rule: smallest
    Khat, then the fewest non-empty slices)."""
    K = w["K"]
    N = len(K)
    kh = [int(np.prod([K[m] for m in range(N) if m != n])) for n in range(N)]
    best = 0
    for n in range(1, N):
        if kh[n] < kh[best] or (kh[n] == kh[best] and R[n] < R[best]):
            best = n
    return best


def host_threads():
    """Host cores the oracle may use: the process's CPU affinity (else nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample_seconds(w, samples, repeats=1):
    """Times `repeats` oracle HOOI invocations (+ core + fit) on each of the
    leading `samples` elements of the stream, from the same initial factors,
    in one fresh process whose BLAS may use every host core (the oracle's
    element loops are single-threaded numpy).  Returns the mean seconds per
    invocation for each sample size."""
    samples = list(samples)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sample.npz")
        F0 = w["F0"]
        top = max(samples)
        np.savez(path, idx=w["idx"][:, :top], vals=w["vals"][:top], L=np.array(w["L"]),
                 **{f"F{m}": F0[m] for m in range(len(F0))})
        code = (
            "import sys, time, numpy as np; sys.path.insert(0, %r)\n"
            "from oracle import tucker_oracle as O\n"
            "d = np.load(%r); L = tuple(int(x) for x in d['L']); N = len(L)\n"
            "F = [d['F%%d' %% m] for m in range(N)]\n"
            "idx_all = d['idx'].astype(np.int64); v_all = d['vals'].astype(np.float64)\n"
            "for n_s in %r:\n"
            "    idx = idx_all[:, :n_s]; v = v_all[:n_s]; ts = []\n"
            "    for _ in range(%d):\n"
            "        t = time.perf_counter(); F1 = O.hooi_invocation(L, idx, v, F); G = O.core(L, idx, v, F1)\n"
            "        f = O.fit(v, G); ts.append(time.perf_counter() - t)\n"
            "    print(n_s, sum(ts) / len(ts), flush=True)\n" % (ROOT, path, samples, int(repeats)))
        nt = str(host_threads())
        env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt,
                   CUDA_VISIBLE_DEVICES="")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode != 0:
            raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
        out = {}
        for line in r.stdout.strip().splitlines():
            a, b = line.split()
            out[int(a)] = float(b)
        return [out[n_s] for n_s in samples]


def extrapolate(samples, secs, nnz):
    """Least-squares line t = a + b * n through the sampled (n, t), evaluated at
    nnz; returns (estimate, a, b, largest relative residual)."""
    x = np.asarray(samples, dtype=np.float64)
    y = np.asarray(secs, dtype=np.float64)
    if len(x) < 2:
        b = float(y[0] / x[0])
        return b * nnz, 0.0, b, 0.0
    A = np.stack([np.ones_like(x), x], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    res = float(np.max(np.abs(A @ np.array([a, b]) - y) / y))
    return float(a + b * nnz), float(a), float(b), res


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_ttmc_fwd_dram_zipf1.1-2Mx1Mx50K-nnz100M.md")
CSRC = os.path.join(ROOT, "paper_1804_09494_gb300", "csrc")


def source_fingerprints():
    """sha256 of the TTM-chain kernel file and of the function choosing the
    core's chain (the launch mix of an invocation): the ncu counters of the
    traffic profile hold while both are unchanged."""
    with open(os.path.join(CSRC, "tk_ttmc.cu"), "rb") as f:
        ttmc = hashlib.sha256(f.read()).hexdigest()
    with open(os.path.join(CSRC, "tk_core.cu")) as f:
        src = f.read()
    i = src.index("int tk_core_mode(")
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            break
    core_mode_fn = hashlib.sha256(src[i:k + 1].encode()).hexdigest()
    return {"tk_ttmc.cu": ttmc, "tk_core_mode": core_mode_fn}


def ttm_traffic_per_launch(args):
    """DRAM bytes (read + write) per TTM-chain launch from the committed ncu
    summary of the full-size workload; None for another workload or when the
    kernel source has changed since the counters were taken."""
    if args.workload != WORKLOAD or args.nnz is not None or not os.path.exists(TRAFFIC_PROFILE):
        return None
    val, sha = None, {}
    with open(TRAFFIC_PROFILE) as f:
        for line in f:
            if line.startswith("traffic_bytes_per_launch:"):
                val = int(line.split(":")[1])
            elif " sha256:" in line:
                name, h = line.split(" sha256:")
                sha[name.strip()] = h.strip()
    for name, h in source_fingerprints().items():
        if sha.get(name) != h:
            return None
    return val


def load_workload(args):
    from paper_1804_09494_gb300 import synth
    w = synth.workload(args.workload, nnz=args.nnz)
    w["F0"] = synth.random_orthonormal_factors(w["L"], w["K"], seed=1234)
    return w


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = load_workload(args)
    nnz = len(w["vals"])
    # one process for all steps; the per-step sample shrinks with the step
    # count so that the whole run stays near a minute and a half of oracle time
    sample = min(nnz, args.cpu_sample, max(50_000, args.cpu_sample * 20 // max(args.steps, 1)))
    samples = sorted({max(1, sample // 4), max(1, sample // 2), sample})
    secs = oracle_sample_seconds(w, samples, repeats=args.steps)
    t, a, b, res = extrapolate(samples, secs, nnz)
    threads = host_threads()
    line = dict(metric=METRIC, value=t, unit="s/iter", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=t * 1e3, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=args.workload, nnz=nnz, L=list(w["L"]), K=list(w["K"])),
                cpu_baseline=dict(value=t, unit="s/iter", cores=threads, threads=threads, nproc=os.cpu_count(),
                                  kind="oracle",
                                  sample=f"first {', '.join(f'{x:,}' for x in samples)} of {nnz:,} elements, "
                                         f"{args.steps} HOOI invocations + core + fit each in one process (BLAS on "
                                         f"{threads} threads; the element loops run on one), s = a + b n fitted "
                                         f"(a = {a:.3g} s, b = {b:.3g} s/element, largest residual {res:.1%}) and "
                                         f"evaluated at n = nnz",
                                  sample_seconds=[round(x, 4) for x in secs]),
                e2e=dict(value=t, unit="s/iter", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1804_09494_gb300.tucker import PHASES, Tucker

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = peaks()

    w = load_workload(args)
    L, K = w["L"], w["K"]
    N = len(L)
    nnz = len(w["vals"])
    idx_d = torch.from_numpy(w["idx"]).to(dev)
    vals_d = torch.from_numpy(w["vals"]).to(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # distribution (Lite partition + permuted copies), timed once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tk = Tucker(idx_d, vals_d, L, K, prec=args.prec, timing=True)
    torch.cuda.synchronize()
    forms = [tk.ttm_form(n)["tensor_cores"] for n in range(N)]
    ttm_kernel = "k_ttmc_tc" if all(forms) else ("k_ttmc_fwd" if not any(forms) else "k_ttmc_fwd + k_ttmc_tc")
    partition_s = time.perf_counter() - t0
    R = tk.R
    stats = [tk.stats(n) for n in range(N)]
    F = [torch.from_numpy(f.astype(np.float32)).to(dev) for f in w["F0"]]
    G = torch.empty(int(np.prod(K)), dtype=torch.float32, device=dev)

    # the adjoint's inputs and accumulators live outside the timed region
    if args.adjoint:
        gen = torch.Generator(device=dev).manual_seed(17)
        dZs = [torch.randn(R[n], int(np.prod([K[m] for m in range(N) if m != n])), device=dev, generator=gen)
               for n in range(N)]
        dFs = [[None if m == n else torch.zeros(L[m], K[m], device=dev) for m in range(N)] for n in range(N)]

    def step(want_fit):
        out = tk.hooi_iter(F, G, want_fit=want_fit)
        if args.adjoint:
            for n in range(N):
                tk.ttm_chain_backward(n, F, dZs[n], dF=dFs[n], want_dval=True)
        return out

    for _ in range(args.warmup):
        step(False)
    tk.timings(reset=True)
    clocks = Clocks(torch.cuda.get_device_properties(dev).uuid and f"GPU-{torch.cuda.get_device_properties(dev).uuid}")
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("timed")  # profilers can restrict a capture to this range
    e0.record(stream)
    for s in range(args.steps):
        _, fit = step(s == args.steps - 1)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    ck = clocks.stop()
    t_loc = e0.elapsed_time(e1) / 1e3
    t_all = job_time(t_loc, world, dev)
    ph = tk.timings(reset=True)
    launches = int(sum(v[1] for v in ph.values()))
    s_per_iter = per_invocation(t_all, args.steps, world)
    fit_mixed = fit

    # roofline of the dominant kernel (the TTM-chain): algorithmic bytes of the
    # launches in the timed region over their summed CUDA-event durations
    per_iter_bytes = 0.0
    per_iter_flops = 0.0
    for n in list(range(N)) + [core_mode(w, R)]:
        b, f = ttm_bytes_flops(w, R, n)
        per_iter_bytes += b
        per_iter_flops += f
    ttm_ms, ttm_launches = ph["ttm_chain"]
    ttm_s_per_launch = ttm_ms / 1e3 / max(ttm_launches, 1)
    launches_per_iter = ttm_launches / args.steps
    bytes_per_launch = per_iter_bytes / launches_per_iter
    achieved_gbs = bytes_per_launch / ttm_s_per_launch / 1e9
    traffic = ttm_traffic_per_launch(args)
    # FP32 FMA lanes: 128 per SM on this architecture; SM count from the device
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak_tflops = sms * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12

    # end to end through the public API with pinned host buffers
    Fh = [torch.from_numpy(f.astype(np.float32)).pin_memory() for f in w["F0"]]
    Fo = [torch.empty_like(f).pin_memory() for f in Fh]
    Gh = torch.empty(G.shape, dtype=torch.float32).pin_memory()
    h2d = sum(f.numel() * 4 for f in Fh)
    d2h = h2d + Gh.numel() * 4 + 8
    e2e_steps = max(1, min(args.steps, 20))

    def e2e_step():
        for fd, fh in zip(F, Fh):
            fd.copy_(fh, non_blocking=True)
        _, fit_e2e = step(True)  # the fit is read back to the host
        for fo, fd in zip(Fo, F):
            fo.copy_(fd, non_blocking=True)
        Gh.copy_(G, non_blocking=True)

    for _ in range(max(1, min(args.warmup, 3))):  # first use of the pinned buffers is not timed
        e2e_step()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_s = e0.elapsed_time(e1) / 1e3 / e2e_steps

    # the plain FP64 form on the same tensor and initial factors; fits compared
    # after the same number of invocations (fixed fit)
    fp64 = None
    if args.fp64_steps > 0:
        tk64 = Tucker(idx_d, vals_d.double(), L, K, prec="fp64", timing=False)
        F64 = [torch.from_numpy(f).to(dev) for f in w["F0"]]
        G64 = torch.empty(int(np.prod(K)), dtype=torch.float64, device=dev)
        Fm = [torch.from_numpy(f.astype(np.float32)).to(dev) for f in w["F0"]]
        fits32, fits64 = [], []
        tk.hooi_iter(Fm, G, want_fit=True)
        tk64.hooi_iter(F64, G64, want_fit=True)
        barrier()
        e0.record(stream)
        for _ in range(args.fp64_steps):
            _, f64 = tk64.hooi_iter(F64, G64, want_fit=True)
            fits64.append(f64)
        e1.record(stream)
        barrier()
        t64 = e0.elapsed_time(e1) / 1e3 / args.fp64_steps
        for _ in range(args.fp64_steps):
            _, f32 = tk.hooi_iter(Fm, G, want_fit=True)
            fits32.append(f32)
        fp64 = dict(s_per_iter=t64, fit_after=[round(x, 12) for x in fits64],
                    mixed_fit_after=[round(x, 12) for x in fits32],
                    max_fit_gap=max(abs(a - b) for a, b in zip(fits32, fits64)),
                    speedup_mixed_over_fp64=t64 / max(s_per_iter * world, 1e-12))
        tk64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        top = min(args.cpu_sample, nnz)
        samples = sorted({max(1, top // 4), max(1, top // 2), top})
        secs = oracle_sample_seconds(w, samples)
        est, a, b, res = extrapolate(samples, secs, nnz)
        threads = host_threads()
        cpu = dict(value=est, unit="s/iter", cores=threads, threads=threads, nproc=os.cpu_count(), kind="oracle",
                   sample=f"first {', '.join(f'{x:,}' for x in samples)} of {nnz:,} elements (same L, K, initial "
                          f"factors): one HOOI invocation + core + fit each, timed in one process with BLAS on "
                          f"{threads} threads (the element loops run on one); s = a + b n fitted (a = {a:.3g} s, "
                          f"b = {b:.3g} s/element, largest residual {res:.1%}) and evaluated at n = nnz",
                   sample_seconds=[round(x, 4) for x in secs])

    if rank == 0:
        line = dict(
            metric=METRIC, value=s_per_iter, unit="s/iter", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=t_all / args.steps * 1e3, higher_is_better=False, scaling="weak", vs_baseline=None,
            dtype="f32", data="synthetic",
            config=dict(workload=args.workload, nnz=nnz, L=list(L), K=list(K), R=R,
                        prec="fp32 TTM-chain, Gram on the tensor cores in split " + ("BF16 (three terms)" if args.prec == "bf16x3" else "TF32")
                        + " with FP64 reductions, FP64-polished eigensolve, CholeskyQR2 with FP64 reductions",
                        l2="inputs larger than L2 (permuted copies ~6 GB per context)",
                        step="HOOI invocation" + (" + adjoint of every mode's TTM-chain" if args.adjoint else ""),
                        parallelism="replicas" if world > 1 else "single GPU"),
            roofline=ttm_roofline(ttm_kernel, bytes_per_launch, per_iter_flops / launches_per_iter, ttm_s_per_launch, pk,
                                  fp32_peak_tflops, traffic),
            ttm_chain_gbs=round(achieved_gbs, 1), ttm_chain_frac_hbm=round(achieved_gbs / pk["hbm_gbs"], 4),
            phases_ms_per_iter={k: round(v[0] / args.steps, 4) for k, v in ph.items()},
            fit=fit_mixed, fp64_form=fp64, partition_s=round(partition_s, 3),
            partition=[dict(E_max=s["E_max"], R_sum=s["R_sum"], R_max=s["R_max"], R_n=s["R_n"], P=s["P"]) for s in stats],
            e2e=dict(value=e2e_s, unit="s/iter", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
            gpu_launches=launches, clocks=dict(sm_mhz=ck["sm_mhz"], sm_max_mhz=ck["sm_max_mhz"], reasons=ck["reasons"],
                                               samples=ck["samples"]),
            cpu_baseline=cpu, memory_bytes=tk.memory())
        print(json.dumps(line), flush=True)
    tk.close()
    if world > 1:
        dist.destroy_process_group()


def run_schemes(args):
    """One JSON line: per mode, the metrics of Lite (the context partitioned with
    P bins), CoarseG and MediumG (device, seeded random orders), and the
    distribution time of each."""
    import numpy as np
    import torch

    from paper_1804_09494_gb300.tucker import Tucker

    w = load_workload(args)
    L, K, P = w["L"], w["K"], args.schemes
    idx_d = torch.from_numpy(w["idx"]).cuda()
    vals_d = torch.from_numpy(w["vals"]).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tk = Tucker(idx_d, vals_d, L, K, prec="fp32", P_bins=P, ttm_path="cuda_cores")
    torch.cuda.synchronize()
    t_lite = time.perf_counter() - t0
    rng = np.random.default_rng(2024)
    pos = [torch.from_numpy(rng.permutation(l).astype(np.int32)).cuda() for l in L]
    modes = []
    for n in range(len(L)):
        row = {"mode": n, "avg_E": -(-len(w["vals"]) // P), "R_n": tk.stats(n)["R_n"]}
        st = tk.stats(n)
        row["lite"] = {k: st[k] for k in ("E_max", "R_sum", "R_max")}
        for name in ("coarseg", "mediumg"):
            t0 = time.perf_counter()
            m = tk.scheme_metrics(n, name, P, pos)
            row[name] = {k: m[k] for k in ("E_max", "R_sum", "R_max")}
            row[name]["metrics_s"] = round(time.perf_counter() - t0, 4)
        modes.append(row)
    tk.close()
    print(json.dumps({"workload": args.workload, "nnz": len(w["vals"]), "P": P, "lite_partition_s": round(t_lite, 3),
                      "modes": modes}))


def main():
    args = parse()
    if args.schemes:
        run_schemes(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
