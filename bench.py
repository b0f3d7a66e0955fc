"""Benchmark of the weighted-NMF hot path.

Workloads (--workload):
  stis     (default) one STIS-shaped reduction: the sequential fit of the
           basis (K = 30 components x 500 multiplicative-update iterations on
           N = 300 references of P = 49343 masked pixels), the projection of
           the M = 50 science frames (500 iterations) and their PSF
           subtraction.
  miri     one MIRI-shaped reduction: N = 1000 references of P = 62961
           pixels, K = 50 x 500 iterations, M = 50 frames.
  wide     the STIS shape with K = 100 components (stages 65 .. 100 run the
           128-component kernels), 100 iterations per stage and projection.
  batched  64 independent reductions of uneven N, P, K and frame counts
           (half in the tensor-core form, half plain FP32) in one
           nmf_fit_batched call, next to the same 64 reductions run one after
           the other in plain FP32.
  table2   the analogue of the paper's Table 2: end-to-end wall time of one
           STIS-shaped reduction for K = 10 ... 110, both GPU forms and the
           FP64 oracle.

One step = the whole workload through libnmfgb's C-ABI on device-resident
inputs.  The headline `value` is fit iterations per second (sum over stages
and problems of the iterations per step / step time); TFLOP/s counts the
algorithmic flops of the whole step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload stis|miri|batched]

Under torchrun each rank runs an independent replica of the workload (the
reductions are independent problems: no data-path collective); the step time
is the max over ranks and `value` sums the ranks' iterations.
`--impl reference` times the FP64 CPU oracle on the host cores instead (each
step a bounded sample, extrapolated to the full step; rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "weighted-NMF iterations/s and TFLOP/s (% of roofline) vs plain FP32 at <=1e-3 residual error"
UNIT = "iterations/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop per FMA x SM clock.
def fp32_simt_peak_tflops(mhz):
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def fp32_peak_measured(nmf, mhz):
    """The FP32 CUDA-core ceiling: the library's FMA-rate microbenchmark
    (best of three runs, CUDA events), with the derived figure as a fallback."""
    try:
        v = max(nmf.fp32_fma_rate(1 << 16) for _ in range(3))
        return v, (f"measured FP32 FMA rate (nmf_fp32_fma_rate: 4 blocks/SM x 512 threads x 8 FMA chains, best of "
                   f"3); derived 152 x 128 x 2 x {mhz:.0f} MHz = {fp32_simt_peak_tflops(mhz):.1f}")
    except Exception as e:  # pragma: no cover
        return fp32_simt_peak_tflops(mhz), f"derived 152 x 128 x 2 x {mhz:.0f} MHz (FMA benchmark failed: {e})"


def code_fingerprint(text):
    """SHA-1 of C/CUDA source with its comments removed and its whitespace
    collapsed: it changes when the code changes, not when a comment does."""
    import hashlib
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha1(" ".join(text.split()).encode()).hexdigest()


def measured_traffic(form="bf16w32", k=30):
    """DRAM bytes of one iteration at rank k (H pass + W pass + update) of the
    tensor-core form `form` on the STIS shape, from the committed ncu capture
    (k = 30 and k = 100), or None if there is none or the kernel code changed
    since."""
    try:
        with open(os.path.join(ROOT, "profiles", f"traffic_stis_k{k}_{form}.json")) as f:
            d = json.load(f)
        with open(os.path.join(ROOT, d["source"])) as f:
            if code_fingerprint(f.read()) != d.get("source_code_sha1"):
                return None
        return d["iteration_dram_bytes"]
    except (OSError, KeyError, ValueError):
        return None


def workload_flops(N, P, K, iters, M, proj_iters):
    """Algorithmic flops of one step (Eq. 3 contractions; O(NP) terms ignored)."""
    fit = iters * 12.0 * N * P * K * (K + 1) / 2.0
    proj = 2.0 * M * P * K + proj_iters * 4.0 * M * P * K
    sub = 2.0 * M * P * K
    return fit + proj + sub


def max_over_ranks(x, dist, device):
    """The slowest rank's value (every rank's timed region is bracketed by
    barriers, so the job's step time is the maximum)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, step_ms):
    """Whole-job units per second: every rank processes its own replica of
    the workload (weak scaling), the step lasts as long as the slowest rank."""
    return world * units_per_rank / (step_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def cpu_reference_sample(prob, iters, K, ks=None, reps=None):
    """Time the FP64 oracle on a bounded sample of the step and extrapolate.

    Sample: `reps` iterations of Eq. 3 at each rank k in `ks` on the full data
    (fit of t(k) = a + b k by least squares: an iteration costs 12 N P k flops
    plus O(NP) terms), and the projection of the M science frames for 1 and 2
    iterations (per-iteration cost = the difference).  The full step (the
    K-stage fit plus the projection) is extrapolated from those."""
    import oracle

    ks = ks or (1, K // 3 or 1, (2 * K) // 3 or 1, K)
    if reps is None:  # size the sample to ~10 s of oracle work on this host
        W = prob.W0[:, :K].astype(np.float64)
        H = prob.H0[:K].astype(np.float64)
        t0 = time.perf_counter()
        oracle.iterate(prob.V, prob.Wt, W, H, 1)
        reps = int(min(20, max(1, round(10.0 / (len(ks) * (time.perf_counter() - t0))))))
    tk = []
    for k in ks:
        W = prob.W0[:, :k].astype(np.float64)
        H = prob.H0[:k].astype(np.float64)
        t0 = time.perf_counter()
        oracle.iterate(prob.V, prob.Wt, W, H, reps)
        tk.append((time.perf_counter() - t0) / reps)
    b, a = np.polyfit(np.asarray(ks, float), np.asarray(tk), 1)
    fit_s = iters * sum(a + b * k for k in range(1, K + 1))
    Hk = prob.H0.astype(np.float64)
    t0 = time.perf_counter()
    oracle.project(Hk, prob.T, prob.WtT, prob.C0, 1)
    t1 = time.perf_counter()
    oracle.project(Hk, prob.T, prob.WtT, prob.C0, 2)
    t2 = time.perf_counter()
    p1, p2 = t1 - t0, t2 - t1
    proj_s = p1 + (iters - 1) * max(p2 - p1, 0.0)
    full = fit_s + proj_s
    sample = (f"{reps} oracle iterations at each k in {list(ks)} on the full {prob.N}x{prob.P} data "
              f"({', '.join(f'{x:.2f}' for x in tk)} s/it) + projection of {prob.M} frames for 1 and 2 "
              f"iterations; the K={K}x{iters} fit and {iters}-iteration projection extrapolated "
              f"(fit affine in k); sample wall {reps * sum(tk) + p1 + p2:.1f} s")
    return {"seconds_full_est": full, "value": K * iters / full, "sample": sample, "cores": oracle.num_threads()}


def cpu_numpy_sample(prob, iters, K, dtype, seconds=4.0):
    """Time the vectorised NumPy form of Eq. 3 (the paper's own CPU setup:
    NumPy arithmetic with BLAS matrix products) on a bounded sample of the
    step and extrapolate, as cpu_reference_sample does for the oracle."""
    from oracle import numpy_baseline as nb

    ks = (1, K // 3 or 1, (2 * K) // 3 or 1, K)
    V = prob.V.astype(dtype)
    Wt = prob.Wt.astype(dtype)
    A = Wt * V
    t0 = time.perf_counter()
    nb.iterate(V, Wt, prob.W0[:, :K], prob.H0[:K], 1, dtype=dtype, A=A)
    reps = int(min(20, max(1, round(seconds / (len(ks) * (time.perf_counter() - t0))))))
    tk = []
    for k in ks:
        nb.iterate(V, Wt, prob.W0[:, :k], prob.H0[:k], 1, dtype=dtype, A=A)  # untimed warm-up at this k
        t0 = time.perf_counter()
        nb.iterate(V, Wt, prob.W0[:, :k], prob.H0[:k], reps, dtype=dtype, A=A)
        tk.append((time.perf_counter() - t0) / reps)
    b, a = np.polyfit(np.asarray(ks, float), np.asarray(tk), 1)
    fit_s = iters * sum(a + b * k for k in range(1, K + 1))
    t0 = time.perf_counter()
    nb.project(prob.H0, prob.T, prob.WtT, prob.C0, 1, dtype=dtype)
    t1 = time.perf_counter()
    nb.project(prob.H0, prob.T, prob.WtT, prob.C0, 2, dtype=dtype)
    t2 = time.perf_counter()
    p1, p2 = t1 - t0, t2 - t1
    full = fit_s + p1 + (iters - 1) * max(p2 - p1, 0.0)
    threads, how = nb.blas_threads()
    name = np.dtype(dtype).name
    return {"value": float(K * iters / full), "unit": UNIT, "dtype": name, "threads": threads, "threads_note": how,
            "numpy": np.__version__,
            "sample": f"{reps} {name} NumPy iterations at each k in {list(ks)} on the full {prob.N}x{prob.P} data "
                      f"({', '.join(f'{x:.3f}' for x in tk)} s/it) + projection of {prob.M} frames for 1 and 2 "
                      f"iterations; the K={K}x{iters} fit and {iters}-iteration projection extrapolated (fit "
                      f"affine in k); sample wall {reps * sum(tk) + p1 + p2:.1f} s"}


def single_problem(args):
    from paper_2309_04623_gb300 import synthetic

    if args.workload == "wide":
        # K = 100 components on the STIS shape (the 64 < k <= 128 kernels for
        # stages 65 .. 100), 100 iterations per stage
        prob = synthetic.make_config(2, n_iter=100)
    else:
        prob = synthetic.make_config(3 if args.workload == "miri" else 1)
    if args.iters:
        prob.n_iter = args.iters
    return prob


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "batched":
        return run_reference_batched(args, world)
    if args.workload == "aux":
        return run_reference_aux(args, world)
    prob = single_problem(args)
    K, iters = prob.K, prob.n_iter
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_reference_sample(prob, iters, K)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median(x["value"] for x in vals)
    step_s = K * iters / v
    flops = workload_flops(prob.N, prob.P, K, iters, prob.M, prob.n_iter)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(prob), "impl": "FP64 C oracle (OpenMP) on the host cores"},
        "tflops": flops / step_s / 1e12,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _workload_name(prob):
    if prob.meta.get("miri"):
        shape = "MIRI-shaped weighted NMF: N={} refs x P={} px (224x288, 4QPM lines + r<5, offsets + read noise)"
    else:
        shape = "STIS-shaped weighted NMF: N={} refs x P={} px (256x256, annulus+wedge+spikes)"
    return (shape.format(prob.N, prob.P) + f", K={prob.K} sequential x {prob.n_iter} it, M={prob.M} frames "
            f"projected ({prob.n_iter} it) + subtracted")


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2309_04623_gb300 import build, nmf, synthetic

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    build.build()
    nmf.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    prob = single_problem(args)
    N, P, K, iters, M = prob.N, prob.P, prob.K, prob.n_iter, prob.M
    if args.precision != "fp32" and K > nmf.tc_max_k():
        raise SystemExit(f"the tensor-core form takes K <= {nmf.tc_max_k()}")
    if args.profile_stage:
        # kernel-capture mode for ncu: only the last stage (k = K from the
        # random start), `--profile-stage` iterations, nothing else
        W, H, c, d = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, args.profile_stage, k_start=K - 1,
                                   normalize=False, precision=args.precision,
                                   polish_iters=0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_stage": True, "k": K, "iterations": int(d[K - 1]), "chi2": float(c[K - 1])}))
        return
    proj_iters = prob.n_iter
    stream = torch.cuda.Stream(device=dev)
    V = torch.from_numpy(prob.V).to(dev)
    Wt = torch.from_numpy(prob.Wt).to(dev)
    W0 = torch.from_numpy(prob.W0).to(dev)
    H0 = torch.from_numpy(prob.H0).to(dev)
    T = torch.from_numpy(prob.T).to(dev)
    WtT = torch.from_numpy(prob.WtT).to(dev)
    C0 = torch.from_numpy(prob.C0).to(dev)
    W = torch.empty_like(W0)
    H = torch.empty_like(H0)
    C = torch.empty_like(C0)
    R = torch.empty_like(T)
    chi2 = torch.zeros(K, dtype=torch.float64, device=dev)
    done = torch.zeros(K, dtype=torch.int32, device=dev)
    prec = nmf.PRECISIONS[args.precision]
    polish = args.polish if prec != nmf.NMF_FP32 else 0
    prm = nmf.make_params(N, P, K, iters, precision=prec, polish_iters=polish)
    ws_fit = nmf.nmf_fit_workspace_bytes(prm)
    ws_proj = nmf.nmf_project_workspace_bytes(M, P, K, prec)
    ws = nmf.workspace(max(ws_fit, ws_proj), dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    sp = nmf._stream(stream)
    p = nmf._ptr

    def step():
        W.copy_(W0)
        H.copy_(H0)
        C.copy_(C0)
        nmf._check(nmf.nmf_fit_basis(p(V), p(Wt), p(W), p(H), p(chi2), p(done), p(ws), ws_fit, prm, sp), "fit")
        nmf._check(nmf.nmf_project_target(p(H), K, P, p(T), p(WtT), M, p(C), proj_iters, 0.0, 1e-30, prec, polish,
                                          p(ws), ws_proj, sp), "project")
        nmf._check(nmf.nmf_subtract(p(T), p(C), p(H), M, K, P, None, p(R), None, 0, None, sp), "subtract")

    with torch.cuda.stream(stream):
        if args.profile:  # launch-list mode for ncu: warm-up steps + one step, nothing else
            for _ in range(args.warmup + 1):
                step()
            stream.synchronize()
            nmf._check(nmf.nmf_workspace_status(p(ws), sp), "device status")
            print(json.dumps({"profile": True, "iters_per_stage": iters, "launches": nmf.nmf_launch_count()}))
            return
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        nmf._check(nmf.nmf_workspace_status(p(ws), sp), "device status")

        sampler = ClockSampler(local_rank)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        launches0 = nmf.nmf_launch_count()
        ms = []
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        launches = nmf.nmf_launch_count() - launches0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        # the step's results, for the comparison with the plain FP32 form
        R_step, C_step, H_step, chi_step = R.clone(), C.clone(), H.clone(), chi2.clone()

        # roofline of the dominant unit: one iteration (H pass + W pass) at
        # k = K, timed live with events on the launching stream from a
        # single-stage fit (k_start = K-1) minus its zero-iteration overhead
        n_rl = 100
        prm_rl = nmf.make_params(N, P, K, n_rl, k_start=K - 1, normalize=False, precision=prec)
        prm_rl0 = nmf.make_params(N, P, K, 0, k_start=K - 1, normalize=False, precision=prec)

        def timed(prmx):
            W.copy_(W0)
            H.copy_(H0)
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            nmf._check(nmf.nmf_fit_basis(p(V), p(Wt), p(W), p(H), p(chi2), p(done), p(ws), ws_fit, prmx, sp), "rl")
            a1.record(stream)
            a1.synchronize()
            return a0.elapsed_time(a1)

        timed(prm_rl)
        t_rl = statistics.median(timed(prm_rl) for _ in range(3))
        t_rl0 = statistics.median(timed(prm_rl0) for _ in range(3))
        it_ms = (t_rl - t_rl0) / n_rl

        # reference selection of the frames (Sec. 4.1): M targets against the
        # N-frame library, the closest half kept (outside the step)
        n_keep = max(1, N // 2)
        dist_sel = torch.empty((M, N), dtype=torch.float64, device=dev)
        idx_sel = torch.empty((M, n_keep), dtype=torch.int32, device=dev)

        def sel():
            nmf._check(nmf.nmf_select_references(p(T), p(WtT), M, p(V), N, P, n_keep, p(dist_sel), p(idx_sel), sp),
                       "select")

        def time_op(fn, reps=5):
            """Median device time of fn on the stream, L2 flushed before each
            call.  The flush (two 256 MB writes, ~80 us) is still running when
            the start event and fn's launch are enqueued, so the interval holds
            the device time of fn alone, not the host's launch latency."""
            fn()
            out_ms = []
            for _ in range(reps):
                torch.cuda.synchronize()
                flush.zero_()
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                out_ms.append(e0.elapsed_time(e1))
            return statistics.median(out_ms)

        sel_ms = time_op(sel)

        # North-up rotation and stacking of the M subtracted frames (Sec. 4.1,
        # 4.2) on the image grid, the masked pixels missing (outside the step)
        ny, nx = prob.img_shape
        grid = torch.full((M, ny * nx), float("nan"), dtype=torch.float32, device=dev)
        grid[:, torch.from_numpy(prob.pix_idx.astype(np.int64)).to(dev)] = R
        valid = torch.zeros(ny * nx, dtype=torch.uint8, device=dev)
        valid[torch.from_numpy(prob.pix_idx.astype(np.int64)).to(dev)] = 1
        ang = synthetic.roll_angles(M)
        rot_out = torch.empty((ny, nx), dtype=torch.float32, device=dev)
        rot_cnt = torch.empty((ny, nx), dtype=torch.int32, device=dev)
        cxy = ((nx - 1) / 2.0, (ny - 1) / 2.0)
        ang_c = ang.ctypes.data_as(ctypes.c_void_p)

        def north_up(method):
            nmf._check(nmf.nmf_derotate_combine(p(grid), M, ny, nx, p(valid), ang_c, cxy[0], cxy[1], method, None,
                                                p(rot_out), p(rot_cnt), sp), "derotate")

        nu_mean = time_op(lambda: north_up(nmf.NMF_COMBINE_MEAN))
        nu_med = time_op(lambda: north_up(nmf.NMF_COMBINE_MEDIAN))
        nu_bytes = M * ny * nx * 4 + ny * nx * (1 + 4 + 4)

        # the metric's comparison: the same step in the plain FP32 form (same
        # inputs, same iteration counts), its time and the agreement of the
        # residual images and of Eq. 2
        fp32_form = None
        if prec != nmf.NMF_FP32 and not args.no_fp32_form:
            prm32 = nmf.make_params(N, P, K, iters, precision=nmf.NMF_FP32)
            ws32_fit = nmf.nmf_fit_workspace_bytes(prm32)
            ws32_proj = nmf.nmf_project_workspace_bytes(M, P, K, nmf.NMF_FP32)

            def step32():
                W.copy_(W0)
                H.copy_(H0)
                C.copy_(C0)
                nmf._check(nmf.nmf_fit_basis(p(V), p(Wt), p(W), p(H), p(chi2), p(done), p(ws), ws32_fit, prm32, sp),
                           "fit fp32")
                nmf._check(nmf.nmf_project_target(p(H), K, P, p(T), p(WtT), M, p(C), proj_iters, 0.0, 1e-30,
                                                  nmf.NMF_FP32, 0, p(ws), ws32_proj, sp), "project fp32")
                nmf._check(nmf.nmf_subtract(p(T), p(C), p(H), M, K, P, None, p(R), None, 0, None, sp),
                           "subtract fp32")

            step32()  # records the FP32 form's graphs
            ms32 = []
            for _ in range(2):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step32()
                e1.record(stream)
                e1.synchronize()
                ms32.append(e0.elapsed_time(e1))
            nmf._check(nmf.nmf_workspace_status(p(ws), sp), "device status fp32")
            relf = lambda a, b: float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))
            fp32_form = {
                "ms_per_step": statistics.mean(ms32), "value": K * iters / (statistics.mean(ms32) / 1e3),
                "unit": UNIT, "speedup_of_this_form": statistics.mean(ms32) / statistics.mean(ms),
                "residual_rel_err_vs_fp32": relf(R_step, R),
                "chi2_rel_err_vs_fp32": float(abs(chi_step[-1] - chi2[-1]) / chi2[-1]),
                "chi2_rel_err_vs_fp32_max_stage": float(((chi_step - chi2).abs() / chi2).max()),
                "H_rel_err_vs_fp32": relf(H_step, H), "C_rel_err_vs_fp32": relf(C_step, C),
            }

    # max over ranks
    step_ms = max_over_ranks(statistics.mean(ms), dist, dev)
    fit_iters = K * iters
    value = job_throughput(fit_iters, world, step_ms)
    flops = workload_flops(N, P, K, iters, M, proj_iters)

    # e2e: the host-buffer C-ABI call (copies inside the timed region)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hV, hWt, hW0, hH0, hT, hWtT, hC0 = (pin(x) for x in (prob.V, prob.Wt, prob.W0, prob.H0, prob.T, prob.WtT,
                                                         prob.C0))
    out = dict(W=pin(np.empty((N, K), np.float32)), H=pin(np.empty((K, P), np.float32)),
               C=pin(np.empty((M, K), np.float32)), R=pin(np.empty((M, P), np.float32)),
               chi2_hist=np.zeros(K), iters_done=np.zeros(K, np.int32))
    rh = dict(precision=args.precision, polish_iters=polish, out=out)
    nmf.reduce_host(hV, hWt, hW0, hH0, hT, hWtT, hC0, iters, proj_iters, **rh)  # warm-up (device cache)
    e2e_s = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nmf.reduce_host(hV, hWt, hW0, hH0, hT, hWtT, hC0, iters, proj_iters, **rh)
        e2e_s.append(time.perf_counter() - t0)
    e2e_val = world * fit_iters / statistics.mean(e2e_s)
    h2d = 4 * (2 * N * P + N * K + K * P + 2 * M * P + M * K)
    d2h = 4 * (N * K + K * P + M * K + M * P) + 8 * K + 4 * K

    pk, pk_kind = peaks()
    mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    it_flops = 12.0 * N * P * K
    if prec == nmf.NMF_FP32:
        # FP32 CUDA-core form: ALU-bound (0.75 k flop/byte against a ~10 flop/byte ridge)
        alu_peak, alu_note = fp32_peak_measured(nmf, mhz)
        achieved_tf = it_flops / (it_ms / 1e3) / 1e12
        roofline = {
            "kernel": f"hpass_f32 + wpass_f32 (one Eq. 3 iteration at k=K={K})",
            "bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved_tf / alu_peak, "traffic": None,
            "peak_note": alu_note,
            "iteration_us": it_ms * 1e3,
        }
    else:
        wbytes = 4 if prec == nmf.NMF_BF16_SPLIT_W32 else 2
        traffic = measured_traffic(args.precision, K) if args.workload in ("stis", "wide") else None
        # tensor-core form: HBM-bound; per element and pass 4 B of V (FP32) + 2 B of Wt (scaled
        # FP16), or 4 B of Wt in the FP32-weights form
        it_bytes = 2.0 * N * P * (4 + wbytes)
        achieved = it_bytes / (it_ms / 1e3) / 1e9
        roofline = {
            "kernel": f"pass_tc_kernel<H> + pass_tc_kernel<W> + wupdate (one Eq. 3 iteration at k=K={K})",
            "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "peak_note": f"HBM copy bandwidth, {pk_kind} (MEASURED_PEAKS hbm_gbs); algorithmic bytes "
                         f"2 passes x N x P x {4 + wbytes} B = {it_bytes / 1e6:.1f} MB per iteration",
            "tensor_tflops": it_flops * 10.0 / 12.0 / (it_ms / 1e3) / 1e12,
            "iteration_us": it_ms * 1e3,
        }

    cpu = None
    cpu_np = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_reference_sample(prob, iters, K)
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"]}
        # the paper's own CPU setup: Eq. 3 as NumPy arithmetic over BLAS
        cpu_np = [cpu_numpy_sample(prob, iters, K, dt) for dt in (np.float64, np.float32)]
    if fp32_form is not None and rank == 0 and not args.no_cpu_baseline:
        # the oracle's projection of a sample of the science frames on this
        # form's basis (every iteration, in FP64), against this form's residuals
        import oracle

        sm = list(range(0, M, max(1, M // 3)))[:3]
        Hb = H_step.double().cpu().numpy()
        Cref = oracle.project(Hb, prob.T[sm], prob.WtT[sm], prob.C0[sm], proj_iters)
        Rref = oracle.subtract(prob.T[sm], Cref, Hb)
        Rb = R_step.double().cpu().numpy()[sm]
        fp32_form["residual_rel_err_vs_oracle_sampled"] = float(np.linalg.norm(Rb - Rref) / np.linalg.norm(Rref))
        fp32_form["oracle_sample"] = (f"science frames {sm}: the FP64 oracle's {proj_iters}-iteration projection "
                                      f"on this form's basis and subtraction")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == nmf.NMF_FP32 else "bf16", "data": "synthetic",
            "config": {"workload": _workload_name(prob),
                       "precision": "fp32 (plain CUDA-core path)" if prec == nmf.NMF_FP32 else
                       f"bf16 tensor cores (tcgen05), split operands, FP32 accumulation and data, "
                       f"{'FP32' if prec == nmf.NMF_BF16_SPLIT_W32 else 'scaled FP16'} weights, {polish} FP32 "
                       f"polish iterations",
                       "l2": "flushed between steps (256 MB write); inputs resident in HBM",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "tflops": flops * world / (step_ms / 1e3) / 1e12,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "cpu_numpy_blas": cpu_np,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "fp32_form": fp32_form,
            "reference_selection": {"ms": sel_ms, "targets": M, "library": N, "n_keep": n_keep,
                                    "l2": "flushed before each call"},
            "north_up": {"frames": M, "shape": [ny, nx], "ms_mean": nu_mean, "ms_median": nu_med,
                         "bytes": nu_bytes, "gbs_mean": nu_bytes / (nu_mean / 1e3) / 1e9,
                         "frac_mean": nu_bytes / (nu_mean / 1e3) / 1e9 / pk["hbm_gbs"],
                         "gbs_median": nu_bytes / (nu_med / 1e3) / 1e9,
                         "l2": "flushed before each call", "launches": 1},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


BATCH_COUNT = 64
BATCH_ITERS = 25  # iterations per stage of every batched reduction (the paper does not fix one)


def batched_problems(args):
    from paper_2309_04623_gb300 import synthetic

    workers = max(1, min(16, os.cpu_count() or 1))
    return synthetic.make_batched(count=BATCH_COUNT, n_iter=args.iters or BATCH_ITERS, workers=workers)


def tc_form(args):
    """The tensor-core form the bench runs: --precision when it names one,
    else the FP32-weights form."""
    return args.precision if args.precision != "fp32" else "bf16w32"


def batched_precisions(probs, tc_k, tc="bf16w32"):
    """Half of the reductions (even index) in the tensor-core form `tc` where
    K allows it, the rest plain FP32."""
    return [tc if (b % 2 == 0 and pr.K <= tc_k) else "fp32" for b, pr in enumerate(probs)]


def batched_name(probs, precs, polish):
    n_bf = sum(p != "fp32" for p in precs)
    return (f"batched: {len(probs)} independent reductions, N in [{min(p.N for p in probs)},"
            f"{max(p.N for p in probs)}], P in [{min(p.P for p in probs)},{max(p.P for p in probs)}], "
            f"K in [{min(p.K for p in probs)},{max(p.K for p in probs)}], M in [{min(p.M for p in probs)},"
            f"{max(p.M for p in probs)}], {probs[0].n_iter} it per stage and projection; {n_bf} in BF16 "
            f"tensor-core form ({'FP32' if 'bf16w32' in precs else 'scaled FP16'} weights, +{polish} FP32 "
            f"polish), {len(probs) - n_bf} plain FP32")


def run_reference_aux(args, world):
    """The oracle on the aux workload (the same inputs as run_aux): each step
    is the reference selection and the rotation with each stacking rule, on
    the host cores, timed whole."""
    import oracle
    from paper_2309_04623_gb300 import synthetic

    prob = synthetic.make_config(1)
    n_keep = prob.N // 2
    grid, valid, ang, cxy = _aux_inputs(prob)
    per = {"select": [], "north_up_mean": [], "north_up_median": []}
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.select(oracle.distances(prob.T, prob.WtT, prob.V), n_keep)
        t1 = time.perf_counter()
        rot = oracle.rotate(grid, ang, cxy, valid=valid)
        t2 = time.perf_counter()
        oracle.combine(rot, "mean")
        t3 = time.perf_counter()
        oracle.combine(rot, "median")
        t4 = time.perf_counter()
        if i >= args.warmup:
            per["select"].append((t1 - t0) * 1e3)
            per["north_up_mean"].append((t3 - t1) * 1e3)
            per["north_up_median"].append((t2 - t1 + t4 - t3) * 1e3)
    ms = {k: statistics.median(v) for k, v in per.items()}
    v = sum(ms.values())
    sample = "the whole step (selection; rotation with each stacking rule), every step"
    line = {
        "impl": "reference", "metric": AUX_METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"STIS-shaped target: {prob.M} science frames, {prob.N}-frame library, {prob.P} "
                               f"pixels, {n_keep} kept; {prob.M} frames of {prob.img_shape[0]}x{prob.img_shape[1]} "
                               f"rotated and stacked", "impl": "FP64 C oracle (OpenMP) on the host cores"},
        "per_op_ms": ms,
        "cpu_baseline": {"value": v, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_batched(args, world):
    """The oracle on a bounded sample of the batched workload: one Eq. 3
    iteration at k = K of three members, timed, and the whole batch
    extrapolated by its flop count (an iteration costs ~12 N P k flops)."""
    import oracle

    probs = batched_problems(args)
    iters = sum(p.K * p.n_iter for p in probs)
    flops = sum(workload_flops(p.N, p.P, p.K, p.n_iter, p.M, p.n_iter) for p in probs)
    vals = []
    for step in range(args.warmup + args.steps):
        t_s, f_s = 0.0, 0.0
        for b in (step % len(probs), (step + 21) % len(probs), (step + 42) % len(probs)):
            pr = probs[b]
            t0 = time.perf_counter()
            oracle.iterate(pr.V, pr.Wt, pr.W0, pr.H0, 1)
            t_s += time.perf_counter() - t0
            f_s += 12.0 * pr.N * pr.P * pr.K
        if step >= args.warmup:
            vals.append(iters / (flops * t_s / f_s))
    v = statistics.median(vals)
    sample = (f"one oracle iteration at k=K of 3 members per step, batch time extrapolated by flops "
              f"({flops / 1e12:.1f} TFLOP per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": iters / v * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batched_name(probs, ["fp64"] * len(probs), 0),
                   "impl": "FP64 C oracle (OpenMP) on the host cores"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local_rank):
    """64 uneven reductions in one nmf_fit_batched call per step."""
    probs = batched_problems(args)  # spawned generator pool, before any CUDA work
    import torch

    from paper_2309_04623_gb300 import build, nmf

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    build.build()
    nmf.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    precs = batched_precisions(probs, nmf.tc_max_k(), tc_form(args))
    polish = args.polish
    stream = torch.cuda.Stream(device=dev)
    d = lambda a: torch.from_numpy(a).to(dev)
    bufs, descs = [], []
    for pr, pc in zip(probs, precs):
        b = dict(V=d(pr.V), Wt=d(pr.Wt), W0=d(pr.W0), H0=d(pr.H0), T=d(pr.T), WtT=d(pr.WtT), C0=d(pr.C0))
        b.update(W=b["W0"].clone(), H=b["H0"].clone(), C=b["C0"].clone(), R=torch.empty_like(b["T"]),
                 chi2=torch.zeros(pr.K, dtype=torch.float64, device=dev),
                 done=torch.zeros(pr.K, dtype=torch.int32, device=dev))
        q = nmf.nmf_problem()
        q.V, q.Wt, q.W, q.H = (b[x].data_ptr() for x in ("V", "Wt", "W", "H"))
        q.chi2_hist, q.iters_done = b["chi2"].data_ptr(), b["done"].data_ptr()
        q.prm = nmf.make_params(pr.N, pr.P, pr.K, pr.n_iter, precision=pc,
                                polish_iters=polish if pc != "fp32" else 0)
        q.T, q.WtT, q.C, q.R = (b[x].data_ptr() for x in ("T", "WtT", "C", "R"))
        q.M, q.proj_iters = pr.M, pr.n_iter
        bufs.append(b)
        descs.append(q)
    need = nmf.nmf_batched_workspace_bytes(descs)
    if need == 0:
        raise SystemExit("invalid batched descriptors")
    ws = nmf.workspace(need, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sp = nmf._stream(stream)

    def reset():
        for b in bufs:
            b["W"].copy_(b["W0"])
            b["H"].copy_(b["H0"])
            b["C"].copy_(b["C0"])

    def step():
        reset()
        nmf._check(nmf.nmf_fit_batched(descs, nmf._ptr(ws), need, sp), "nmf_fit_batched")

    fit_iters = sum(p.K * p.n_iter for p in probs)
    flops = sum(workload_flops(p.N, p.P, p.K, p.n_iter, p.M, p.n_iter) for p in probs)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        code, _ = nmf.nmf_batched_status(descs, nmf._ptr(ws), sp)
        nmf._check(code, "batched device status")
        sampler = ClockSampler(local_rank)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        launches0 = nmf.nmf_launch_count()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        launches = nmf.nmf_launch_count() - launches0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        code, _ = nmf.nmf_batched_status(descs, nmf._ptr(ws), sp)
        nmf._check(code, "batched device status")
        got_R = [b["R"].clone() for b in bufs]
        got_chi2 = [b["chi2"].clone() for b in bufs]

        # the same reductions one after the other in plain FP32 (separate calls)
        seq = None
        if not args.no_sequential:
            descs32 = []
            for q, pr in zip(descs, probs):
                q32 = nmf.nmf_problem.from_buffer_copy(q)
                q32.prm = nmf.make_params(pr.N, pr.P, pr.K, pr.n_iter)
                descs32.append(q32)
            ws_fit = [nmf.nmf_fit_workspace_bytes(q.prm) for q in descs32]
            ws_proj = [nmf.nmf_project_workspace_bytes(q.M, q.prm.P, q.prm.K, 0) for q in descs32]
            ws32 = nmf.workspace(max(max(ws_fit), max(ws_proj)), dev)
            p = nmf._ptr

            def seq_step():
                reset()
                for q, b, wf, wp in zip(descs32, bufs, ws_fit, ws_proj):
                    nmf._check(nmf.nmf_fit_basis(q.V, q.Wt, q.W, q.H, q.chi2_hist, q.iters_done, p(ws32), wf,
                                                 q.prm, sp), "fit")
                    nmf._check(nmf.nmf_project_target(q.H, q.prm.K, q.prm.P, q.T, q.WtT, q.M, q.C, q.proj_iters,
                                                      0.0, 1e-30, 0, 0, p(ws32), wp, sp), "project")
                    nmf._check(nmf.nmf_subtract(q.T, q.C, q.H, q.M, q.prm.K, q.prm.P, None, q.R, None, 0, None,
                                                sp), "subtract")

            seq_step()  # records the per-call graphs
            stream.synchronize()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            seq_step()
            e1.record(stream)
            e1.synchronize()
            seq_ms = e0.elapsed_time(e1)
            # residual agreement of every member with its plain-FP32 run
            errs = []
            for b, r, pc in zip(bufs, got_R, precs):
                errs.append(float(torch.linalg.norm((r - b["R"]).double()) /
                                  torch.linalg.norm(b["R"].double()).clamp_min(1e-300)))
            bf_err = [e for e, pc in zip(errs, precs) if pc != "fp32"]
            # members of the precision form beyond 1e-3: how far the problem
            # itself moves when the FP32 form starts from factors changed by
            # one part in 10^6 (an ill-conditioned member moves that much
            # under any rounding)
            over = []
            for bi, (pr, pc, e) in enumerate(zip(probs, precs, errs)):
                if pc == "fp32" or e <= 1e-3:
                    continue
                rng = np.random.default_rng(12345)
                pert = lambda x: (x * (1 + 1e-6 * rng.uniform(-1, 1, x.shape))).astype(np.float32)
                Wp, Hp, _, _ = nmf.fit_basis(pr.V, pr.Wt, pert(pr.W0), pert(pr.H0), pr.n_iter, stream=stream)
                Cp = nmf.project_target(Hp, pr.T, pr.WtT, pert(pr.C0), pr.n_iter, stream=stream)
                Rp = nmf.subtract(pr.T, Cp, Hp, stream=stream)
                stream.synchronize()
                Rf = bufs[bi]["R"]
                s_err = float(torch.linalg.norm((Rp - Rf).double()) / torch.linalg.norm(Rf.double()))
                over.append({"member": bi, "N": pr.N, "P": pr.P, "K": pr.K, "residual_rel_err_vs_fp32": e,
                             "fp32_sensitivity_1e-6": s_err})
            seq = {"ms_per_step": seq_ms, "value": fit_iters / (seq_ms / 1e3), "unit": UNIT,
                   "speedup_batched": seq_ms / statistics.mean(ms),
                   "residual_rel_err_bf16_vs_fp32_max": max(bf_err) if bf_err else None,
                   "residual_rel_err_bf16_vs_fp32_median": statistics.median(bf_err) if bf_err else None,
                   "bf16_members_within_1e-3": sum(e <= 1e-3 for e in bf_err),
                   "bf16_members": len(bf_err),
                   "bf16_members_beyond_1e-3": over,
                   "residual_rel_err_fp32_members_max": max((e for e, pc in zip(errs, precs) if pc == "fp32"),
                                                            default=None)}

    step_ms = max_over_ranks(statistics.mean(ms), dist, dev)
    value = job_throughput(fit_iters, world, step_ms)

    # e2e: the public Python call on host (numpy) inputs, results read back
    batch_np = [dict(V=pr.V, Wt=pr.Wt, W0=pr.W0, H0=pr.H0, T=pr.T, WtT=pr.WtT, C0=pr.C0, precision=pc,
                     polish_iters=polish if pc != "fp32" else 0, iters_per_stage=pr.n_iter, proj_iters=pr.n_iter)
                for pr, pc in zip(probs, precs)]
    e2e_s = []
    for i in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = nmf.fit_batched(batch_np, 0, 0, stream=stream)
        host = [(o["W"].cpu(), o["H"].cpu(), o["C"].cpu(), o["R"].cpu()) for o in out]
        if i:
            e2e_s.append(time.perf_counter() - t0)
        del host, out
    e2e_val = world * fit_iters / statistics.mean(e2e_s)
    h2d = sum(4 * (2 * p.N * p.P + p.N * p.K + p.K * p.P + 2 * p.M * p.P + p.M * p.K) for p in probs)
    d2h = sum(4 * (p.N * p.K + p.K * p.P + p.M * p.K + p.M * p.P) for p in probs)

    pk, pk_kind = peaks()
    mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    # roofline time of the step: per member and iteration, the slower of its
    # algorithmic bytes over HBM and its flops at its form's peak
    t_roof = 0.0
    alg_bytes = 0.0
    fp32_pk, fp32_note = fp32_peak_measured(nmf, mhz)
    for pr, pc in zip(probs, precs):
        for k in range(1, pr.K + 1):
            bts = 2.0 * pr.N * pr.P * (6 if pc == "bf16" else 8)
            fl = 12.0 * pr.N * pr.P * k
            peak_f = pk["bf16_tflops_sustained"] * 1e12 if pc != "fp32" else fp32_pk * 1e12
            t_roof += pr.n_iter * max(bts / (pk["hbm_gbs"] * 1e9), fl / peak_f)
            alg_bytes += pr.n_iter * bts
    achieved = alg_bytes / (step_ms / 1e3) / 1e9
    roofline = {
        "kernel": "whole batched step (fit stages; projection and subtraction excluded from the roof)",
        "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
        "frac": t_roof / (step_ms / 1e3), "traffic": None,
        "peak_note": f"frac = roofline time / step time; roofline time = sum over members and iterations of "
                     f"max(bytes / HBM ({pk_kind}), flops / peak of the member's form: bf16 sustained "
                     f"({pk_kind}) or FP32 CUDA-core: {fp32_note})",
        "roofline_ms": t_roof * 1e3,
    }
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": batched_name(probs, precs, polish),
                       "l2": "flushed between steps (256 MB write); inputs resident in HBM",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "tflops": flops * world / (step_ms / 1e3) / 1e12,
            "roofline": roofline,
            "sequential_fp32": seq,
            "cpu_baseline": None,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "final_chi2_sum": float(sum(c[-1].item() for c in got_chi2)),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# The paper's Table 2 (Sec. 5.4): whole NMF reductions, CPU against GPU
# (CuPy), hardware, data and iteration counts not stated.  Context only.
PAPER_TABLE2 = {10: (210, 273), 30: (1162, 425), 50: (4776, 1135), 70: (11676, 2609), 90: (18471, 3852),
                110: (30610, 5907)}


def run_table2(args, rank, world, local_rank):
    """Synthetic analogue of Table 2: end-to-end wall time of one reduction
    (host arrays in, residual images out: transfers, the sequential fit of K
    components, the projection and the subtraction) for K = 10 ... 110 on the
    STIS-shaped data, tensor-core form and plain FP32 form on the GPU, and the
    FP64 oracle on the host cores (sampled and extrapolated)."""
    import torch

    from paper_2309_04623_gb300 import build, nmf, synthetic

    if rank != 0:
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    build.build()
    nmf.load()
    iters = args.iters or 100
    rows = []
    for K in (10, 30, 50, 70, 90, 110):
        prob = synthetic.make_config(1, K=K, n_iter=iters)
        row = {"K": K, "iters_per_stage": iters}
        for key, prec, pol in (("bf16", tc_form(args), args.polish), ("fp32", "fp32", 0)):
            kw = dict(precision=prec, polish_iters=pol)
            nmf.reduce_host(prob.V, prob.Wt, prob.W0, prob.H0, prob.T, prob.WtT, prob.C0, iters, iters, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nmf.reduce_host(prob.V, prob.Wt, prob.W0, prob.H0, prob.T, prob.WtT, prob.C0, iters, iters, **kw)
            row[f"gpu_{key}_s"] = time.perf_counter() - t0
        if not args.no_cpu_baseline:
            r = cpu_reference_sample(prob, iters, K)
            row["cpu_oracle_s"] = r["seconds_full_est"]
            row["cpu_cores"] = r["cores"]
            row["speedup_bf16_vs_cpu"] = row["cpu_oracle_s"] / row["gpu_bf16_s"]
        row["speedup_bf16_vs_fp32"] = row["gpu_fp32_s"] / row["gpu_bf16_s"]
        row["paper_cpu_s"], row["paper_gpu_s"] = PAPER_TABLE2[K]
        rows.append(row)
        print(json.dumps(row), flush=True)
    total_iters = sum(r["K"] * iters for r in rows)
    total_bf16 = sum(r["gpu_bf16_s"] for r in rows)
    line = {
        "metric": METRIC, "value": total_iters / total_bf16, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": total_bf16 * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"Table 2 analogue: one STIS-shaped reduction (N=300, P=49343, M=50) per K in "
                               f"10..110, {iters} it per stage and projection, end to end from host arrays"},
        "table2": rows,
    }
    print(json.dumps(line), flush=True)


AUX_METRIC = "reference selection and North-up stacking per target, ms (STIS-shaped)"


def _aux_inputs(prob):
    """The North-up step's frames for the STIS-shaped target: science minus
    library frames scattered to the image grid (masked pixels NaN), the mask,
    the roll angles and the rotation centre."""
    from paper_2309_04623_gb300 import synthetic

    M = prob.M
    ny, nx = prob.img_shape
    grid = np.full((M, ny * nx), np.nan, dtype=np.float32)
    grid[:, prob.pix_idx] = (prob.T - prob.V[:M]).astype(np.float32)
    valid = np.zeros(ny * nx, dtype=np.uint8)
    valid[prob.pix_idx] = 1
    return grid.reshape(M, ny, nx), valid.reshape(ny, nx), synthetic.roll_angles(M), ((nx - 1) / 2.0, (ny - 1) / 2.0)


def run_aux(args, rank, world, local_rank):
    """The steps around the fit on the STIS-shaped target (Sec. 4.1, 4.2):
    reference selection of the 300-frame library for the 50 science frames
    (the 150 closest kept), then North-up rotation and stacking of the 50
    subtracted frames on the 256 x 256 grid (mean, and median).  One step =
    the three calls, each timed alone with the L2 flushed before it; the
    frames to rotate are science-minus-library differences scattered to the
    grid with the mask's pixels missing (their values do not change the
    work).  Rank 0 only."""
    import torch

    import oracle
    from paper_2309_04623_gb300 import build, nmf, synthetic

    if rank != 0:
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    build.build()
    nmf.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    prob = synthetic.make_config(1)
    M, N, P = prob.M, prob.N, prob.P
    ny, nx = prob.img_shape
    n_keep = N // 2
    T = torch.from_numpy(prob.T).to(dev)
    WtT = torch.from_numpy(prob.WtT).to(dev)
    V = torch.from_numpy(prob.V).to(dev)
    grid_h, valid_h, ang, cxy = _aux_inputs(prob)
    grid = torch.from_numpy(grid_h).to(dev)
    valid = torch.from_numpy(valid_h).to(dev)
    ang_c = ang.ctypes.data_as(ctypes.c_void_p)
    dist_sel = torch.empty((M, N), dtype=torch.float64, device=dev)
    idx_sel = torch.empty((M, n_keep), dtype=torch.int32, device=dev)
    out = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    cnt = torch.empty((ny, nx), dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)
    sp = nmf._stream(stream)
    p = nmf._ptr
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def sel():
        nmf._check(nmf.nmf_select_references(p(T), p(WtT), M, p(V), N, P, n_keep, p(dist_sel), p(idx_sel), sp),
                   "select")

    def north_up(method):
        nmf._check(nmf.nmf_derotate_combine(p(grid), M, ny, nx, p(valid), ang_c, cxy[0], cxy[1], method, None, p(out),
                                            p(cnt), sp), "derotate")

    ops = (("select", sel), ("north_up_mean", lambda: north_up(nmf.NMF_COMBINE_MEAN)),
           ("north_up_median", lambda: north_up(nmf.NMF_COMBINE_MEDIAN)))

    def one(fn):
        # the two flushes are still running while the start event and fn's
        # launch are enqueued: the interval is fn's device time alone
        torch.cuda.synchronize()
        flush.zero_()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            for _, fn in ops:
                one(fn)
        sampler = ClockSampler(local_rank)
        sampler.start()
        launches0 = nmf.nmf_launch_count()
        times = {name: [] for name, _ in ops}
        t_start = time.perf_counter()
        steps = 0
        # at least --steps steps, and at least 1.5 s so the clock sampler sees the region
        while steps < args.steps or time.perf_counter() - t_start < 1.5:
            for name, fn in ops:
                times[name].append(one(fn))
            steps += 1
        launches = nmf.nmf_launch_count() - launches0
        clocks = sampler.stop()
    ms = {k: statistics.mean(v) for k, v in times.items()}
    step_ms = sum(ms.values())

    pk, pk_kind = peaks()
    mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    alu_peak, alu_note = fp32_peak_measured(nmf, mhz)
    sel_flops = 4.0 * M * N * P  # per pixel and pair: subtract, multiply, fused multiply-add
    nu_bytes = M * ny * nx * 4 + ny * nx * (1 + 4 + 4)
    kernels = {
        "select": {
            "ms": ms["select"], "targets": M, "library": N, "pixels": P, "n_keep": n_keep,
            "roofline": {"kernel": "distances_kernel (+ select_kernel)", "bound": "alu",
                         "achieved": sel_flops / (ms["select"] / 1e3) / 1e12, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": sel_flops / (ms["select"] / 1e3) / 1e12 / alu_peak,
                         "traffic": None,
                         "peak_note": f"FP32 CUDA-core peak: {alu_note}; 4 flop in 3 instructions per term, so the "
                                      f"instruction mix caps frac at 0.67"},
        },
    }
    for name in ("north_up_mean", "north_up_median"):
        gbs = nu_bytes / (ms[name] / 1e3) / 1e9
        kernels[name] = {
            "ms": ms[name], "frames": M, "shape": [ny, nx],
            "roofline": {"kernel": f"rotate_kernel<{'mean' if name.endswith('mean') else 'median'}>",
                         "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / pk["hbm_gbs"], "traffic": None,
                         "peak_note": f"HBM copy bandwidth, {pk_kind}; algorithmic bytes: the frames once, the "
                                      f"mask, the stacked image and the counts = {nu_bytes / 1e6:.1f} MB"},
        }

    cpu = None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        D = oracle.distances(prob.T, prob.WtT, prob.V)
        oracle.select(D, n_keep)
        t1 = time.perf_counter()
        t2 = time.perf_counter()
        rot = oracle.rotate(grid_h, ang, cxy, valid=valid_h)
        t3 = time.perf_counter()
        oracle.combine(rot, "mean")
        t4 = time.perf_counter()
        oracle.combine(rot, "median")
        t5 = time.perf_counter()
        cpu_ms = {"select": (t1 - t0) * 1e3, "north_up_mean": (t4 - t2) * 1e3,
                  "north_up_median": ((t3 - t2) + (t5 - t4)) * 1e3}
        cpu = {"value": sum(cpu_ms.values()), "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "the whole step once (selection; rotation with each stacking rule)", "per_op_ms": cpu_ms}

    line = {
        "metric": AUX_METRIC,
        "value": step_ms, "unit": "ms", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"STIS-shaped target: {M} science frames, {N}-frame library, {P} pixels, "
                               f"{n_keep} kept; {M} frames of {ny}x{nx} rotated and stacked",
                   "l2": "flushed before each call (two 256 MB writes); inputs resident in HBM"},
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": launches, "launches_per_step": launches / steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16w32"], default="bf16w32",
                    help="bf16w32: tensor-core form with FP32 weights and FP32 polish (default); bf16: the same "
                         "with the weights streamed as scaled FP16; fp32: plain CUDA-core form")
    ap.add_argument("--polish", type=int, default=20, help="FP32 polish iterations of the split form")
    ap.add_argument("--iters", type=int, default=0,
                    help="iterations per stage (default: the workload's 500); for profiling only")
    ap.add_argument("--workload", choices=["stis", "miri", "wide", "batched", "table2", "aux"], default="stis",
                    help="stis: one STIS-shaped reduction (default); miri: one MIRI-shaped reduction; "
                         "wide: the STIS shape at K = 100, 100 it per stage; "
                         "batched: 64 uneven reductions in one call; table2: end-to-end wall time per K = 10..110; "
                         "aux: reference selection and North-up stacking of the STIS-shaped target")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="stis/miri in the BF16 form: skip the timed plain-FP32 comparison run")
    ap.add_argument("--no-sequential", action="store_true",
                    help="batched: skip the sequential plain-FP32 comparison run")
    ap.add_argument("--profile-stage", type=int, default=0,
                    help="run only the last stage (k = K) for this many iterations and exit (for ncu captures)")
    ap.add_argument("--profile", action="store_true",
                    help="run warm-up steps and one step and print only the launch count (for ncu)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "table2":
        run_table2(args, rank, world, local_rank)
    elif args.workload == "aux":
        run_aux(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
