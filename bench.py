"""Benchmark: two-site DMRG steps at chi = 1024 (XXZ chain, L = 128, d = 2, w = 5).

A step is one pass of the whole hot path at a saturated bulk bond: theta
formation, Lanczos on H_eff (each iteration one H_eff.theta product plus
float64 reorthogonalisation), the float64 Gram/eigendecomposition split with
truncation, and the environment update. Steps walk the orthogonality centre
to the right from bond 40, so every timed step is a genuine step of a sweep.

Reported value: credited H_eff.theta FLOPs executed in the timed steps
divided by the timed wall time (logical TFLOP/s; identity environment
channels are not credited). Also reported: ms per step, a full left-right-
left sweep at chi_max = 1024 (seconds), the plain float64 GPU path on the same
steps, the roofline of the dominant kernel (tcgen05 GEMM, timed per launch
with CUDA events on its stream), an end-to-end number through the C ABI with
host buffers, and the CPU oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_SITES, D, W_MPO, CHI = 128, 2, 5, 1024
CENTER0 = 40
LANCZOS_CAP, LANCZOS_TOL = 20, 1e-10
WORKLOAD = ("XXZ chain J=1 Delta=1, L=128, d=2, MPO w=5, chi_max=1024: two-site DMRG steps "
            "at saturated bulk bonds (theta, Lanczos on H_eff.theta, Gram/eig split, env update)")
METRIC = "H_eff.theta TFLOP/s at chi=1024 within DMRG steps (XXZ L=128); sweep seconds reported alongside"
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense tensor ratio


def heff_credited_flops(chi_l, chi_r, d1=D, d2=D, wl=W_MPO, wm=W_MPO, wr=W_MPO):
    """Algorithmic FLOPs of one H_eff.theta: the two GEMM stages without the
    identity channel of L (last) and of R (first), plus the two W-steps."""
    nl, nr = max(wl - 1, 1), max(wr - 1, 1)
    return (2.0 * d1 * d2 * chi_l * chi_r * (nl * chi_l + nr * chi_r)
            + 2.0 * chi_l * chi_r * d1 * d2 * (d1 * wl * wm + d2 * wm * wr))


def heff_gemm_credited_flops(chi_l, chi_r, d1=D, d2=D, wl=W_MPO, wr=W_MPO):
    """The two GEMM stages of one H_eff.theta without the identity channels."""
    nl, nr = max(wl - 1, 1), max(wr - 1, 1)
    return 2.0 * d1 * d2 * chi_l * chi_r * (nl * chi_l + nr * chi_r)


def step_gemm_credited_flops(chi_l, chi_m, chi_r, iters, d=D, w=W_MPO):
    """Credited tensor-core GEMM work of one left-to-right step: the H_eff.theta
    GEMM stages of every Lanczos product, theta = A_k A_(k+1), and the two GEMMs
    of the left environment update (identity channel not credited)."""
    theta = 2.0 * chi_l * d * chi_m * d * chi_r
    env = 2.0 * d * chi_l * chi_m * ((w - 1) * chi_l + (w - 1) * chi_m)
    return iters * heff_gemm_credited_flops(chi_l, chi_r) + theta + env


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, max, throttle reasons) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier_max(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_sum(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm only)
# ---------------------------------------------------------------------------
def oracle_step_sample(seed=0):
    """One oracle two-site step at chi=1024 on seeded symmetric environments:
    theta formation, Lanczos (same cap), eigendecomposition split, env update.
    Returns (seconds, credited FLOPs, iterations)."""
    from oracle import dmrg as od
    from oracle import mpo as ompo
    from paper_1703_00387_gb300 import inputs
    W = ompo.xxz_mpo(L_SITES, 1.0, 1.0, 0.0)
    k = CENTER0
    Lenv = inputs.random_symmetric_env(CHI, W_MPO, seed=seed)
    Renv = inputs.random_symmetric_env(CHI, W_MPO, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    A1 = rng.standard_normal((CHI, D, CHI // 2))
    A2 = rng.standard_normal((CHI // 2, D, CHI))
    t0 = time.perf_counter()
    theta = np.tensordot(A1, A2, axes=([2], [0]))
    mv = lambda x: od.heff_apply(Lenv, W[k], W[k + 1], Renv, x)
    e, theta, iters, _ = od.lanczos_ground(mv, theta, LANCZOS_CAP, LANCZOS_TOL)
    a, b, info = od.split_eig(theta, CHI, 1e-12 / (4 * L_SITES), True)
    od.env_left(Lenv, a, W[k])
    dt = time.perf_counter() - t0
    return dt, iters * heff_credited_flops(CHI, CHI), iters


def cpu_threads():
    return os.cpu_count()


def blas_threads():
    """Threads of the BLAS under NumPy: threadpoolctl where installed, else the
    thread count the OpenBLAS bundled with NumPy reports, else the usual
    environment variables, else None (unknown)."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    try:
        import ctypes
        with open("/proc/self/maps") as f:
            libs = {ln.split()[-1] for ln in f
                    if "openblas" in os.path.basename(ln.split()[-1]).lower() and ".so" in ln}
        for path in sorted(libs):
            lib = ctypes.CDLL(path)
            for sym in ("scipy_openblas_get_num_threads64_", "openblas_get_num_threads64_",
                        "openblas_get_num_threads"):
                fn = getattr(lib, sym, None)
                if fn is not None:
                    return int(fn())
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return None


def run_reference(args, ws, rank):
    if rank != 0:
        return
    for i in range(args.warmup):
        oracle_step_sample(seed=100 + i)
    total_t, total_f = 0.0, 0.0
    for i in range(args.steps):
        dt, f, _ = oracle_step_sample(seed=i)
        total_t += dt
        total_f += f
    value = total_f / total_t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "chi": CHI, "L": L_SITES, "lanczos_cap": LANCZOS_CAP},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_threads(),
                         "blas_threads": blas_threads(), "kind": "oracle",
                         "sample": "per step: one FP64 NumPy two-site step at chi=1024 on seeded "
                                   "symmetric environments"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, ws, rank, local):
    import torch
    from paper_1703_00387_gb300 import binding as B
    from paper_1703_00387_gb300 import hamiltonians, inputs

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    B.lib()  # raises if the library is missing: no fallback
    stream = torch.cuda.current_stream()
    ctx = B.Context(local)
    prec = args.precision
    Wh = hamiltonians.xxz(L_SITES, 1.0, 1.0, 0.0)
    mpo = B.MPO(ctx, Wh)
    mps = B.MPS(ctx, inputs.random_mps(L_SITES, D, CHI, seed=rank), chi_cap=CHI)
    B.osmps_mps_canonicalize(ctx, mps, mpo, CENTER0, prec)
    params = B.sweep_params(CHI, 1, prec, lanczos_tol=LANCZOS_TOL, lanczos_max_iter=LANCZOS_CAP)

    k = CENTER0
    for _ in range(args.warmup):
        B.osmps_sweep_step(ctx, mps, mpo, k, 1, params)
        k += 1
    torch.cuda.synchronize()
    barrier(ws)
    sampler = ClockSampler(local)
    sampler.start()
    B.osmps_profile_enable(ctx, True)
    launches0 = B.osmps_kernel_launches()
    torch.cuda.synchronize()
    barrier(ws)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # a profiler started with capture off records the timed steps only
    ev0.record(stream)
    flops, gemm_flops, iters = 0.0, 0.0, []
    for _ in range(args.steps):
        out = B.osmps_sweep_step(ctx, mps, mpo, k, 1, params)
        chi = mps.bond_dims()
        flops += out["iters"] * heff_credited_flops(chi[k], chi[k + 2])
        gemm_flops += step_gemm_credited_flops(chi[k], chi[k + 1], chi[k + 2], out["iters"])
        iters.append(out["iters"])
        k += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier(ws)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = B.osmps_kernel_launches() - launches0
    prof = B.osmps_profile_read(ctx, "gemm_tc")
    prof_other = {k: B.osmps_profile_read(ctx, k) for k in ("sytrd_panel", "gemm_emu", "gemm_f64")}
    B.osmps_profile_enable(ctx, False)
    clocks = sampler.stop()
    t_max = barrier_max(elapsed, ws)
    flops_all = barrier_sum(flops, ws)
    value = flops_all / t_max / 1e12

    peaks, peak_src = load_peaks()
    peak_bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    peak = peak_bf16 * (TF32_OVER_BF16 if prec == "tf32x3" else 1.0)
    # credited work (identity channels excluded), per the kernel's own CUDA-event time;
    # the x3 split issues three tensor products per credited one
    gemm_s = prof["ms"] / 1e3
    logical = gemm_flops / gemm_s / 1e12 if gemm_s > 0 else None
    issued = 3.0 * logical if logical else None
    dense_issued = prof["tensor_flops"] / gemm_s / 1e12 if gemm_s > 0 else None
    roofline = {"kernel": "k_gemm_tc (tcgen05 split-precision GEMM)", "bound": "tensor",
                "achieved": issued, "peak": peak, "unit": "TFLOP/s",
                "frac": (issued / peak) if issued else None,
                "achieved_basis": "3 x credited FLOPs (identity environment channels not credited) "
                                  "per CUDA-event second of the kernel",
                "achieved_logical": logical, "frac_logical": (logical / peak) if logical else None,
                "achieved_dense_issued": dense_issued,
                "frac_dense_issued": (dense_issued / peak) if dense_issued else None,
                "peak_source": f"{peak_src} bf16_tflops_sustained" + (" x 1.1/2.25 (tf32)" if prec == "tf32x3" else ""),
                "launches": prof["launches"],
                "avg_launch_ms": prof["ms"] / max(prof["launches"], 1),
                "share_of_step_time": prof["ms"] / 1e3 / elapsed if elapsed > 0 else None,
                "traffic": traffic_per_launch(prof)}

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (contractions " + prec + ")",
        "data": "synthetic (seeded random MPS, XXZ MPO)",
        "config": {"workload": WORKLOAD, "chi": CHI, "L": L_SITES, "d": D, "w": W_MPO,
                   "precision": prec, "lanczos_cap": LANCZOS_CAP, "lanczos_tol": LANCZOS_TOL,
                   "lanczos_iters": iters, "l2": "inputs larger than L2 (each step streams ~1 GB: "
                                                 "20 Krylov vectors of 33.5 MB, 42 MB environments)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline, "step_roofline": step_roofline(prof_other, elapsed, peaks, peak_src),
        "tile_tuning": ctx.tuning(),
        "clocks": clocks, "gpu_launches": launches,
    }

    if rank == 0 and not args.quick:
        line["fp64_gpu"] = fp64_leg(B, ctx, mps, mpo, k, args)
        k = line["fp64_gpu"].pop("_k")
        line["fp64emu_gpu"] = fp64_leg(B, ctx, mps, mpo, k, args, prec="fp64emu")
        k = line["fp64emu_gpu"].pop("_k")
        line["fp64emu_gpu"]["note"] = ("float64-accurate contractions emulated on the bf16 tensor "
                                       "cores (the refinement-sweep precision)")
        line["e2e"] = e2e_leg(B, ctx, Wh, prec, args)
        if not args.no_sweep:
            line["sweep_s"] = sweep_leg(B, ctx, mpo, prec)
            line["time_to_accuracy"] = accuracy_leg(B, ctx, args)
        if not args.no_batch:
            line["batch_sweeps"] = batch_leg(B, args)
        line["u1_heff"] = u1_leg(B, ctx, args)
        line["u1_sweep"] = u1_sweep_leg(B, ctx, args)
        line["long_range_sweep"] = long_range_leg(B, ctx, args)
        line["excited_state"] = excited_leg(B, ctx, args)
        line["tdvp"] = tdvp_leg(B, ctx, args)
        line["gradients"] = grad_leg(B, ctx, args)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], line["matvec_rel_err"] = cpu_leg(B, ctx, Wh)
    mps.close()
    mpo.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


# nominal float64 rate of a GB300 (CUDA cores and DMMA alike): 152 SMs x
# 2 FMA per clock x 2.07 GHz ~ 1.26 TFLOP/s; no measured float64 peak exists
FP64_NOMINAL_TFLOPS = 1.25


def step_roofline(prof, elapsed, peaks, peak_src):
    """Per-kernel rooflines over the timed steps for the kernels the library
    times with CUDA events: the Householder panel of the split's
    tridiagonalisation (float64 CUDA-core arithmetic, algorithmic FLOPs of
    the panel's A22 v products and corrections), the emulated-FP64 GEMM
    (Gram, projections and trailing updates of the split; logical float64
    FLOPs against the bf16 tensor peak / 36 slice products) and the float64
    DMMA GEMM. The entry with the largest share of the step is the
    step-level bound."""
    out = {}
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    specs = {"sytrd_panel": ("k_sytrd_panel (cooperative Householder panel)", "alu", FP64_NOMINAL_TFLOPS,
                             "nominal float64 1.25 TFLOP/s"),
             "gemm_emu": ("k_gemm_emu (float64-accurate GEMM on bf16 tensor cores)", "tensor", bf16 / 36.0,
                          f"{peak_src} bf16_tflops_sustained / 36 slice products"),
             "gemm_f64": ("k_gemm_f64 / k_gemm_grouped (float64 DMMA)", "alu", FP64_NOMINAL_TFLOPS,
                          "nominal float64 1.25 TFLOP/s")}
    for key, (name, bound, peak, src) in specs.items():
        p = prof[key]
        if p["launches"] == 0 or p["ms"] <= 0:
            continue
        ach = p["flops"] / (p["ms"] / 1e3) / 1e12
        out[key] = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "peak_source": src, "launches": p["launches"],
                    "ms_total": p["ms"], "share_of_step_time": p["ms"] / 1e3 / elapsed if elapsed > 0 else None}
    if out:
        out["dominant"] = max((k for k in out), key=lambda k: out[k]["share_of_step_time"] or 0.0)
    return out


def traffic_per_launch(prof):
    """DRAM bytes per launch of k_gemm_tc from the committed ncu summary, if the
    kernel source is unchanged since it was taken (else null)."""
    p = os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")
    src = os.path.join(ROOT, "paper_1703_00387_gb300", "csrc", "gemm_tc.cu")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if d.get("gemm_tc_sha256") != h:
        return None
    return d.get("bytes_per_launch")


def fp64_leg(B, ctx, mps, mpo, k, args, prec="fp64"):
    import torch
    params = B.sweep_params(CHI, 1, prec, lanczos_tol=LANCZOS_TOL, lanczos_max_iter=LANCZOS_CAP)
    B.osmps_sweep_step(ctx, mps, mpo, k, 1, params)  # warm-up
    k += 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    flops, n = 0.0, args.fp64_steps
    for _ in range(n):
        out = B.osmps_sweep_step(ctx, mps, mpo, k, 1, params)
        chi = mps.bond_dims()
        flops += out["iters"] * heff_credited_flops(chi[k], chi[k + 2])
        k += 1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "ms_per_step": 1e3 * dt / n, "steps": n,
            "_k": k}


def e2e_leg(B, ctx, Wh, prec, args):
    """The same step through the standalone C-ABI calls with inputs in pinned
    host memory: copies host->device, theta, Lanczos, split, env update, and
    device->host copies of the new site tensors, environment and energy."""
    import torch
    from paper_1703_00387_gb300 import inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    k = CENTER0
    rng = np.random.default_rng(7)
    host = {
        "L": torch.from_numpy(inputs.random_symmetric_env(CHI, W_MPO, seed=11)).pin_memory(),
        "R": torch.from_numpy(inputs.random_symmetric_env(CHI, W_MPO, seed=12)).pin_memory(),
        "A1": torch.from_numpy(rng.standard_normal((CHI, D, CHI // 2))).pin_memory(),
        "A2": torch.from_numpy(rng.standard_normal((CHI // 2, D, CHI))).pin_memory(),
        "W1": torch.from_numpy(np.ascontiguousarray(Wh[k])).pin_memory(),
        "W2": torch.from_numpy(np.ascontiguousarray(Wh[k + 1])).pin_memory(),
    }
    out_host = {"A1": torch.empty(CHI * D * CHI, dtype=torch.float64).pin_memory(),
                "A2": torch.empty(CHI * D * CHI, dtype=torch.float64).pin_memory(),
                "Lout": torch.empty(CHI * W_MPO * CHI, dtype=torch.float64).pin_memory()}
    d = {n: torch.empty_like(t, device=dev) for n, t in host.items()}
    theta = torch.empty((CHI, D, D, CHI), dtype=torch.float64, device=dev)
    A1o = torch.empty(CHI * D * CHI, dtype=torch.float64, device=dev)
    A2o = torch.empty(CHI * D * CHI, dtype=torch.float64, device=dev)
    Lout = torch.empty(CHI * W_MPO * CHI, dtype=torch.float64, device=dev)
    h2d = sum(t.numel() * 8 for t in host.values())
    d2h = sum(t.numel() * 8 for t in out_host.values()) + 8

    def one():
        for n in host:
            d[n].copy_(host[n], non_blocking=True)
        B.osmps_theta_form(ctx, d["A1"], d["A2"], theta)
        e, it, _, _ = B.osmps_lanczos_ground(ctx, d["L"], d["W1"], d["W2"], d["R"], theta,
                                             max_iter=LANCZOS_CAP, tol=LANCZOS_TOL, precision=prec)
        chn, _, _, _ = B.osmps_split(ctx, theta, A1o, A2o, 1, CHI, 1e-12 / (4 * L_SITES), precision=prec)
        A1v = A1o[: CHI * D * chn].view(CHI, D, chn)
        Lv = Lout[: chn * W_MPO * chn].view(chn, W_MPO, chn)
        B.osmps_env_update(ctx, 0, d["L"], A1v, d["W1"], Lv, precision=prec)
        out_host["A1"].copy_(A1o, non_blocking=True)
        out_host["A2"].copy_(A2o, non_blocking=True)
        out_host["Lout"].copy_(Lout, non_blocking=True)
        torch.cuda.synchronize()
        return it, e

    one()
    t0 = time.perf_counter()
    flops = 0.0
    n = max(1, min(args.steps, 3))
    for _ in range(n):
        it, _ = one()
        flops += it * heff_credited_flops(CHI, CHI)
    dt = time.perf_counter() - t0
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": n, "ms_per_step": 1e3 * dt / n}


def sweep_leg(B, ctx, mpo, prec):
    """One full left->right->left sweep at chi_max = 1024 from a fresh seeded MPS."""
    import torch
    from paper_1703_00387_gb300 import inputs
    mps = B.MPS(ctx, inputs.random_mps(L_SITES, D, CHI, seed=123), chi_cap=CHI)
    p = B.sweep_params(CHI, 1, prec, lanczos_tol=LANCZOS_TOL, lanczos_max_iter=LANCZOS_CAP)
    torch.cuda.synchronize()
    st = B.osmps_sweep(ctx, mps, mpo, p, record_steps=False)
    t0 = time.perf_counter()
    E, V = B.osmps_variance(ctx, mps, mpo)
    var_s = time.perf_counter() - t0
    # the float64-accurate refinement sweep that follows the split-precision one
    pr = B.sweep_params(CHI, 1, "fp64emu", lanczos_tol=LANCZOS_TOL, lanczos_max_iter=LANCZOS_CAP)
    torch.cuda.synchronize()
    sr = B.osmps_sweep(ctx, mps, mpo, pr, record_steps=False)
    mps.close()
    return {"seconds": st["sweep_seconds"] + sr["sweep_seconds"],
            "split_precision_sweep_seconds": st["sweep_seconds"],
            "refinement_sweep_seconds": sr["sweep_seconds"],
            "steps": st["steps"] + sr["steps"], "lanczos_iters": st["lanczos_iters"] + sr["lanczos_iters"],
            "variance_after_split_precision_sweep": V, "variance_seconds": var_s,
            "precision": prec + " sweep + fp64emu refinement sweep",
            "energy_after_split_precision_sweep": st["energy"], "energy_fp64": sr["energy"],
            "setup_seconds": st["setup_seconds"] + sr["setup_seconds"],
            "energy_seconds": st["energy_seconds"] + sr["energy_seconds"],
            "note": "one left-right-left sweep in the split precision, then one float64-accurate "
                    "(emulated) refinement sweep; QR canonicalisation + environment build (setup) "
                    "and the float64-accurate energies are timed separately"}


def accuracy_leg(B, ctx, args):
    """Time to a float64-accurate ground energy at bond dimension 1024: the
    open XXZ chain (J=1, Delta=1) at L=20 needs exactly 2^10 = 1024 at its
    middle bond, and its exact ground energy comes from the oracle's sparse
    diagonalisation (tests/golden/xxz_l20_ground_energy.json). From the same
    seeded random MPS at chi_max=1024:
      mixed: one bf16x3 sweep, then float64-accurate (emulated) refinement
             sweeps until |E - E_exact| <= 1e-10 |E_exact|;
      fp64:  plain float64 (DMMA) sweeps until the same bar.
    Each sweep is one osmps_sweep call (QR canonicalisation, environments,
    one L->R->L sweep, float64-accurate energy), all inside the wall time,
    after one untimed sweep in each precision (first-use costs)."""
    import torch
    from paper_1703_00387_gb300 import hamiltonians, inputs
    with open(os.path.join(ROOT, "tests", "golden", "xxz_l20_ground_energy.json")) as f:
        e0 = json.load(f)["ground_energy"]
    L, chi = 20, 1024
    mpo = B.MPO(ctx, hamiltonians.xxz(L, 1.0, 1.0, 0.0))
    bar = 1e-10 * abs(e0)

    def run(phases):
        mps = B.MPS(ctx, inputs.random_mps(L, 2, chi, seed=0), chi_cap=chi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        log, e_prev = [], None
        for prec, until, cap in phases:
            p = B.sweep_params(chi, 1, prec, lanczos_tol=1e-12, lanczos_max_iter=100)
            for _ in range(cap):
                e = B.osmps_sweep(ctx, mps, mpo, p, record_steps=False)["energy"]
                log.append((prec, e - e0))
                done = until(e, e_prev)
                e_prev = e
                if done:
                    break
        dt = time.perf_counter() - t0
        mps.close()
        err = abs(log[-1][1])
        return {"seconds": dt, "sweeps": [x[0] for x in log], "energy_error": log[-1][1],
                "relative_error": err / abs(e0), "reached": err <= bar}

    exact = lambda e, ep: abs(e - e0) <= bar
    once = lambda e, ep: True
    run([("bf16x3", once, 1), ("fp64emu", once, 1), ("fp64", once, 1)])  # untimed warm-up
    mixed = run([("bf16x3", once, 1), ("fp64emu", exact, 4)])
    plain = run([("fp64", exact, 6)])
    mpo.close()
    return {"workload": "open XXZ J=1 Delta=1, L=20, chi_max=1024 (exact at chi=1024), "
                        "seeded random start (seed 0)",
            "exact_energy": e0, "bar": "|E - E_exact| <= 1e-10 |E_exact|",
            "mixed_bf16x3_plus_refinement": mixed, "plain_fp64": plain,
            "speedup": plain["seconds"] / mixed["seconds"] if mixed["seconds"] > 0 else None}


def batch_leg(B, args):
    """64 independent TFI / XXZ chains (L in [16, 128], chi_max in {32, 64, 128,
    256}, g or Delta in [0.5, 1.5], seeded) swept at once by the native batch
    scheduler: one worker thread, context and stream each, longest chains
    first. One untimed sweep of every chain first (allocations, workspace
    growth), then one timed sweep of every chain; aggregate sweeps per second."""
    import torch
    from paper_1703_00387_gb300 import hamiltonians, inputs
    chains = inputs.chain_batch(64, seed=0)
    ctxs = [B.Context(torch.cuda.current_device()) for _ in range(args.batch_workers)]
    mps, mpo, par = [], [], []
    for i, c in enumerate(chains):
        W = (hamiltonians.ising(c["L"], 1.0, c["param"]) if c["model"] == "tfi"
             else hamiltonians.xxz(c["L"], 1.0, c["param"], 0.0))
        mpo.append(B.MPO(ctxs[0], W))
        mps.append(B.MPS(ctxs[0], inputs.random_mps(c["L"], D, c["chi_max"], seed=1000 + i),
                         chi_cap=c["chi_max"]))
        par.append(B.sweep_params(c["chi_max"], 1, args.precision, lanczos_tol=LANCZOS_TOL,
                                  lanczos_max_iter=LANCZOS_CAP))
    B.osmps_sweep_batch(ctxs, mps, mpo, par)  # untimed
    torch.cuda.synchronize()
    launches0 = B.osmps_kernel_launches()
    t0 = time.perf_counter()
    stats, _ = B.osmps_sweep_batch(ctxs, mps, mpo, par)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = B.osmps_kernel_launches() - launches0
    for x in mps + mpo + ctxs:
        x.close()
    steps = sum(s["steps"] for s in stats)
    return {"value": len(chains) / dt, "unit": "sweeps/s", "chains": len(chains),
            "sweeps_per_chain": 1, "seconds": dt, "workers": args.batch_workers,
            "precision": args.precision, "two_site_steps": steps,
            "lanczos_iters": sum(s["lanczos_iters"] for s in stats), "gpu_launches": launches,
            "workload": "64 chains from seed 0: TFI or XXZ (p = 1/2), L ~ U{16..128}, "
                        "chi_max ~ U{32, 64, 128, 256}, g or Delta ~ U[0.5, 1.5]; "
                        "random seeded MPS at chi_max"}


def u1_leg(B, ctx, args):
    """Config 3: U(1) block-sparse H_eff.theta of the Bose-Hubbard chain (L=64,
    N=64, n <= 4, d=5, w=4, chi=512 per bond, sector sizes from the Gaussian
    profile around N k / L at bonds 31 and 33), each GEMM stage one grouped
    tcgen05 launch over all sector blocks. Inputs resident; the operator is
    prepared once (timed apart), then CUDA events over `reps` products after
    3 warm-up products, as inside Lanczos."""
    import torch
    from paper_1703_00387_gb300 import hamiltonians, inputs
    from paper_1703_00387_gb300 import u1 as pu1
    dev = torch.device("cuda", torch.cuda.current_device())
    W = hamiltonians.bose_hubbard(64, 1.0, 4.0, 4)
    q = pu1.channel_charges(W)
    left = inputs.u1_sector_profile(31.0, total=512, width=8.0)
    right = inputs.u1_sector_profile(33.0, total=512, width=8.0)
    out = {}
    for prec in ("tf32x3", "bf16x3"):
        op = pu1.U1Operator(ctx, left, right, 5, 5, W[31], W[32], q[31], q[33])
        pl = op.plan
        t = [torch.from_numpy(inputs.random_dense((n,), seed)).to(dev)
             for n, seed in ((pl.n_L, 1), (pl.n_R, 2), (pl.n_theta, 3))]
        W1, W2 = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (W[31], W[32]))
        y = torch.empty_like(t[2])
        stream = torch.cuda.current_stream()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        B.osmps_u1_heff_prepare(ctx, pl, t[0], W1, W2, t[1], precision=prec)
        p1.record(stream)
        for _ in range(3):
            B.osmps_u1_heff_apply(ctx, pl, t[2], y)
        reps = 20
        B.osmps_profile_enable(ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            B.osmps_u1_heff_apply(ctx, pl, t[2], y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prep_ms = p0.elapsed_time(p1)
        prof = B.osmps_profile_read(ctx, "gemm_tc")
        wst = B.osmps_profile_read(ctx, "u1_wstep")  # "flops" = algorithmic bytes
        B.osmps_profile_enable(ctx, False)
        peaks, peak_src = load_peaks()
        w_gbs = wst["flops"] / (wst["ms"] / 1e3) / 1e9 if wst["ms"] > 0 else None
        dense = 2.0 * 25 * 512 * 512 * (4 * 512 + 4 * 512)
        out[prec] = {"ms_per_product": ms, "prepare_ms": prep_ms,
                     "block_gemm_tflops": pl.flops / (ms / 1e3) / 1e12,
                     "block_gemm_gflop": pl.flops / 1e9, "dense_equivalent_gflop": dense / 1e9,
                     "grouped_gemm_share": prof["ms"] / (ms * reps) if ms > 0 else None,
                     "grouped_gemm_launches": prof["launches"],
                     "grouped_gemm_issued_tflops": (prof["tensor_flops"] / (prof["ms"] / 1e3) / 1e12
                                                   if prof["ms"] > 0 else None),
                     "n_theta": pl.n_theta, "n_theta_dense": 512 * 25 * 512,
                     "wstep": {"kernel": "k_u1_wsteps_seg (fused sector W-step)", "bound": "hbm",
                               "bytes_per_launch": wst["flops"] / max(wst["launches"], 1),
                               "bytes_basis": "T1 read once (float32) + split stage-4 operand entries "
                                              "written once (2 pieces)",
                               "avg_launch_ms": wst["ms"] / max(wst["launches"], 1),
                               "achieved": w_gbs, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                               "frac": w_gbs / peaks["hbm_gbs"] if w_gbs else None,
                               "peak_source": f"{peak_src} hbm_gbs",
                               "share_of_product": wst["ms"] / (ms * reps) if ms > 0 else None,
                               "n_T1": pl.n_T1, "n_A4": pl.n_A4}}
        op.close()
    return {"workload": "Bose-Hubbard J=1 U=4, L=64, N=64, n<=4 (d=5), w=4, chi=512 per bond "
                        "(13 sectors each), two-site H_eff.theta at sites 31,32", **out}


def u1_sweep_leg(B, ctx, args):
    """Config 3 end to end: two-site sweeps of the Bose-Hubbard chain
    (J=1, U=4, L=64, N=64, n <= 4, d=5) on a particle-number-conserving MPS
    with block-sparse tensors: U(1) Lanczos on the grouped tcgen05 H_eff,
    per-charge Gram eigenpairs with the truncation rule applied jointly
    across sectors, block environment updates on the grouped float64 GEMM.
    A seeded random U(1) MPS (chi 64) is swept once at chi_max = 128 to warm
    up; then one timed left-right-left sweep at chi_max = 512 with
    eps_local = 0 (the bond dimension grows to the cap), and one with
    eps_local = 1e-12 (the converged state's own bond dimension). Seconds by
    the host clock around each sweep (the calls synchronise), energies in
    float64."""
    from paper_1703_00387_gb300 import hamiltonians
    from paper_1703_00387_gb300 import u1sweep as us
    L, nmax, N = 64, 4, 64
    W = hamiltonians.bose_hubbard(L, 1.0, 4.0, nmax)
    ex = us.DeviceExecutor(ctx)
    mps = us.random_u1_mps(ex, L, nmax + 1, N, chi=64, seed=0)
    us.u1_sweep(mps, W, n_sweeps=1, chi_max=128, eps_local=0.0, precision=args.precision,
                lanczos_tol=1e-10, lanczos_max_iter=LANCZOS_CAP)
    out = {"workload": "Bose-Hubbard J=1 U=4, L=64, N=64, n<=4 (d=5), w=4: one sweep at chi_max=512 "
                       "(eps_local=0, bond dimension saturating), then one at eps_local=1e-12; "
                       "seeded random U(1) MPS (chi 64), one warm-up sweep at chi_max=128",
           "precision": args.precision}
    for key, eps in (("saturating", 0.0), ("eps_1e-12", 1e-12)):
        l0 = B.osmps_kernel_launches()
        r = us.u1_sweep(mps, W, n_sweeps=1, chi_max=512, eps_local=eps, precision=args.precision,
                        lanczos_tol=1e-10, lanczos_max_iter=LANCZOS_CAP)
        out[key] = {"sweep_seconds": r["sweep_seconds"], "canonicalize_seconds": r["setup_seconds"],
                    "steps": r["steps"], "lanczos_iters": r["lanczos_iters"], "energy_fp64": r["energy"],
                    "max_chi": r["max_chi"], "max_discarded": r["max_discarded"],
                    "middle_bond_sectors": len(mps.bonds[L // 2].q),
                    "gpu_launches": B.osmps_kernel_launches() - l0}
    out["eig_workers"] = ex.eig_workers
    ex.close()
    return out


def long_range_leg(B, ctx, args):
    """Long-range transverse-field Ising chain (Eq. LRIsing), J=1, g=1,
    alpha=1.5 written as 8 exponentials (MPO w=10), L=128, chi_max=256: one
    left-right-left sweep from a seeded random MPS (split-precision
    contractions, float64 Lanczos and split)."""
    from paper_1703_00387_gb300 import hamiltonians, inputs
    L, chi = 128, 256
    a, lam, err = hamiltonians.exponential_fit(lambda r: r ** -1.5, L - 1, 8)
    mpo = B.MPO(ctx, hamiltonians.long_range_ising(L, 1.0, 1.0, a, lam))
    mps = B.MPS(ctx, inputs.random_mps(L, D, chi, seed=5), chi_cap=chi)
    st = B.osmps_sweep(ctx, mps, mpo, B.sweep_params(chi, 1, args.precision, lanczos_tol=LANCZOS_TOL,
                                                     lanczos_max_iter=LANCZOS_CAP), record_steps=False)
    mps.close()
    mpo.close()
    return {"workload": "long-range TFI J=1 g=1 alpha=1.5 (8 exponentials, w=10), L=128, chi_max=256",
            "fit_max_error": err, "sweep_seconds": st["sweep_seconds"], "steps": st["steps"],
            "lanczos_iters": st["lanczos_iters"], "energy_fp64": st["energy"],
            "precision": args.precision}


def excited_leg(B, ctx, args):
    """Excited-state search (eMPS) on the paper's example system, the
    long-range Ising chain: L=32, J=1, g=4 (paramagnetic, gapped; at g=1 the
    chain is ordered and the first excited state is the other member of the
    ground doublet), alpha=1.5 as 3 exponentials (w=5), chi_max=64. Ground
    state by 3 sweeps, first excited state by 4 projected sweeps; seconds of
    each and the overlap of the two."""
    import torch
    from paper_1703_00387_gb300 import hamiltonians, inputs
    from paper_1703_00387_gb300.excited import excited_state
    L, chi = 32, 64
    a, lam, _ = hamiltonians.exponential_fit(lambda r: r ** -1.5, L - 1, 3)
    W = hamiltonians.long_range_ising(L, 1.0, 4.0, a, lam)
    mpo = B.MPO(ctx, W)
    mps = B.MPS(ctx, inputs.random_mps(L, D, chi, seed=11), chi_cap=chi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = B.osmps_sweep(ctx, mps, mpo, B.sweep_params(chi, 3, "fp64", lanczos_tol=1e-12),
                       record_steps=False)
    t_ground = time.perf_counter() - t0
    ground = mps.tensors()
    mps.close()
    mpo.close()
    t0 = time.perf_counter()
    r = excited_state(ctx, W, [ground], inputs.random_mps(L, D, chi, seed=12), chi, n_sweeps=4)
    t_exc = time.perf_counter() - t0
    return {"workload": "long-range TFI J=1 g=4 alpha=1.5 (3 exponentials, w=5), L=32, chi_max=64",
            "ground_energy": st["energy"], "excited_energy": r["energy"],
            "overlap": r["overlaps"][0], "ground_seconds": t_ground, "excited_seconds": t_exc}


def tdvp_leg(B, ctx, args):
    """Two-site TDVP real-time evolution (Sec. 5.4) of the XXZ chain (J=1,
    Delta=1), L=64, at saturated bond dimension chi=128: a seeded random MPS
    right-canonicalised on the GPU (osmps_mps_canonicalize), then one untimed
    and two timed steps of dt=0.05 (Krylov tolerance 1e-10, at most 40
    vectors), split-precision contractions, float64 Krylov and split."""
    from paper_1703_00387_gb300 import hamiltonians, inputs
    L, chi, dt = 64, 128, 0.05
    W = hamiltonians.xxz(L, 1.0, 1.0, 0.0)
    mpo = B.MPO(ctx, W)
    mps = B.MPS(ctx, inputs.random_mps(L, D, chi, seed=21), chi_cap=chi)
    B.osmps_mps_canonicalize(ctx, mps, mpo, 0, precision="fp64")
    start = [t.astype(np.complex128) for t in mps.tensors()]
    mps.close()
    warm, _, _, _ = B.osmps_tdvp_evolve(ctx, mpo, start, dt, 1, chi_max=chi, krylov_tol=1e-10,
                                        krylov_max_iter=40, precision=args.precision)
    out, energy, norm, st = B.osmps_tdvp_evolve(ctx, mpo, warm, dt, 2, chi_max=chi,
                                                krylov_tol=1e-10, krylov_max_iter=40,
                                                precision=args.precision)
    mpo.close()
    steps = 2
    return {"workload": "XXZ J=1 Delta=1, L=64, d=2, w=5, chi=128 (saturated), dt=0.05, "
                        "two-site TDVP second-order steps from a random right-canonical MPS",
            "seconds_per_step": st["seconds"] / steps, "steps": steps,
            "krylov_vectors_per_step": st["krylov_vectors"] / steps,
            "krylov_calls_per_step": st["krylov_calls"] / steps, "max_krylov": st["max_krylov"],
            "nonconverged": st["nonconverged"], "max_chi": st["max_chi"],
            "max_discarded": st["max_discarded"],
            "energy_drift": float(abs(energy[-1] - energy[0])), "norm_last": float(norm[-1]),
            "precision": args.precision}


def grad_leg(B, ctx, args):
    """Config 5 (differentiation): XXZ L=64, chi=256, J_i in [0.8, 1.2], h_i in
    [-0.5, 0.5] from seed 0. Times of the H_eff.theta backward at chi=256
    (g_theta, g_W1, g_W2) and of the energy gradient dE/d(J, h) with
    checkpointed right environments; the gradient of one coupling against a
    central difference of the energy with step 1e-6."""
    import torch
    from paper_1703_00387_gb300 import hamiltonians, inputs
    from paper_1703_00387_gb300.autograd import xxz_energy
    dev = torch.device("cuda", torch.cuda.current_device())
    ops = inputs.random_heff_operands(256, 2, 2, 256, 5, 5, 5, seed=256)
    t = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in ops]
    gy = torch.from_numpy(np.random.default_rng(257).standard_normal(ops[4].shape)).to(dev)
    out = {}
    for prec in ("bf16x3", "fp64emu"):
        gt, g1, g2 = torch.empty_like(t[4]), torch.empty_like(t[1]), torch.empty_like(t[2])
        B.osmps_heff_backward(ctx, *t[:4], t[4], gy, gt, g1, g2, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            B.osmps_heff_backward(ctx, *t[:4], t[4], gy, gt, g1, g2, precision=prec)
        torch.cuda.synchronize()
        out[f"heff_backward_ms_{prec}"] = 1e3 * (time.perf_counter() - t0) / 5
    L = 64
    J, h = inputs.random_couplings(L, seed=0)
    mps = B.MPS(ctx, inputs.random_mps(L, 2, 256, seed=0), chi_cap=256)
    model = xxz_energy(ctx, mps, L, delta=1.0, checkpoint_every=8)
    p = torch.tensor(np.concatenate([J, h]), dtype=torch.float64, device=dev, requires_grad=True)
    model(p).backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = model.coupling_grad()
    torch.cuda.synchronize()
    out["energy_grad_seconds"] = time.perf_counter() - t0
    j = 10
    e = []
    for sgn in (1.0, -1.0):
        q = np.concatenate([J, h])
        q[j] += sgn * 1e-6
        e.append(model(torch.tensor(q, dtype=torch.float64, device=dev)).item())
    fd = (e[0] - e[1]) / 2e-6
    out["fd_check"] = {"coupling": "J_10", "gradient": float(g[j]), "central_difference": fd,
                       "abs_error": abs(fd - float(g[j]))}
    mps.close()
    out["workload"] = ("XXZ Delta=1, L=64, chi=256, J_i ~ U[0.8,1.2], h_i ~ U[-0.5,0.5] (seed 0); "
                       "H_eff backward at chi_l=chi_r=256, w=5")
    return out


def cpu_leg(B, ctx, Wh):
    import torch
    from oracle import dmrg as od
    from paper_1703_00387_gb300 import inputs
    dt, f, it = oracle_step_sample(seed=0)
    base = {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_threads(),
            "blas_threads": blas_threads(), "kind": "oracle",
            "sample": f"one FP64 NumPy two-site step at chi=1024 ({it} Lanczos matvecs), {dt:.1f} s"}
    # matvec error of the GPU path at this size against the oracle
    k = CENTER0
    Lh = inputs.random_symmetric_env(CHI, W_MPO, seed=21)
    Rh = inputs.random_symmetric_env(CHI, W_MPO, seed=22)
    th = np.random.default_rng(23).standard_normal((CHI, D, D, CHI))
    ref = od.heff_apply(Lh, Wh[k], Wh[k + 1], Rh, th)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (Lh, Wh[k], Wh[k + 1], Rh, th)]
    errs = {}
    for prec in ("bf16x3", "tf32x3", "fp64"):
        y = torch.empty_like(t[4])
        B.osmps_heff_apply(ctx, *t, y, precision=prec)
        torch.cuda.synchronize()
        errs[prec] = float(np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref))
    return base, errs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="timed steps only (for profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.quick:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
