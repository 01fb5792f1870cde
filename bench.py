#!/usr/bin/env python3
"""Benchmark: forward+adjoint path-steps/s of the projected-gradient Armijo iteration.

One step = one iteration of the optimizer (Algorithm 5.4) on the d=2 double-well
jump-diffusion workload (M = 2^20 paths, N_t = 1000 steps, FP32 paths, FP64
reductions): the gradient (forward sweep with stored trajectories, adjoint sweep,
cross-path reductions), the Armijo line search (forward cost sweeps and the FP64
test) and the projected update.  value = M * N_t gradient path-steps per step / time
per step, so line-search sweeps count as overhead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--variant stored|recompute]

Under torchrun (N > 1) every rank solves its own independent problem instance (the
same workload with Philox seed = rank): weak scaling, no collective on the data path;
only the timing is reduced (max over ranks).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "forward+adjoint path-steps/s vs roofline; ∇Ĵ error vs FP64; serve p50/p99 latency"
UNIT = "path-steps/s"
L2_BYTES = 129 * 1024 * 1024


def _sm_count() -> int:
    """SMs of the current device (the issue-rate peaks scale with it)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:   # no torch / no device: the GB300's count
        pass
    return 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms (start before the
    timed region, stop after)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_problem(p, rank: int):
    """Rank r solves an independent instance: same workload, Philox seed p.seed + r."""
    return p.replace(seed=p.seed + rank)


def max_over_ranks(dist, value: float, device="cpu") -> float:
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


WORKLOADS = {
    "double_well": workloads.double_well,   # d=2 cubic, M=2^20, Nt=1000 (the headline)
    "linear32": workloads.linear32,         # d=32 linear, M=2^18, Nt=500
    "lq_scalar": workloads.lq_scalar,       # d=1 linear-quadratic, M=1000, Nt=100 (FP64)
    # autograd form: J(u, theta) forward + backward, M=2^22, Nt=4096, checkpointed states
    "double_well_autograd": workloads.double_well_autograd,
    # Keilson-Storer velocity resets (beta=10, gamma=0.9), d=2 oscillator, M=2^20, Nt=500
    "ks_oscillator": workloads.ks_oscillator,
    # feedback control mu(t)^T phi(z), 10x10 bumps, Gaussian tracking, resets; M=2^20, Nt=100
    "feedback_centering": lambda: workloads.feedback_centering()[0],
    # the same with eta = 0, eps = 0.1 and the piecewise-linear target of Sec. 6.3
    "feedback_trajectory": lambda: workloads.feedback_trajectory()[0],
    # Sec. 6.4: rings of 32 coupled oscillators, ellipse cost; M=2^20 (2^15 rings), Nt=100
    "feedback_coupled": lambda: workloads.feedback_coupled()[0],
}
FB_WORKLOADS = {"feedback_centering": workloads.feedback_centering,
                "feedback_trajectory": workloads.feedback_trajectory,
                "feedback_coupled": workloads.feedback_coupled}


def bench_workload(M=None, Nt=None, name="double_well", keep_dt=False):
    """The named workload, with M and N_t overridden when given; keep_dt shortens the
    horizon with N_t so that the step length (and with it the jump rate per step, which
    sets the kernels' instruction mix) stays the full workload's."""
    p = WORKLOADS[name]()
    if M is not None:
        p = p.replace(M=M)
    if Nt is not None:
        p = p.replace(Nt=Nt, T=p.T * Nt / p.Nt) if keep_dt else p.replace(Nt=Nt)
    return p


# --------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------------------
def oracle_step_rate(p_sample, steps: int, warmup: int):
    """Time `steps` oracle optimizer iterations (gradient + Armijo search + update) on a
    bounded sample of the workload; returns (path-steps/s, seconds per step, threads)."""
    import oracle
    threads = oracle.default_threads()
    u = np.zeros((p_sample.Nt, p_sample.du))
    zeta = 1.0
    for _ in range(warmup):
        u, r, _ = oracle.optimize(p_sample, u, max_iter=1, tol_rel_grad=0.0, zeta0=zeta)
        zeta = min(2 * r["zeta"], 1e3)
    t0 = time.perf_counter()
    for _ in range(steps):
        u, r, _ = oracle.optimize(p_sample, u, max_iter=1, tol_rel_grad=0.0, zeta0=zeta)
        zeta = min(2 * r["zeta"], 1e3)
    dt = (time.perf_counter() - t0) / max(1, steps)
    return p_sample.M * p_sample.Nt / dt, dt, threads


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    full = bench_workload()
    sample_M = args.reference_paths
    ps = full.replace(M=sample_M)
    rate, sec, threads = oracle_step_rate(ps, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "double_well d=2 M=2^20 Nt=1000 (oracle on a path sample)",
                   "d": full.d, "M": full.M, "Nt": full.Nt, "sample_paths": sample_M},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{sample_M} of {full.M} paths, all {full.Nt} steps, one "
                                   "optimizer iteration per step"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------
# path sharding: one problem's paths over the ranks (--shard)
# --------------------------------------------------------------------------------------
UNIT_PATHS = 16384   # JD_UNIT_PATHS


def ring_lanes(N: int) -> int:
    """Lanes of a ring of N interacting particles (32 up to 32 particles, the next power of
    two up to 256, then the next multiple of 256): the path-index stride of its rings."""
    if N <= 32:
        return 32
    if N <= 256:
        return 1 << (N - 1).bit_length()
    return 256 * -(-N // 256)


def shard_range(M, rank, world, unit=UNIT_PATHS):
    """Paths [m0, m0 + n) of one rank: whole units of the path reduction in rank order,
    split as evenly as possible (a rank may get none)."""
    nun = -(-M // unit)
    per, extra = divmod(nun, world)
    u0 = rank * per + min(rank, extra)
    u1 = u0 + per + (1 if rank < extra else 0)
    m0 = min(u0 * unit, M)
    return m0, min(u1 * unit, M) - m0


def gather_units(dist, units, ne):
    """Every rank's unit sums, concatenated in rank (that is, path) order."""
    if dist is None:
        return units
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, units)
    return np.concatenate([np.asarray(q).reshape(-1, ne) for q in parts])


def run_shard(args, p, stream, dist, ws, rank, local):
    """One gradient of the whole problem per step, its paths split over the ranks: each
    rank runs the units of its shard (jd_gradient_units), the units are all-gathered
    (about 64 KB per rank), every rank combines them (jd_combine_units) into the whole
    problem's J and gradient, bit for bit the single-GPU jd_gradient.  Strong scaling."""
    import torch
    import paper_2505_04328_gb300 as jd
    m0, n = shard_range(p.M, rank, ws)
    prec = "fp64" if args.workload == "lq_scalar" else "fp32"
    shard = jd.JdProblem(p.replace(M=n, m_offset=m0), prec=prec, mode=args.variant or "stored",
                         stream=stream) if n else None
    Nt, du = p.Nt, p.du
    ne = 1 + Nt * du
    u = np.zeros((Nt, du))

    def step():
        units = shard.gradient_units(u) if shard else np.zeros((0, ne))
        return jd.combine_units(p, u, gather_units(dist, units, ne))

    for _ in range(args.warmup):
        step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        J, g = step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    if dist is not None:
        ms = max_over_ranks(dist, ms, device="cuda")
    ms_per_step = ms / args.steps
    value = p.M * Nt / (ms_per_step * 1e-3)
    if shard:
        shard.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": f"{p.name} d={p.d} M={p.M} Nt={Nt}, paths sharded over {ws} ranks",
                           "step": "one whole-problem gradient: shard units, all-gather, combine",
                           "l2": "inputs larger than L2 (stored states); no flush"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": Nt * du * 8,
                        "d2h_bytes_per_step": -(-p.M // UNIT_PATHS) * ne * 8 / ws},
                "J": J}
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2505_04328_gb300 as jd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    jd.build()
    stream = torch.cuda.current_stream()

    if args.shard:   # every rank works on the same sample
        return run_shard(args, bench_workload(args.paths, args.steps_t, args.workload, args.keep_dt), stream, dist, ws, rank,
                         local)
    p = replica_problem(bench_workload(args.paths, args.steps_t, args.workload, args.keep_dt), rank)
    if args.workload == "double_well_autograd":
        return run_autograd(args, p, stream, dist, ws, rank, local)
    if args.workload in FB_WORKLOADS:
        return run_feedback(args, p, stream, dist, ws, rank, local)
    M, Nt, du = p.M, p.Nt, p.du
    prec = "fp64" if args.workload == "lq_scalar" else "fp32"
    prob = jd.JdProblem(p, prec=prec, mode=args.variant or "stored", stream=stream,
                        use_tensor_cores=args.tc)
    n = Nt * du
    u = torch.zeros(n, dtype=torch.float64, device="cuda")

    # warm-up iterations, then K timed iterations of one jd_optimize call on the
    # device-resident control (the optimizer state zeta carries over)
    r = optimize_device(prob, u, args.warmup, 1.0)
    zeta = min(2 * r["zeta"], 1e3)
    u_start, zeta_start = u.detach().cpu().numpy().reshape(Nt, du).copy(), zeta   # e2e replays this window
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    jd.profile_enable(True)
    l0 = jd.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    r = optimize_device(prob, u, args.steps, zeta)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = jd.launch_count() - l0
    kstats = jd.profile_read()
    jd.profile_enable(False)
    clk = clocks.stop()
    evals = r["evals"]
    if dist is not None:
        ms = max_over_ranks(dist, ms, device="cuda")
    ms_per_step = ms / args.steps
    value = ws * M * Nt / (ms_per_step * 1e-3)

    # end to end through the public API with host buffers, over the same K iterations: the
    # control at the start of the timed window goes host -> device, the K iterations run
    # (each reads its cost and Armijo decision back to the host; the fixed sample makes
    # them the timed iterations bit for bit), and the new control comes back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u_host, r2, _ = prob.optimize(u_start, max_iter=args.steps, tol_rel_grad=0.0, zeta0=zeta_start)
    e2e_sec = (time.perf_counter() - t0) / args.steps
    trials = (r2["sweeps"] - 1) / args.steps   # trial phases (a pair is one); the first gradient's sweep
    e2e = {"value": ws * M * Nt / e2e_sec, "unit": UNIT,
           "h2d_bytes_per_step": n * 8 / args.steps,
           "d2h_bytes_per_step": n * 8 / args.steps + 64 * (1 + trials),
           "same_iterations": bool(r2["evals"] == evals and r2["J"] == r["J"])}

    # gradient error of the FP32 path against FP64 at the final control: the FP64 GPU path
    # on all paths (it equals the oracle within 1e-12 pathwise in the parity tests); the
    # oracle itself on a path sample is compared in the cpu_baseline leg below
    u_fin = u.cpu().numpy().reshape(Nt, du).copy()
    grad_err = None
    if prec == "fp32" and p.d <= 8:   # FP64 paths are built for d <= 8
        J32, g32, _ = prob.gradient(u_fin)
        with jd.JdProblem(p, prec="fp64", mode=args.variant or "stored", stream=stream,
                          use_tensor_cores=0) as p64:
            J64, g64, _ = p64.gradient(u_fin)
        grad_err = {"vs": "FP64 GPU path, all paths, at the final control",
                    "J_rel": abs(J32 - J64) / abs(J64),
                    "grad_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64))}

    peaks, peak_kind = _peaks()
    rl = {k: kernel_roofline(k, v, p, peaks, peak_kind, args.tc, prob.info()["mode"]) for k, v in kstats.items()
          if k in KERNEL_BOUND}
    dom = max(rl, key=lambda k: kstats[k][1]) if rl else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload} d={p.d} M={M} Nt={Nt}",
                       "tensor_cores": {0: "off", 1: "bf16", 2: "bf16x3", 3: "bf16x3 adjoint only"}[args.tc],
                       "variant": prob.info()["mode"], "paths_per_gpu": M, "Nt": Nt,
                       "evals_per_step": evals / args.steps,
                       "sweeps_per_step": r["sweeps"] / args.steps,
                       "step": "one projected-gradient Armijo iteration (gradient, line search, "
                               "update) inside one jd_optimize call",
                       "l2": ("inputs larger than L2: the %s buffers (%.2f GB) exceed the 129 MB "
                              "L2; no flush" % (prob.info()["mode"], prob.info()["device_bytes"] / 1e9))
                       if prob.info()["device_bytes"] > 129e6 else
                       ("inputs fit in L2 (%.3f GB of %s buffers) and no flush: the K iterations run "
                        "inside one jd_optimize call; the problem is latency-bound (per-step chains of "
                        "few paths), not memory-bound" % (prob.info()["device_bytes"] / 1e9,
                                                          prob.info()["mode"]))},
            "gpu_launches": launches,
            "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kstats.items()},
            "roofline": rl.get(dom),
            "roofline_all": rl,
            "e2e": e2e,
            "clocks": clk,
            "grad_error_vs_fp64": grad_err,
        }
        if not args.no_cpu_baseline:
            ps = p.replace(M=min(M, args.reference_paths))
            rate, sec, threads = oracle_step_rate(ps, 1, 0)
            line["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": f"{ps.M} of {M} paths, all {Nt} steps, one optimizer iteration"}
            # the same path sample in this path's precision against the oracle (FP64)
            import oracle
            with jd.JdProblem(ps, prec=prec, stream=stream, use_tensor_cores=args.tc) as q:
                Js, gs, _ = q.gradient(u_fin)
            Jo, go, _ = oracle.gradient(ps, u_fin)
            line["grad_error_vs_oracle"] = {
                "paths": ps.M, "J_rel": abs(Js - Jo) / abs(Jo),
                "grad_rel_l2": float(np.linalg.norm(gs - go) / np.linalg.norm(go))}
        if args.oracle_paths:
            # this path's gradient at the final control against the FP64 oracle on the first
            # oracle_paths paths (all of them for a full-size FP64 reference where no FP64
            # GPU form is built, d = 32)
            import oracle
            pf = p.replace(M=min(M, args.oracle_paths))
            with jd.JdProblem(pf, prec=prec, stream=stream, use_tensor_cores=args.tc) as q:
                Jf, gf, _ = q.gradient(u_fin)
            t0 = time.perf_counter()
            Jo, go, _ = oracle.gradient(pf, u_fin)
            line["grad_error_vs_oracle_paths"] = {
                "paths": pf.M, "J_rel": abs(Jf - Jo) / abs(Jo),
                "grad_rel_l2": float(np.linalg.norm(gf - go) / np.linalg.norm(go)),
                "oracle_seconds": time.perf_counter() - t0, "oracle_threads": oracle.default_threads()}
        print(json.dumps(line), flush=True)
    prob.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def fb_forward_ops(p, fb):
    """Lane operations per path-step of the feedback forward sweep: the open-loop step
    (draws, drift, Euler, cost) plus the feedback: per bump r, r^2, 1 - eps^2 r^2, rcp,
    scale, 2^y (6), the bilinear form (nx nv + nx FMA), the control cost (3) and the
    Gaussian tracking term (6)."""
    return forward_ops(p) + 6 * (fb.nx + fb.nv) + fb.nx * fb.nv + fb.nx + 3 + 6


def fb_adjoint_ops(p, fb):
    """Lane operations per path-step of the feedback adjoint: bumps with derivatives (10
    each), the bilinear forms for u and u_v (2 nx nv + 3 nx), the outer product
    delta w phi_x phi_v^T summed over paths (nx nv FMA per path), the costate update
    (2 d^2 + 4) and the tracking gradient (6)."""
    return 10 * (fb.nx + fb.nv) + 2 * fb.nx * fb.nv + 3 * fb.nx + fb.nx * fb.nv + 2 * p.d * p.d + 4 + 6


def run_feedback(args, p, stream, dist, ws, rank, local):
    """One step = one feedback gradient dJ/dmu (forward sweep storing X_k, adjoint sweep
    with the per-step outer-product reduction, FP64 reductions) on device-resident mu."""
    import torch
    import paper_2505_04328_gb300 as jd
    from paper_2505_04328_gb300.binding import JD_MEM_DEVICE, _check, lib, make_feedback
    import ctypes

    fb = FB_WORKLOADS[args.workload]()[1]
    if args.particles is not None and fb.particles:
        # rings of another size: the same number of lanes, rounded to whole rings
        S = ring_lanes(args.particles)
        fb = fb.replace(particles=args.particles)
        p = p.replace(M=max(S, p.M // S * S))
    if args.fb_adjoint == "surrogate":
        fb = fb.replace(adjoint=workloads.FB_SURROGATE, sur_rate=args.sur_rate)
    M, Nt, L = p.M, p.Nt, fb.L
    prob = jd.JdProblem(p, prec="fp32", stream=stream)
    mu = torch.tensor(workloads.random_mu(p, fb, seed=23, scale=0.5), dtype=torch.float64, device="cuda")
    g = torch.empty_like(mu)
    F = make_feedback(fb)
    J = ctypes.c_double()

    def step():
        _check(lib().jd_fb_gradient(prob.h, ctypes.byref(F), ctypes.c_void_p(mu.data_ptr()), JD_MEM_DEVICE,
                                    ctypes.byref(J), ctypes.c_void_p(g.data_ptr())), "jd_fb_gradient")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    jd.profile_enable(True)
    l0 = jd.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = jd.launch_count() - l0
    kstats = jd.profile_read()
    jd.profile_enable(False)
    clk = clocks.stop()
    if dist is not None:
        ms = max_over_ranks(dist, ms, device="cuda")
    ms_per_step = ms / args.steps
    value = ws * M * Nt / (ms_per_step * 1e-3)

    # end to end: mu from host memory, the gradient back to host memory, every step
    mu_h = mu.cpu().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Jh, gh = prob.fb_gradient(fb, mu_h)
    e2e_sec = (time.perf_counter() - t0) / args.steps
    e2e = {"value": ws * M * Nt / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": Nt * L * 8,
           "d2h_bytes_per_step": Nt * L * 8 + 8}
    # dJ/dmu of the FP32 path against the FP64 GPU path on all paths (the FP64 kernels
    # equal the oracle within 1e-12 in the parity tests)
    with jd.JdProblem(p, prec="fp64", stream=stream) as p64:
        J64, g64 = p64.fb_gradient(fb, mu_h)
    grad_err = {"vs": "FP64 GPU path, all paths", "J_rel": abs(Jh - J64) / abs(J64),
                "grad_rel_l2": float(np.linalg.norm(gh - g64) / np.linalg.norm(g64))}

    peaks, _ = _peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    nsm = _sm_count()
    peak = nsm * 4 * 32 * sm_mhz * 1e6 / 1e9
    rl = {}
    for name, ops in (("fb_fwd", fb_forward_ops(p, fb)), ("fb_adj", fb_adjoint_ops(p, fb)),
                      ("fb_sur", fb_forward_ops(p, fb) + fb_adjoint_ops(p, fb))):
        if name in kstats:
            launches_k, total_ms = kstats[name]
            achieved = ops * M * Nt / (total_ms / launches_k * 1e-3) / 1e9
            rl[name] = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Glane-op/s",
                        "frac": achieved / peak, "traffic": None,
                        "peak_source": f"derived: {nsm} SMs x 4 schedulers x 32 lanes x 1 instruction/clock x "
                                       f"{sm_mhz:.0f} MHz (max SM clock)",
                        "algorithmic_ops_per_path_step": ops}
            iss = issue_fraction(args.workload, name, M * Nt, total_ms / launches_k * 1e-3, peaks)
            if iss and fb.adjoint == workloads.FB_EXACT:
                rl[name]["issue"] = iss
    dom = max(rl, key=lambda k: kstats[k][1]) if rl else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload} d=2 M={M} Nt={Nt} L={fb.nx}x{fb.nv}",
                       "variant": "stored" if fb.adjoint == workloads.FB_EXACT else
                                  f"surrogate adjoint (Sec. 6.5), rate {fb.sur_rate}",
                       "paths_per_gpu": M, "Nt": Nt, "eps": fb.eps,
                       "particles_per_ring": fb.particles or None,
                       "step": "one feedback gradient dJ/dmu (forward sweep, adjoint sweep, reductions)",
                       "l2": "inputs larger than L2: the stored states (%.2f GB) and warp partials exceed "
                             "the 129 MB L2; no flush" % ((Nt + 1) * 2 * M * 4 / 1e9)},
            "gpu_launches": launches,
            "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kstats.items()},
            "roofline": rl.get(dom),
            "roofline_all": rl,
            "e2e": e2e,
            "clocks": clk,
            "J": J.value,
            "grad_error_vs_fp64": grad_err,
        }
        if not args.no_cpu_baseline:
            import oracle
            ps = p.replace(M=min(M, args.reference_paths // 4))
            t0 = time.perf_counter()
            Jo, go = oracle.fb_gradient(ps, fb, mu_h)
            sec = time.perf_counter() - t0
            with jd.JdProblem(ps, prec="fp32", stream=stream) as q:
                Js, gs = q.fb_gradient(fb, mu_h)
            line["grad_error_vs_oracle"] = {
                "paths": ps.M, "J_rel": abs(Js - Jo) / abs(Jo),
                "grad_rel_l2": float(np.linalg.norm(np.asarray(gs) - np.asarray(go)) / np.linalg.norm(go))}
            line["cpu_baseline"] = {
                "value": ps.M * Nt / sec, "unit": UNIT,
                "cores": 1 if fb.particles else oracle.default_threads(),   # the ring sweep is one thread
                "kind": "oracle", "sample": f"{ps.M} of {M} paths, all {Nt} steps, one feedback gradient"}
        print(json.dumps(line), flush=True)
    prob.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_autograd(args, p, stream, dist, ws, rank, local):
    """One step = J(u, theta) and its backward through the torch.autograd.Function
    (jd_forward with checkpoints, then the recompute adjoint with parameter gradients)."""
    import torch
    import paper_2505_04328_gb300 as jd
    from paper_2505_04328_gb300.autograd import JumpDiffusionCost
    mode = args.variant or "recompute"
    f = JumpDiffusionCost(p, rho0=0.5, mode=mode, stream=stream)
    M, Nt, du = p.M, p.Nt, p.du
    u = torch.tensor(workloads.random_control(p, seed=41, scale=0.5), dtype=torch.float64,
                     device="cuda", requires_grad=True)
    th = torch.tensor((0.5, 0.3, 0.2), dtype=torch.float64, requires_grad=True)

    def step():
        u.grad = None
        th.grad = None
        J = f(u, th)
        J.backward()
        return J

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    jd.profile_enable(True)
    l0 = jd.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        J = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = jd.launch_count() - l0
    kstats = jd.profile_read()
    jd.profile_enable(False)
    clk = clocks.stop()
    if dist is not None:
        ms = max_over_ranks(dist, ms, device="cuda")
    ms_per_step = ms / args.steps
    value = ws * M * Nt / (ms_per_step * 1e-3)

    # end to end: the control comes from pinned host memory each step; J, dJ/du and
    # dJ/dtheta go back to the host
    u_pin = torch.empty((Nt, du), dtype=torch.float64).pin_memory()
    u_pin.copy_(u.detach().cpu())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ud = u_pin.to("cuda", non_blocking=True).requires_grad_(True)
        th.grad = None
        J = f(ud, th)
        J.backward()
        _ = (float(J), ud.grad.cpu(), th.grad.clone())
    e2e_sec = (time.perf_counter() - t0) / args.steps
    e2e = {"value": ws * M * Nt / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": Nt * du * 8,
           "d2h_bytes_per_step": 8 + Nt * du * 8 + 3 * 8}

    # dJ/du and the parameter gradients of the FP32 path against the FP64 GPU path on all
    # paths (the problem's own coefficients, through the C ABI)
    u_np = u.detach().cpu().numpy()
    with jd.JdProblem(p, prec="fp32", mode=mode, stream=stream) as q32, \
            jd.JdProblem(p, prec="fp64", mode=mode, stream=stream) as q64:
        J32, g32, t32 = q32.gradient(u_np, theta=True)
        J64, g64, t64 = q64.gradient(u_np, theta=True)
    grad_err = {"vs": "FP64 GPU path, all paths, the problem's coefficients",
                "J_rel": abs(J32 - J64) / abs(J64),
                "grad_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
                "theta_rel": [float(abs(a - b) / abs(b)) for a, b in zip(t32, t64)]}

    peaks, peak_kind = _peaks()
    rl = {k: kernel_roofline(k, v, p, peaks, peak_kind) for k, v in kstats.items() if k in KERNEL_BOUND}
    dom = max(rl, key=lambda k: kstats[k][1]) if rl else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "grad_error_vs_fp64": grad_err,
            "config": {"workload": f"double_well_autograd d=2 M={M} Nt={Nt}", "variant": mode,
                       "theta": "(damping 0.5, sigma 0.3, jump half-width 0.2)",
                       "step": "J(u, theta) forward + backward (dJ/du, dJ/dtheta) through the "
                               "torch.autograd.Function",
                       "l2": "inputs larger than L2: the %s buffers (%.2f GB) exceed the 129 MB "
                             "L2; no flush" % (mode, f.problem.info()["device_bytes"] / 1e9)},
            "gpu_launches": launches,
            "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kstats.items()},
            "roofline": rl.get(dom), "roofline_all": rl, "e2e": e2e, "clocks": clk,
            "J": float(J),
        }
        if not args.no_cpu_baseline:
            import oracle
            ps = p.replace(M=min(M, 2048))
            t0 = time.perf_counter()
            Jo, go, to = oracle.gradient(ps, u_np, theta=True)
            sec = time.perf_counter() - t0
            with jd.JdProblem(ps, prec="fp32", mode=mode, stream=stream) as q:
                Js, gs, ts = q.gradient(u_np, theta=True)
            line["grad_error_vs_oracle"] = {
                "paths": ps.M, "J_rel": abs(Js - Jo) / abs(Jo),
                "grad_rel_l2": float(np.linalg.norm(gs - go) / np.linalg.norm(go)),
                "theta_rel": [float(abs(a - b) / abs(b)) for a, b in zip(ts, to)]}
            line["cpu_baseline"] = {"value": ps.M * ps.Nt / sec, "unit": UNIT,
                                    "cores": oracle.default_threads(), "kind": "oracle",
                                    "sample": f"{ps.M} of {M} paths, all {Nt} steps, one gradient "
                                              "with parameter gradients"}
        print(json.dumps(line), flush=True)
    f.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def serve(jd, reqs, opt, slots, batch_paths=None):
    """Submit (arrival_time, problem) pairs at their arrival times to one jd_server and
    wait for all; returns (infos, results, wall seconds, kernels launched, (batched
    launch sequences, request phases in them))."""
    import threading as th
    srv = jd.JdServer(max_slots=slots, batch_paths=batch_paths)
    tickets = [None] * len(reqs)

    def submitter():
        t0 = time.perf_counter()
        for i, (ta, p) in enumerate(reqs):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(p, **opt)

    l0 = jd.launch_count()
    t_start = time.perf_counter()
    sub = th.Thread(target=submitter)
    sub.start()
    sub.join()
    for t in tickets:
        srv.wait(t)
    wall = time.perf_counter() - t_start
    launches = jd.launch_count() - l0
    infos = [srv.info(t) for t in tickets]
    results = [srv.poll(t)[1] for t in tickets]
    bstats = srv.batch_stats()
    srv.close()
    return infos, results, wall, launches, bstats


def small_stream(n, rate, seed=5):
    """The small requests of the serving stream (d <= 2, M <= 2^16: the ones that share
    batched launches), n of them, re-timed as Poisson arrivals at rate."""
    reqs, k = [], 0
    while len(reqs) < n:
        k += 5 * n
        reqs = [(t, p) for t, p in workloads.serving_requests(n=k, rate=rate, seed=seed)
                if p.d <= 2 and p.M <= (1 << 16)][:n]
    t = np.cumsum(np.random.default_rng(seed + 1000).exponential(1.0 / rate, size=n))
    return [(float(ti), p) for ti, (_, p) in zip(t, reqs)]


def plain_rate(jd, torch, reqs, prec, iters=3):
    """Path-steps per second of requests solved one at a time (jd_optimize, iters
    iterations each, no tolerance stop), gradient path-steps as in the served value."""
    steps, t = 0, 0.0
    for _, p in reqs:
        with jd.JdProblem(p, prec=prec) as jp:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, r, _ = jp.optimize(np.zeros((p.Nt, p.du)), max_iter=iters, tol_rel_grad=0.0)
            t += time.perf_counter() - t0
            steps += (r["iters"] + (0 if r["iters"] == iters else 1)) * p.M * p.Nt
    return steps / t if t > 0 else None


def run_serving_small(args, jd, clocks, ws, rank):
    """The small requests of the stream, served with batched launches and with one launch
    sequence per request (batching off): throughput, latency, kernels, mean batch."""
    reqs = small_stream(args.requests, args.rate, seed=5 + rank)
    opt = dict(max_iter=args.max_iter, tol_rel_grad=1e-4)
    out = {}
    for name, bp in (("batched", None), ("unbatched", 0)):
        infos, results, wall, launches, (bl, bph) = serve(jd, reqs, opt, args.slots, batch_paths=bp)
        st = serve_stats(infos, results)
        st.update(kernels=launches, batched_launches=bl, batched_phases=bph,
                  mean_batch=(bph / bl) if bl else None)
        out[name] = st
    clk = clocks.stop()
    value = out["batched"]["path_steps_per_s"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": len(reqs), "warmup": 0,
            "ms_per_step": out["batched"]["makespan_s"] * 1e3 / len(reqs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: the small requests of the stream (d <= 2, M <= 2^16), "
                                   f"{len(reqs)} requests, Poisson arrivals {args.rate}/s",
                       "slots": args.slots, "max_iter": args.max_iter, "tol_rel_grad": 1e-4,
                       "step": "one request; value = gradient path-steps / makespan (batched)"},
            "batched": out["batched"], "unbatched": out["unbatched"],
            "batched_vs_unbatched": value / out["unbatched"]["path_steps_per_s"],
            "latency_s": out["batched"]["latency_s"], "gpu_launches": out["batched"]["kernels"],
            "roofline": None, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serving_sample(jd, torch, reqs, slots):
    """The same requests three ways, 3 optimizer iterations each: served together (FP32),
    and one at a time through jd_optimize in FP32 (what serving itself adds) and in FP64
    (the plain per-problem GPU form)."""
    si, sr, _, _, _ = serve(jd, [(0.0, p) for _, p in reqs], dict(max_iter=3, tol_rel_grad=0.0), slots)
    served = serve_stats(si, sr)["path_steps_per_s"]
    plain64 = plain_rate(jd, torch, reqs, "fp64")
    plain32 = plain_rate(jd, torch, reqs, "fp32")
    return {"requests": len(reqs), "iterations": 3, "served_fp32": served, "one_at_a_time_fp32": plain32,
            "one_at_a_time_fp64": plain64, "unit": UNIT,
            "served_vs_one_at_a_time_fp32": (served / plain32) if plain32 else None,
            "served_vs_one_at_a_time_fp64": (served / plain64) if plain64 else None}


def run_serving_sample(args, jd, torch, clocks, ws, rank):
    """Only the served / one-at-a-time comparison on the first --plain-sample d <= 8
    requests of the stream."""
    reqs = workloads.serving_requests(n=args.requests, rate=args.rate, seed=5 + rank)
    sample = [(t, p) for t, p in reqs if p.d <= 8][: args.plain_sample]
    res = serving_sample(jd, torch, sample, args.slots)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": res["served_fp32"], "unit": UNIT, "n_gpus": ws, "steps": len(sample),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: the first {len(sample)} d <= 8 requests of the stream, served "
                                   "together vs one at a time", "slots": args.slots},
            "sample": res, "roofline": None, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serving_sweep(args, jd, clocks, ws, rank):
    """Rate sweep over the whole stream: --requests requests at each rate of --rates;
    per rate the completion rate (requests / makespan), latency p50/p99 and whether the
    server kept up (completion rate at least 0.9 of the arrival rate)."""
    opt = dict(max_iter=args.max_iter, tol_rel_grad=1e-4)
    rows = []
    for rate in [float(r) for r in args.rates.split(",")]:
        reqs = workloads.serving_requests(n=args.requests, rate=rate, seed=5 + rank)
        infos, results, wall, launches, (bl, bph) = serve(jd, reqs, opt, args.slots)
        st = serve_stats(infos, results)
        span = reqs[-1][0] - reqs[0][0]
        done_rate = len(reqs) / st["makespan_s"]
        rows.append({"rate": rate, "arrival_span_s": span, "completed_per_s": done_rate,
                     "kept_up": done_rate >= 0.9 * rate, "latency_s": st["latency_s"],
                     "path_steps_per_s": st["path_steps_per_s"], "kernels": launches,
                     "batched_phases": bph, "requests_ok": st["requests_ok"]})
    clk = clocks.stop()
    ok = [r["rate"] for r in rows if r["kept_up"]]
    best = max(rows, key=lambda r: r["path_steps_per_s"])
    line = {"metric": METRIC, "value": best["path_steps_per_s"], "unit": UNIT, "n_gpus": ws,
            "steps": args.requests * len(rows), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving rate sweep, {args.requests} requests of the stream per rate",
                       "slots": args.slots, "max_iter": args.max_iter, "tol_rel_grad": 1e-4},
            "sweep": rows, "highest_rate_kept_up": max(ok) if ok else None,
            "gpu_launches": sum(r["kernels"] for r in rows), "roofline": None, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serve_stats(infos, results):
    lat = np.array([i["done_s"] - i["submit_s"] for i in infos])
    makespan = max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos)
    steps = sum(i["path_steps"] for i in infos)
    return dict(makespan_s=makespan, path_steps_per_s=steps / makespan,
                sweep_path_steps_per_s=sum(i["sweep_steps"] for i in infos) / makespan,
                latency_s={"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
                requests=len(infos), requests_ok=sum(1 for r in results if r["status"] == 0),
                requests_converged=sum(1 for r in results if r["status"] == 0 and r["rel_grad_norm"] <= 1e-4),
                mean_iters=float(np.mean([r["iters"] for r in results])))


def run_serving(args):
    """Serving workload: requests of the serving stream (d in {1,2,8,32}, M log-uniform in
    [2^12, 2^22], N_t in [50, 2000], lambda in [0.5, 10], Poisson arrivals) submitted at
    their arrival times to one jd_server; each runs projected-gradient steps to a
    relative projected-gradient norm of 1e-4 (at most --max-iter updates).  value =
    gradient path-steps of all requests / makespan; latency = done - submit.  The
    comparison with the plain per-problem FP64 GPU form uses the d <= 8 requests only
    (d = 32 runs in FP32 only): the same requests served in FP32 vs a sample of them
    solved one at a time in FP64."""
    import torch
    import paper_2505_04328_gb300 as jd
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    jd.build()
    clocks = ClockSampler(local)
    clocks.start()
    if args.small:
        return run_serving_small(args, jd, clocks, ws, rank)
    if args.rates:
        return run_serving_sweep(args, jd, clocks, ws, rank)
    if args.sample_only:
        return run_serving_sample(args, jd, torch, clocks, ws, rank)
    reqs = workloads.serving_requests(n=args.requests, rate=args.rate, seed=5 + rank)
    opt = dict(max_iter=args.max_iter, tol_rel_grad=1e-4)
    infos, results, wall, launches, (bl, bph) = serve(jd, reqs, opt, args.slots)
    clk = clocks.stop()
    mix = serve_stats(infos, results)
    if args.mix_only:   # e.g. a rate below capacity: latency of the mix alone
        line = {"metric": METRIC, "value": mix["path_steps_per_s"], "unit": UNIT, "n_gpus": ws,
                "steps": len(reqs), "warmup": 0, "ms_per_step": mix["makespan_s"] * 1e3 / len(reqs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"serving {len(reqs)} requests, Poisson arrivals {args.rate}/s",
                           "slots": args.slots, "max_iter": args.max_iter, "tol_rel_grad": 1e-4},
                "mix": mix, "latency_s": mix["latency_s"], "gpu_launches": launches, "roofline": None,
                "batched": {"launches": bl, "phases": bph}, "clocks": clk}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0

    small = [(t, p) for t, p in reqs if p.d <= 8]
    i8, r8, _, _, _ = serve(jd, small, opt, args.slots)
    sub = serve_stats(i8, r8)
    # the same sample of these requests three ways, 3 optimizer iterations each: served
    # (all submitted at once), and one at a time through jd_optimize in FP32 (what
    # serving itself adds) and in FP64 (the plain per-problem GPU form)
    sample = serving_sample(jd, torch, small[: args.plain_sample], args.slots)
    value = mix["path_steps_per_s"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": len(reqs),
        "warmup": 0, "ms_per_step": mix["makespan_s"] * 1e3 / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving {len(reqs)} requests, Poisson arrivals {args.rate}/s, "
                               "d in {1,2,8,32}, M log-uniform [2^12,2^22], Nt U[50,2000], lambda U[0.5,10]",
                   "slots": args.slots, "max_iter": args.max_iter, "tol_rel_grad": 1e-4,
                   "step": "one request (ms_per_step = makespan / requests); value = gradient "
                           "path-steps / makespan",
                   "l2": "inputs larger than L2 for most requests; no flush"},
        "mix": mix,
        "d_le_8": {**sub, "sample": sample},
        "batched": {"launches": bl, "phases": bph},
        "latency_s": mix["latency_s"],
        "gpu_launches": launches, "roofline": None, "clocks": clk,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "requests enter and leave through host memory (jd_server_submit/poll)"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0

def optimize_device(prob, u_t, iters, zeta0):
    """iters optimizer iterations (jd_optimize) on a device-resident control tensor."""
    import ctypes
    from paper_2505_04328_gb300 import binding as b
    o = b.OptParams(max_iter=iters, tol_rel_grad=0.0, tol_step=0.0, armijo_c=1e-4, zeta0=zeta0,
                    zeta_max=1e3, max_backtracks=40)
    r = b.OptResult()
    st = b.lib().jd_optimize(prob.h, ctypes.c_void_p(u_t.data_ptr()), b.JD_MEM_DEVICE,
                             ctypes.byref(o), ctypes.byref(r), None)
    b._check(st, "jd_optimize")
    return dict(iters=r.iters, evals=r.evals, J=r.J, zeta=r.zeta, sweeps=r.sweeps)


# Algorithmic work per path-step.  Forward sweeps
# are bound by issue slots (lane-operations): Philox blocks x 40 (20 wide multiplies,
# 20 XORs), 3 per uniform, 7 per Box-Muller pair, the drift's multiply-adds (the A x
# contraction leaves the CUDA cores when it runs on tensor cores), 2 d for the Euler
# update, 3 d + 4 for the running cost, and lambda dt times the cost of a jump.  The
# stored adjoint is bound by HBM: state (4 d bytes), jump-flag bit, jump log.
KERNEL_BOUND = {"fwd_cost": "alu", "fwd_store": "alu", "fwd_ckpt": "alu", "fwd_pair": "alu",
                "adj_stored": "hbm", "adj_recompute": "alu"}


def forward_ops(p, tc=0, controls=1):
    """controls = 2: the paired sweep of two Armijo trials, which draws once and runs the
    drift, Euler update, cost and jump sub-steps once per control."""
    d, du = p.d, p.du
    P = (d + 1) // 2
    blocks = (1 + 2 * P + 3) // 4
    drift = (0 if tc else d * d) + d * du + (d * d + 2 * d if p.drift == workloads.CUBIC else 0)
    draws = 40 * blocks + 3 * 2 * P + 7 * P + 1
    base = draws + controls * (drift + 2 * d + 3 * d + 4)
    slot_blocks = (1 + 4 * P + 3) // 4
    per_jump = 40 * slot_blocks + 3 * 4 * P + 7 * 2 * P + controls * 2 * (d * d + d * du + 2 * d)
    return base + p.lam * p.dt * per_jump


def adjoint_ops(p):
    d, du = p.d, p.du
    return d * d + d * du + 2 * d + (d * d + 2 * d if p.drift == workloads.CUBIC else 0) + 10


# Counters of ncu captures (profiles/*.md), per path-step for DRAM bytes and per
# warp-step (32 path-steps) for issued warp-instructions.  Each entry records the
# fingerprint of the kernel sources it was counted on; when the sources have changed
# since, the entry is stale and the figures derived from it are reported as null.
COUNTERS = {
    # (workload, kernel): (fingerprint of the kernel sources, DRAM bytes per path-step or
    # None, warp-instructions per warp-step).  The headline's stored-plan kernels: one
    # launch each over the headline's N_t = 1000 steps on M = 2^18 paths (2048 blocks; the
    # counts per warp-step and the bytes per path-step do not depend on M), from
    # smsp__inst_executed.sum and dram__bytes_{read,write}.sum; the recompute adjoint: a
    # full capture at M = 2^20 over N_t = 100 steps of the workload's step length.  Both
    # in profiles/*_double_well_d2_*.md
    ("double_well", "fwd_pair"): ("999d9a9c5bfe", 18.06, 316.4),
    ("double_well", "fwd_store"): ("999d9a9c5bfe", 8.64, 293.9),
    ("double_well", "adj_stored"): ("999d9a9c5bfe", 8.79, 60.2),
    ("double_well", "adj_recompute"): ("999d9a9c5bfe", 0.79, 338.5),
    # the d = 32 kernels in BF16 tensor-core mode, M = 2^16 (512 tiles), N_t = 100 at the
    # workload's step length: profiles/fwd32_adj32_linear32_d32_M2p16_Nt100_dt2e-3_bf16.md
    ("linear32/tc1", "fwd_store"): ("999d9a9c5bfe", 127.7, 2145.7),
    ("linear32/tc1", "adj_stored"): ("999d9a9c5bfe", 143.0, 662.2),
}


def _kernel_fingerprint() -> str:
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2505_04328_gb300", "csrc")
    for f in ("jd_kernels.cuh", "jd_device.cuh", "jd_feedback.cuh", "jd_internal.h", "jd_tc32.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _counter(workload, name, which):
    e = COUNTERS.get((workload, name))
    if e is None or e[0] != _kernel_fingerprint():
        return None
    return e[1] if which == "traffic" else e[2]


def issue_fraction(workload, name, units, per_launch_s, peaks):
    n = _counter(workload, name, "inst")
    if n is None:
        return None
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = _sm_count() * 4 * sm_mhz * 1e6
    achieved = n * units / 32 / per_launch_s
    return {"inst_per_warp_step": n, "achieved_warp_inst_per_s": achieved, "peak_warp_inst_per_s": peak,
            "frac": achieved / peak,
            "source": "ncu smsp__inst_executed.sum of the same kernel sources (profiles/), per warp-step"}


def kernel_roofline(name, stat, p, peaks, peak_kind, tc=0, plan="stored"):
    """plan: the adjoint plan, which decides the mode of the paired-trial sweep (states
    stored or checkpoints); the captured counters belong to the stored plan's kernels."""
    launches, total_ms = stat
    per_launch_s = total_ms / launches * 1e-3
    units = p.M * p.Nt
    # counters exist for the headline's kernels and for the d = 32 kernels in BF16 mode
    wl = p.name if p.name != "linear32" else f"linear32/tc{tc}"
    captured = ((p.d == 2 and p.name == "double_well" and (name != "fwd_pair" or plan == "stored"))
                or (p.name == "linear32" and tc == 1))
    tr = _counter(wl, name, "traffic") if captured else None
    traffic = None if tr is None else tr * units
    if KERNEL_BOUND[name] == "hbm":
        bytes_per = 4 * p.d + 0.125 + p.lam * p.dt * (2 + p.d) * 4
        achieved = bytes_per * units / per_launch_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": achieved / peak, "traffic": traffic,
               "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
               else "fallback 6.8 TB/s",
               "algorithmic_bytes_per_path_step": bytes_per}
        iss = issue_fraction(wl, name, units, per_launch_s, peaks) if captured else None
        if iss:
            out["issue"] = iss
        return out
    tc = 0 if tc == 3 else tc   # mode 3: the forward runs on the CUDA cores
    ops = forward_ops(p, tc, 2 if name == "fwd_pair" else 1) + (adjoint_ops(p) if name == "adj_recompute" else 0.0)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    nsm = _sm_count()
    peak = nsm * 4 * 32 * sm_mhz * 1e6 / 1e9   # G lane-operations per second
    achieved = ops * units / per_launch_s / 1e9
    out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Glane-op/s",
           "frac": achieved / peak, "traffic": traffic,
           "frac_kind": "algorithmic only: the method's lane-operations per path-step (a Box-Muller pair "
                        "counted as 7, though the library log and sincospi take about 76 instructions) "
                        "against the issue peak; the instructions actually issued are in 'issue'",
           "peak_source": f"derived: {nsm} SMs x 4 schedulers x 32 lanes x 1 instruction/clock x "
                          f"{sm_mhz:.0f} MHz (max SM clock)",
           "algorithmic_ops_per_path_step": ops}
    if tc:
        flops = 2.0 * p.d * p.d * (3 if tc == 2 else 1) * units
        out["tensor_tflops"] = flops / per_launch_s / 1e12
    iss = issue_fraction(wl, name, units, per_launch_s, peaks) if captured else None
    if iss:
        out["issue"] = iss
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default=None, choices=["stored", "recompute", "auto"],
                    help="adjoint plan (default: stored; recompute for double_well_autograd)")
    ap.add_argument("--workload", default="double_well", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--requests", type=int, default=64, help="serving: requests from the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (1/s)")
    ap.add_argument("--slots", type=int, default=16, help="serving: requests in flight at most")
    ap.add_argument("--max-iter", type=int, default=50, help="serving: optimizer updates at most")
    ap.add_argument("--plain-sample", type=int, default=32,
                    help="serving: requests of the d <= 8 subset served together and timed one at a time")
    ap.add_argument("--mix-only", action="store_true",
                    help="serving: the whole stream only (no d <= 8 pass, no plain FP64 sample)")
    ap.add_argument("--small", action="store_true",
                    help="serving: the stream's small requests (d <= 2, M <= 2^16), batched vs unbatched")
    ap.add_argument("--sample-only", action="store_true",
                    help="serving: only the served vs one-at-a-time comparison on --plain-sample requests")
    ap.add_argument("--rates", default=None,
                    help="serving: comma-separated arrival rates (1/s) for a rate sweep of the stream")
    ap.add_argument("--tc", type=int, default=0, choices=[0, 1, 2, 3],
                    help="tensor cores for the d=32 workload: 0 off, 1 BF16, 2 BF16x3, "
                         "3 BF16x3 in the adjoint only")
    ap.add_argument("--paths", type=int, default=None, help="override M (paths per GPU)")
    ap.add_argument("--steps-t", type=int, default=None, help="override N_t")
    ap.add_argument("--keep-dt", action="store_true",
                    help="with --steps-t: shorten the horizon so that the step length stays the workload's")
    ap.add_argument("--reference-paths", type=int, default=1 << 14)
    ap.add_argument("--oracle-paths", type=int, default=0,
                    help="also compare the gradient at the final control with the FP64 oracle on "
                         "this many paths (0 = no)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--particles", type=int, default=None,
                    help="feedback_coupled: particles per ring (3..2048; the paper's Sec. 6 uses 2000)")
    ap.add_argument("--shard", action="store_true",
                    help="one problem's paths split over the ranks (one gradient per step, strong scaling)")
    ap.add_argument("--fb-adjoint", default="exact", choices=["exact", "surrogate"],
                    help="feedback workloads: exact adjoint or the surrogate-state adjoint of Sec. 6.5")
    ap.add_argument("--sur-rate", type=float, default=0.05, help="surrogate variance growth per unit time")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
