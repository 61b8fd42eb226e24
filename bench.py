#!/usr/bin/env python3
"""Benchmark: one SVGD iteration of multiple-shooting inference per step.

Workload: the 5-link damped planar chain (theta = 5 masses + 5 damping
coefficients), T = 1000 steps at dt = 0.005, W = 20 shooting windows,
N = 16384 particles, adjoint checkpoint stride K = 1 (every pre-step state on
the tape) -- the largest particle count of the chain workload.  A step is log p + gradient of every particle
(rollout + adjoint + window reduction) followed by the SVGD + Adam update
(median bandwidth, phi, Adam).  Metric: particle-step-gradients per second =
N * T / step time (one unit = one particle x one time step, forward and
adjoint, with the SVGD update's time included).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pds|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Under torchrun each rank runs an independent
replica (the chain problems are independent; no collective on the data path).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2109_08815_gb300 import workloads as wlmod  # noqa: E402

METRIC = "particle-step-gradients/sec"
UNIT = "particle-steps/s"
N_DEFAULT = 16384
K_CKPT = 1  # every state on the tape: the reverse sweep recomputes nothing
FAST_MATH = 1  # __sincosf / __fdividef in the rollout (parity tests cover it at the same tolerances)
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def flops_per_particle_step(n: int, D: int, lengths: bool = True) -> tuple[int, int]:
    """Algorithmic FP32 flops of one time step of the n-link chain with D
    observed components (FMA = 2; sincos and reciprocals run on the MUFU and
    are not counted; operations on values that are zero by construction, at
    the ends of the chain, are not counted): the forward step with its
    observation term (the rank-1 link-frame articulated-body recursion,
    semi-implicit Euler, the residual and its running sum), and the reverse
    step (the observation seed, Euler's adjoint, one solve mu = H^-1 abar
    with the same rank-1 recursion, the closed-form gradient of mu^T ID).
    The two products that the kernel re-forms inside a fused multiply-add
    (qdd_i and mu_i, one per link after the first) and the checkpoint
    segment recompute of K > 1 are implementation costs and are not counted.
    The parameter adjoints are running sums over a window's steps, so their
    accumulation counts in full.  With lengths=False (no link length among
    the parameters) the reverse step leaves out the length adjoint, 9 flops
    per link.  tests/test_flopcount.py counts these operations by executing
    the step on a counting scalar that it first pins to the FP64 oracle."""
    drop = 0 if lengths else 9 * n
    if n == 1:
        return 19 + 3 * D, 66 + 3 * D - drop
    return 60 * n - 43 + 3 * D, 110 * n - 54 + 3 * D - drop


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x: float, device) -> float:
    """Maximum of a per-rank float over all ranks (the job's time is the
    slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_problem_inputs(N: int):
    wl = wlmod.chain5(N=N)
    return wl


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_rate(wl, obs, x, sample: int, threads: int):
    """FP64 oracle: log p + gradient of `sample` particles (full T), on the
    FP32 values of every input (those the GPU sees).  Returns the rate, the
    seconds taken, and the oracle's log p and gradient."""
    from oracle import pds_oracle as orc
    op = orc.Problem(mass=_f32(wl.mass), length=_f32(wl.length), damping=_f32(wl.damping),
                     theta_kind=wl.theta_kind, theta_link=wl.theta_link, dt=float(np.float32(wl.dt)), T=wl.T,
                     W=wl.W, obs=obs.astype(np.float64), obs_index=wl.obs_index, sigma_obs=wl.sigma_obs,
                     sigma_def=wl.sigma_def, s0=_f32(wl.s0), lo=_f32(wl.lo), hi=_f32(wl.hi),
                     g=float(np.float32(wl.g)), c_lim=wl.c_lim)
    xs = np.ascontiguousarray(_f32(x[:sample]))
    t0 = time.perf_counter()
    lp, g = op.loglik_grad(xs, threads=threads)
    dt = time.perf_counter() - t0
    return sample * wl.T / dt, dt, lp, g


def grad_error_in_tolerances(g, g_ref, M):
    """Largest |g - g_ref| over the per-component tolerance the parity tests
    use, 1e-3 |g_ref| + 1e-5 x the largest |g_ref| of the component's block
    (theta rows; shooting-state rows), per particle."""
    worst = 0.0
    for blk in (slice(0, M), slice(M, g.shape[1])):
        r = np.abs(g_ref[:, blk])
        tol = 1e-3 * r + 1e-5 * np.max(r, axis=1, keepdims=True)
        worst = max(worst, float(np.max(np.abs(g[:, blk] - g_ref[:, blk]) / np.maximum(tol, 1e-300))))
    return worst


def c0_posterior(api, dev, threads: int, iters: int = 100):
    """The double-pendulum configuration (N = 100, 100 iterations): the GPU's
    pds_iterate against the FP64 oracle's loop from the same particles.
    Returns the oracle's rate and the errors of the GPU's final theta
    moments."""
    import torch
    from oracle import metrics_oracle as mo
    from oracle import pds_oracle as orc
    wl = wlmod.double_pendulum(N=100)
    for name in ("mass", "length", "damping", "lo", "hi", "s0", "theta_true", "theta_init"):
        setattr(wl, name, _f32(getattr(wl, name)))
    wl.dt, wl.g = float(np.float32(wl.dt)), float(np.float32(wl.g))
    st = orc.simulate(wl.mass, wl.length, wl.damping, wl.s0, wl.dt, wl.T, g=wl.g)
    obs = wlmod.observations(wl, st).astype(np.float32)
    x = _f32(wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=7))
    prob = api.Problem.from_workload(wl, obs)
    sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr)
    X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).to(dev)
    api.iterate(prob, sv, X, iters)
    torch.cuda.synchronize()
    xg = X.cpu().numpy().T.astype(np.float64)
    sv.close()
    prob.close()
    op = orc.Problem(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                     theta_link=wl.theta_link, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64),
                     obs_index=wl.obs_index, sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo,
                     hi=wl.hi, g=wl.g, c_lim=wl.c_lim)
    ost = orc.SvgdState(wl.N, wl.P, wl.lo, wl.hi, lr=wl.lr)
    xo = np.ascontiguousarray(x.copy())
    t0 = time.perf_counter()
    for _ in range(iters):
        _, g = op.loglik_grad(xo, threads=threads)
        ost.step(xo, g)
    secs = time.perf_counter() - t0
    tg, to = xg[:, :wl.M], xo[:, :wl.M]
    mu_g, mu_o = tg.mean(0), to.mean(0)
    cg, co = np.cov(tg.T), np.cov(to.T)
    sd = np.sqrt(np.diag(co))
    ug, uo = (tg - wl.lo) / (wl.hi - wl.lo), (to - wl.lo) / (wl.hi - wl.lo)
    err = {"workload": "double pendulum, N=100, T=200, W=10, 100 SVGD iterations from the same particles",
           "mean_rel_err_max": float(np.max(np.abs(mu_g - mu_o) / np.abs(mu_o))),
           "cov_err_max_over_sd_sd": float(np.max(np.abs(cg - co) / np.outer(sd, sd))),
           "mmd2_unit_box": mo.mmd2_unbiased(ug, uo, orc.median_sqdist(uo)),
           "particle_max_abs_diff_over_box": float(np.max(np.abs(tg - to) / (wl.hi - wl.lo))),
           "tolerance": "means relative 5e-2; covariances 5e-2 sd_k sd_l"}
    rate = {"value": wl.N * wl.T * iters / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "svgd_iters_per_s": iters / secs,
            "sample": f"the whole double-pendulum configuration: {wl.N} particles x T={wl.T}, {iters} SVGD "
                      f"iterations (log p + gradient + SVGD step), {secs:.1f} s on {threads} threads"}
    return rate, err


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import pds_oracle as orc
    orc.build()
    wl = wlmod.chain5(N=args.n)
    # true trajectory: the oracle's own FP64 rollout of the true parameters
    st = orc.simulate(wl.mass, wl.length, wl.damping, wl.s0, wl.dt, wl.T, g=wl.g)
    obs = wlmod.observations(wl, st).astype(np.float32)
    x = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)
    threads = os.cpu_count() or 1
    sample = args.ref_sample
    op = orc.Problem(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                     theta_link=wl.theta_link, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64),
                     obs_index=wl.obs_index, sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo,
                     hi=wl.hi, g=wl.g, c_lim=wl.c_lim)
    xs = np.ascontiguousarray(x[:sample].astype(np.float64))
    svgd = orc.SvgdState(sample, wl.P, wl.lo, wl.hi, lr=wl.lr)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, g = op.loglik_grad(xs, threads=threads)
        svgd.step(xs, g)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = sum(times) / len(times)
    value = sample * wl.T / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(wl, args.n, note=f"FP64 CPU oracle, {sample}-particle sample per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{sample} particles x T={wl.T} (log p + gradient) + SVGD step on the sample"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(wl, N, note=None):
    c = {"workload": f"chain5 planar damped chain, N={N} particles, T={wl.T}, W={wl.W}, K={K_CKPT}",
         "system": "5-link planar chain, point masses, viscous damping", "N": N, "T": wl.T, "W": wl.W,
         "K": K_CKPT, "M": wl.M, "P": wl.P, "dt": wl.dt, "fast_math": bool(FAST_MATH),
         "l2": "flushed between timed steps (256 MiB device write outside the timed events)"}
    if note:
        c["note"] = note
    return c


def run_pds(args):
    import torch
    import torch.distributed as dist

    from paper_2109_08815_gb300 import api
    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.n
    wl = wlmod.chain5(N=N)
    stream = torch.cuda.Stream(device=dev)

    # --- synthetic observations: roll out the true parameters with f_sim
    with torch.cuda.stream(stream):
        gen = api.Problem.from_workload(wl, np.zeros((wl.T, wl.D), np.float32), stream=stream)
        th = torch.tensor(wl.theta_true, dtype=torch.float32, device=dev).reshape(wl.M, 1).contiguous()
        states = gen.simulate(th)
    stream.synchronize()
    obs = wlmod.observations(wl, states[:, :, 0].cpu().numpy().astype(np.float64)).astype(np.float32)
    gen.close()
    x0 = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)

    prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
    prob.reserve(N)
    svgd = api.Svgd(N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
    X = torch.from_numpy(np.ascontiguousarray(x0.T, dtype=np.float32)).to(dev)
    logp = torch.empty(N, device=dev)
    grad = torch.empty_like(X)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    L = api.lib()

    def step():
        rc = L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(grad), None)
        api._check(rc, "pds_loglik_grad")
        n1 = L.pds_last_launch_count()
        return n1

    def update():
        rc = L.pds_svgd_step(svgd.handle, api._ptr(X), api._ptr(grad), None, None)
        api._check(rc, "pds_svgd_step")
        return L.pds_last_launch_count()

    def iteration():
        # one SVGD iteration through the public call: the step's median phase
        # runs beside the likelihood, replayed from the iteration's graph
        rc = L.pds_iterate(prob.handle, svgd.handle, api._ptr(X), 1, api._ptr(logp))
        api._check(rc, "pds_iterate")
        return L.pds_last_launch_count()

    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            iteration()
            step()
            update()
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            e0, _, e2 = evs[k]
            e0.record(stream)
            launches += iteration()
            e2.record(stream)
    stream.synchronize()
    t_wall = time.perf_counter() - t_wall0
    # the breakdown (likelihood and SVGD step launched as two calls, each
    # event-timed): the roofline's kernel time
    evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            b0, b1, b2 = evb[k]
            b0.record(stream)
            step()
            b1.record(stream)
            update()
            b2.record(stream)
    stream.synchronize()
    clocks = sampler.stop()
    # particles whose log p was not finite in the last timed step (they sit
    # out the SVGD step), and particles with a non-finite entry after it
    nonfinite = {"logp_last_step": int((~torch.isfinite(logp)).sum().item()),
                 "particles_after": int((~torch.isfinite(X)).any(dim=0).sum().item())}
    torch.cuda.synchronize()
    step_ms = [evs[k][0].elapsed_time(evs[k][2]) for k in range(args.steps)]
    lg_ms = [evb[k][0].elapsed_time(evb[k][1]) for k in range(args.steps)]
    sv_ms = [evb[k][1].elapsed_time(evb[k][2]) for k in range(args.steps)]
    t_total = max_over_ranks(sum(step_ms) / 1e3, dev)
    if world > 1:
        dist.barrier()
    ms_per_step = t_total * 1e3 / args.steps
    value = world * N * wl.T * args.steps / t_total

    # --- end to end through the public C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        xh_t = torch.empty((wl.P, N), dtype=torch.float32, pin_memory=True)
        lh_t = torch.empty(N, dtype=torch.float32, pin_memory=True)
        xh, lh = xh_t.numpy(), lh_t.numpy()
        xh[...] = X.cpu().numpy()
        for _ in range(3):  # warm: the first calls set up and capture the host path's step
            api.iterate_host(prob, svgd, xh, 1, lh)
        ts = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            api.iterate_host(prob, svgd, xh, 1, lh)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(ts) / len(ts), dev)
        e2e = {"value": world * N * wl.T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": wl.P * N * 4,
               "d2h_bytes_per_step": wl.P * N * 4 + N * 4}

    # --- roofline of the dominant kernel (the fused rollout + adjoint)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    fwd, rev = flops_per_particle_step(wl.n, wl.D, lengths=bool(np.any(wl.theta_kind == wlmod.PARAM_LENGTH)))
    flops_launch = N * wl.T * (fwd + rev)
    lg_s = statistics.mean(lg_ms) / 1e3
    achieved = flops_launch / lg_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": TRAFFIC_BYTES_PER_LAUNCH,
                "kernel": "rollout_pair_kernel<5> (two particles per thread, no length adjoint; + window_reduce, 3%)",
                "peak_basis": f"FP32 {sm_count} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max_mhz:.0f} MHz "
                              "(MEASURED_PEAKS sm_max_mhz)",
                "flops_per_particle_step": fwd + rev,
                "loglik_grad_ms": statistics.mean(lg_ms), "svgd_step_ms": statistics.mean(sv_ms),
                "kernel_timing": "pds_loglik_grad and pds_svgd_step as separate event-timed calls, after the "
                                 "timed pds_iterate steps (in pds_iterate the step's median runs beside the "
                                 "likelihood)"}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (sm_count * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import pds_oracle as orc
        orc.build()
        threads = os.cpu_count() or 1
        sample = args.ref_sample_baseline
        rate, secs, lp_ref, g_ref = oracle_rate(wl, obs, x0, sample, threads)
        # the same oracle on one thread, on a smaller sample
        rate1, secs1, _, _ = oracle_rate(wl, obs, x0, 64, 1)
        c0_rate, c0_err = c0_posterior(api, dev, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{sample} particles x T={wl.T} log p + gradient (FP64, forward-mode "
                         f"duals), {secs:.1f} s on {threads} threads",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"64 particles x T={wl.T}, {secs1:.1f} s on 1 thread"},
               "double_pendulum": c0_rate}
        # the GPU's log p and gradient of the same particles, outside the timed region
        Xs = torch.from_numpy(np.ascontiguousarray(_f32(x0[:sample]).T, dtype=np.float32)).to(dev)
        with torch.cuda.stream(stream):
            lp_s, g_s, _ = prob.loglik_grad(Xs)
        stream.synchronize()
        lp_s = lp_s.cpu().numpy().astype(np.float64)
        g_s = g_s.cpu().numpy().T.astype(np.float64)
        errors = {"loglik_grad": {"workload": f"the benchmark workload's first {sample} initial particles",
                                  "logp_rel_err_max": float(np.max(np.abs(lp_s - lp_ref) / np.abs(lp_ref))),
                                  "logp_tolerance": 1e-4,
                                  "grad_err_max_in_tolerances": grad_error_in_tolerances(g_s, g_ref, wl.M),
                                  "grad_tolerance": "1e-3 |g_ref| + 1e-5 max |g_ref| of the block, per component"},
                  "posterior_double_pendulum": c0_err}

    extra = {}
    if rank == 0 and world == 1 and not args.no_batched:
        extra["batched"] = run_batched(api, dev, stream)
    if rank == 0 and world == 1 and not args.no_serving:
        extra["serving"] = run_serving(api, dev, stream)
        extra["serving"]["other_rates"] = [run_serving(api, dev, stream, rate=r, brief=True) for r in (5.0, 200.0)]
        extra["serving"]["gated"] = run_serving(api, dev, stream, gate=True)
    if rank == 0 and world == 1 and not args.no_csvgd:
        extra["csvgd"] = run_csvgd(api, dev, stream, wl, obs, x0, flush)
    if rank == 0 and world == 1 and not args.no_sgld:
        extra["sgld"] = run_sgld(api, dev, stream, wl, obs, x0, flush)
    if rank == 0 and world == 1 and not args.no_rigid:
        extra["rigid_double_pendulum"] = run_rigid2(api, dev, stream, flush)
    if rank == 0 and world == 1 and not args.no_trajset:
        extra["trajectory_set"] = run_trajset(api, dev, stream, flush)
    if rank == 0 and world == 1 and not args.no_metrics:
        extra["metrics"] = run_metrics(api, dev, X, wl)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(wl, N),
            "svgd_iters_per_sec": 1e3 / ms_per_step, "gpu_launches": launches, "e2e": e2e,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "wall_s_timed": t_wall,
            "error_vs_oracle": errors, "nonfinite_particles": nonfinite,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _gen_obs(api, wl, dev, stream):
    """Observations from the library's own f_sim of the true parameters."""
    import torch
    with torch.cuda.stream(stream):
        gen = api.Problem.from_workload(wl, np.zeros((wl.T, wl.D), np.float32), stream=stream)
        th = torch.tensor(wl.theta_true, dtype=torch.float32, device=dev).reshape(wl.M, 1).contiguous()
        states = gen.simulate(th)
    stream.synchronize()
    obs = wlmod.observations(wl, states[:, :, 0].cpu().numpy().astype(np.float64)).astype(np.float32)
    gen.close()
    return obs


def run_batched(api, dev, stream, n_jobs=64, iters=10):
    """64 uneven problems: batched (persistent launches + graph, autotuned)
    against the plain path (each problem's iteration launched separately)."""
    import torch
    wls = wlmod.batched_problems(n_jobs=n_jobs, seed=4000)
    obs = [_gen_obs(api, w, dev, stream) for w in wls]
    x0 = [np.ascontiguousarray(wlmod.initial_particles(w, o.astype(np.float64), rng_seed=1).T, dtype=np.float32)
          for w, o in zip(wls, obs)]
    units = sum(w.N * w.T for w in wls)
    probs = [api.Problem.from_workload(w, o, stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
             for w, o in zip(wls, obs)]
    svgds = [api.Svgd(w.N, w.M, w.P, w.lo, w.hi, lr=w.lr, stream=stream) for w in wls]
    Xs = [torch.from_numpy(x).to(dev) for x in x0]
    b = api.Batch(probs, svgds, Xs, stream=stream)
    t_tune = time.perf_counter()
    choices = b.autotune(allow_fast_math=bool(FAST_MATH))
    t_tune = time.perf_counter() - t_tune
    b.iterate(3)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.iterate(iters)
    e1.record(stream)
    e1.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3 / iters
    ng, lpi = b.info()
    b.close()
    # plain: same problems, one after another, separate launches per iteration
    Xp = [torch.from_numpy(x).to(dev) for x in x0]
    for p, s, x in zip(probs, svgds, Xp):
        s.reset()
        api.iterate(p, s, x, 1)
    stream.synchronize()
    e0.record(stream)
    for _ in range(2):
        for p, s, x in zip(probs, svgds, Xp):
            api.iterate(p, s, x, 1)
    e1.record(stream)
    e1.synchronize()
    t_p = e0.elapsed_time(e1) / 1e3 / 2
    for o in probs + svgds:
        o.close()
    return {"workload": f"{n_jobs} uneven problems: chains of 2-8 links, T 100-2000, W 5-50, N 64-4096 "
                        "(log-uniform), pendulum/damped parameter types 50/50",
            "particle_steps_per_iter": units, "value": units / t_b, "unit": UNIT, "ms_per_iter": t_b * 1e3,
            "plain_value": units / t_p, "plain_ms_per_iter": t_p * 1e3, "speedup_vs_plain": t_p / t_b,
            "chain_length_groups": ng, "launches_per_iter_in_graph": lpi,
            "autotune": [{"links": c[0], "K": c[1], "fast_math": c[2], "grid_blocks": c[3], "units_per_thread": c[4]}
                         for c in choices],
            "autotune_s": t_tune}


def run_csvgd(api, dev, stream, wl, obs, x0, flush, iters=10, warmup=3):
    """Constrained SVGD (Sec. IV-E, Algorithm 1) on the benchmark workload:
    log p_obs with the defect and limit constraints' MDMM gradient (second
    adjoint), then the constrained update; multipliers start at zero."""
    import torch
    N = wl.N
    prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
    prob.set_csvgd(True, 1.0)
    prob.reserve(N)
    sv = api.Svgd(N, wl.M, prob.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
    sv.set_csvgd(wl.W - 1)
    # the headline run's particles (shooting states from the observations),
    # multipliers 0; particles whose rollout diverges sit out the SVGD steps
    xa = np.concatenate([np.ascontiguousarray(x0.T, dtype=np.float32),
                         np.zeros((prob.P - wl.P, N), np.float32)], axis=0)
    X = torch.from_numpy(np.ascontiguousarray(xa)).to(dev)
    logp = torch.empty(N, device=dev)
    G = torch.empty((prob.grad_rows, N), device=dev)
    status = torch.empty(N, dtype=torch.int32, device=dev)
    L = api.lib()

    def lg():
        api._check(L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(G), None), "csvgd loglik")

    def up():
        api._check(L.pds_svgd_step(sv.handle, api._ptr(X), api._ptr(G), None, None), "csvgd step")

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lg()
            up()
    stream.synchronize()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(iters)]
    with torch.cuda.stream(stream):
        for k in range(iters):
            flush.zero_()
            evs[k][0].record(stream)
            lg()
            evs[k][1].record(stream)
            up()
            evs[k][2].record(stream)
    stream.synchronize()
    tot = sum(e[0].elapsed_time(e[2]) for e in evs) / iters
    lgt = sum(e[0].elapsed_time(e[1]) for e in evs) / iters
    with torch.cuda.stream(stream):
        api._check(L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(G), api._ptr(status)),
                   "csvgd loglik")
    stream.synchronize()
    nonfinite = int((status != 0).sum().item())
    sv.close()
    prob.close()
    return {"workload": f"constrained SVGD (MDMM, c = 1) on the chain5 workload, N={N}, T={wl.T}, W={wl.W}, "
                        f"K={K_CKPT}; particles carry {wl.W - 1} defect and {wl.M} limit multipliers",
            "value": N * wl.T / (tot / 1e3), "unit": UNIT, "ms_per_iter": tot, "loglik_grad_ms": lgt,
            "svgd_step_ms": tot - lgt, "iters": iters,
            "init": "the headline run's particles; multipliers 0",
            "nonfinite_particles_after": nonfinite}


def run_sgld(api, dev, stream, wl, obs, x0, flush, iters=10, warmup=3):
    """SGLD chains (the other estimator of Sec. V-B) on the multiple-shooting
    likelihood of the benchmark workload: per iteration log p + gradient of
    every particle, then one Langevin step of every chain."""
    import torch
    N, P = wl.N, wl.P
    prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
    prob.reserve(N)
    sg = api.Sgld(N, wl.M, P, wl.lo, wl.hi, a=1e-7, b=1.0, gamma=0.55, seed=2021, stream=stream)
    X = torch.from_numpy(np.ascontiguousarray(x0.T, dtype=np.float32)).to(dev)
    logp = torch.empty(N, device=dev)
    G = torch.empty((P, N), device=dev)
    L = api.lib()
    # theta rows from the Sobol sequence over the box (App. A-A), on the device
    api.sobol_box(X[:wl.M], wl.lo, wl.hi, stream=stream)  # first launch loads the module
    sob = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(2)) for _ in range(5)]
    for e0, e1 in sob:
        e0.record(stream)
        api.sobol_box(X[:wl.M], wl.lo, wl.hi, stream=stream)
        e1.record(stream)
    stream.synchronize()
    sobol_us = 1e3 * sum(e0.elapsed_time(e1) for e0, e1 in sob) / len(sob)

    def lg():
        api._check(L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(G), None), "sgld loglik")

    def up():
        api._check(L.pds_sgld_step(sg.handle, api._ptr(X), api._ptr(G), None), "sgld step")

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lg()
            up()
    stream.synchronize()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(iters)]
    with torch.cuda.stream(stream):
        for k in range(iters):
            flush.zero_()
            evs[k][0].record(stream)
            lg()
            evs[k][1].record(stream)
            up()
            evs[k][2].record(stream)
    stream.synchronize()
    tot = sum(e[0].elapsed_time(e[2]) for e in evs) / iters
    lgt = sum(e[0].elapsed_time(e[1]) for e in evs) / iters
    step_ms = tot - lgt
    nonfinite = int((~torch.isfinite(X)).any(dim=0).sum().item())
    sg.close()
    prob.close()
    return {"workload": f"SGLD on the chain5 workload, N={N} chains, T={wl.T}, W={wl.W}, K={K_CKPT}, "
                        f"eps_t = 1e-7 (1 + t)^-0.55; theta initialised from the Sobol sequence over the box",
            "value": N * wl.T / (tot / 1e3), "unit": UNIT, "ms_per_iter": tot, "loglik_grad_ms": lgt,
            "sgld_step_ms": step_ms, "sgld_step_gbs": 12.0 * P * N / (step_ms / 1e3) / 1e9, "iters": iters,
            "sobol_init_us": sobol_us,
            "nonfinite_chains_after": nonfinite}


def run_rigid2(api, dev, stream, flush, N=16384, iters=10, warmup=3):
    """The physical double pendulum's 11-parameter rigid-body model (Sec. V,
    synthetic): per iteration log p + gradient of N particles (the rigid
    system's reverse sweep) and the SVGD update over the 11 parameters;
    theta rows start from the Sobol sequence over the limits (App. A-A)."""
    import torch
    wl = wlmod.rigid_double_pendulum(N=N)
    obs = _gen_obs(api, wl, dev, stream)
    x0 = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)
    prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
    prob.reserve(N)
    sv = api.Svgd(N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
    X = torch.from_numpy(np.ascontiguousarray(x0.T, dtype=np.float32)).to(dev)
    api.sobol_box(X[:wl.M], wl.lo, wl.hi, stream=stream)
    logp = torch.empty(N, device=dev)
    G = torch.empty((wl.P, N), device=dev)
    L = api.lib()

    def lg():
        api._check(L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(G), None), "rigid loglik")

    def up():
        api._check(L.pds_svgd_step(sv.handle, api._ptr(X), api._ptr(G), None, None), "rigid step")

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lg()
            up()
    stream.synchronize()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(iters)]
    with torch.cuda.stream(stream):
        for k in range(iters):
            flush.zero_()
            evs[k][0].record(stream)
            lg()
            evs[k][1].record(stream)
            up()
            evs[k][2].record(stream)
    stream.synchronize()
    tot = sum(e[0].elapsed_time(e[2]) for e in evs) / iters
    lgt = sum(e[0].elapsed_time(e[1]) for e in evs) / iters
    nonfinite = int((~torch.isfinite(logp)).sum().item())
    sv.close()
    prob.close()
    return {"workload": f"rigid double pendulum, 11 parameters (masses, inertias, COMs, frictions, joint offset), "
                        f"N={N}, T={wl.T} at 400 Hz, W={wl.W}, K={K_CKPT}; Sobol initialisation",
            "value": N * wl.T / (tot / 1e3), "unit": UNIT, "ms_per_iter": tot, "loglik_grad_ms": lgt,
            "svgd_step_ms": tot - lgt, "iters": iters, "nonfinite_particles": nonfinite}


def run_trajset(api, dev, stream, flush, N=8192, R=2, iters=10, warmup=3):
    """Likelihood of a set of R trajectories (Sec. IV-C, the equally weighted
    mixture) on the chain5 system: R trajectories from R parameter draws and
    start states, N particles each carrying R sets of shooting states."""
    import dataclasses

    import torch
    wl = wlmod.chain5(N=N)
    rng = np.random.default_rng(7000)
    wls = [wl] + [dataclasses.replace(wl, theta_true=rng.uniform(wl.lo, wl.hi),
                                      s0=np.concatenate([rng.uniform(-1.0, 1.0, wl.n), np.zeros(wl.n)]),
                                      noise=rng.standard_normal(wl.noise.shape)) for _ in range(R - 1)]
    obs = np.stack([_gen_obs(api, w, dev, stream) for w in wls])
    s0s = np.stack([w.s0 for w in wls]).astype(np.float32)
    prob = api.Problem.from_workload(wl, obs[0], stream=stream, checkpoint_stride=K_CKPT, fast_math=FAST_MATH)
    prob.set_trajectories(obs, s0s, "sum")
    prob.reserve(N)
    parts = [wlmod.initial_particles(w, o.astype(np.float64), rng_seed=1) for w, o in zip(wls, obs)]
    x = np.concatenate([parts[0][:, :wl.M]] + [p[:, wl.M:] for p in parts], axis=1)
    X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).to(dev)
    sv = api.Svgd(N, wl.M, prob.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
    logp = torch.empty(N, device=dev)
    G = torch.empty((prob.P, N), device=dev)
    L = api.lib()

    def lg():
        api._check(L.pds_loglik_grad(prob.handle, api._ptr(X), N, api._ptr(logp), api._ptr(G), None), "set loglik")

    def up():
        api._check(L.pds_svgd_step(sv.handle, api._ptr(X), api._ptr(G), None, None), "set step")

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lg()
            up()
    stream.synchronize()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(iters)]
    with torch.cuda.stream(stream):
        for k in range(iters):
            flush.zero_()
            evs[k][0].record(stream)
            lg()
            evs[k][1].record(stream)
            up()
            evs[k][2].record(stream)
    stream.synchronize()
    tot = sum(e[0].elapsed_time(e[2]) for e in evs) / iters
    lgt = sum(e[0].elapsed_time(e[1]) for e in evs) / iters
    sv.close()
    prob.close()
    return {"workload": f"set of {R} chain5 trajectories (equally weighted mixture), N={N}, T={wl.T}, W={wl.W}, "
                        f"K={K_CKPT}; each particle carries {R} sets of shooting states",
            "value": N * R * wl.T / (tot / 1e3), "unit": UNIT, "ms_per_iter": tot, "loglik_grad_ms": lgt,
            "svgd_step_ms": tot - lgt, "iters": iters}


def run_metrics(api, dev, X, wl, reps=5):
    """Posterior metrics on the benchmark's particles: KNN-KL (k = 3) and the
    unbiased MMD^2 of the N particles' theta against a reference sample of the
    same size (particles jittered by 1 % of the box), event-timed."""
    import torch
    N = X.shape[1]
    P = X[:wl.M].contiguous()
    width = torch.tensor(wl.hi - wl.lo, dtype=torch.float32, device=dev).reshape(-1, 1)
    g = torch.Generator(device=dev).manual_seed(8000)
    Q = (P + 0.01 * width * torch.randn(P.shape, generator=g, device=dev)).contiguous()
    h = float(np.mean((wl.hi - wl.lo) ** 2))
    out = {}
    for name, fn in (("knn_kl", lambda: api.knn_kl(P, Q, k=3)), ("mmd2", lambda: api.mmd2(P, Q, h))):
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            v = fn()
            ts.append(time.perf_counter() - t0)
        out[name] = {"value": v, "ms": 1e3 * float(np.median(ts))}
    out["workload"] = f"{N} particles' theta (d = {wl.M}) against {N} jittered copies"
    return out


def run_serving(api, dev, stream, n_jobs=48, rate=50.0, iters=300, brief=False, gate=False):
    """Poisson arrivals of jobs from the uneven-problem distribution, each
    run to `iters` SVGD iterations: continuous batching against one job at a
    time with plain launches."""
    from paper_2109_08815_gb300 import serve
    wls = wlmod.serving_mix(n_jobs=n_jobs, seed=5000)
    jobs = []
    for w in wls:
        o = _gen_obs(api, w, dev, stream)
        jobs.append((w, o, wlmod.initial_particles(w, o.astype(np.float64), rng_seed=1), iters))
    arrivals = serve.poisson_arrivals(n_jobs, rate, seed=5000)
    units = sum(w.N * w.T for w in wls) * iters
    lat_s, _, wall_s = serve.run_server(jobs, arrivals, mem_budget=64 << 30, stream=stream,
                                        checkpoint_stride=K_CKPT, fast_math=bool(FAST_MATH))
    lat_p, _, wall_p = serve.run_plain(jobs, arrivals, checkpoint_stride=K_CKPT, fast_math=bool(FAST_MATH),
                                       stream=stream)
    n_arm = sum(1 for w in wls if hasattr(w, "arm_len"))
    if gate:
        # the convergence gate: MMD^2 between theta snapshots 10 iterations
        # apart (unit-box coordinates, bandwidth 1/6 per coordinate) at or
        # below 0 retires a job before its iteration cap
        used = []
        lat_g, _, wall_g = serve.run_server(jobs, arrivals, mem_budget=64 << 30, stream=stream,
                                            checkpoint_stride=K_CKPT, fast_math=bool(FAST_MATH),
                                            gate=(1, 10, 0.0, 1.0 / 6.0), iters_out=used)
        units_g = sum(w.N * w.T * k for w, k in zip(wls, used))
        return {"gate": "MMD^2 (unbiased, RBF, bandwidth M/6 in unit-box coordinates) between theta snapshots "
                        "10 iterations apart <= 0", "rate_per_s": rate,
                "served": {**serve.percentiles(lat_g), "value": units_g / wall_g, "wall_s": wall_g},
                "iterations_mean": float(np.mean(used)), "iterations_min": int(np.min(used)),
                "jobs_at_cap": int(sum(1 for k in used if k >= iters))}
    if brief:
        return {"rate_per_s": rate, "served": {**serve.percentiles(lat_s), "value": units / wall_s},
                "plain_sequential": {**serve.percentiles(lat_p), "value": units / wall_p}}
    return {"workload": f"{n_jobs} jobs, Poisson arrivals at {rate:g}/s, {iters} SVGD iterations each: "
                        f"{n_jobs - n_arm} uneven chain problems, {n_arm} arm-box jobs at 512 particles",
            "served": {**serve.percentiles(lat_s), "value": units / wall_s, "wall_s": wall_s},
            "plain_sequential": {**serve.percentiles(lat_p), "value": units / wall_p, "wall_s": wall_p},
            "unit": UNIT, "time_to_posterior": "arrival to final particles on the host"}


# dram bytes (read + write) per full-size rollout launch, from the committed
# ncu capture of this kernel (set to None when the kernel changes)
TRAFFIC_BYTES_PER_LAUNCH = 362851328 + 655211776


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pds", choices=["pds", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-problems measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-csvgd", action="store_true", help="skip the constrained-SVGD measurement")
    ap.add_argument("--no-sgld", action="store_true", help="skip the SGLD measurement")
    ap.add_argument("--no-rigid", action="store_true", help="skip the rigid double pendulum measurement")
    ap.add_argument("--no-trajset", action="store_true", help="skip the trajectory-set measurement")
    ap.add_argument("--no-metrics", action="store_true", help="skip the posterior-metric timing")
    ap.add_argument("--ref-sample", type=int, default=64, help="particles per reference-arm step")
    ap.add_argument("--ref-sample-baseline", type=int, default=4096, help="particles in the cpu_baseline sample")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_pds(args)


if __name__ == "__main__":
    sys.exit(main())
