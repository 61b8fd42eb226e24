"""Small, self-contained invocations of the hot path for profiling one kernel
at a time (for example under ``ncu -k``), on seeded synthetic inputs.

    python -m paper_2109_08815_gb300.profile_cases rollout [--n 4096] [--calls 2]
        pds_loglik_grad on the 5-link damped chain (T = 1000, W = 20, K = 1,
        fast math) with N particles: ``--calls`` launches of rollout_kernel
        and window_reduce_kernel.

    python -m paper_2109_08815_gb300.profile_cases csvgd [--n 16384] [--steps 3]
        constrained SVGD (Sec. IV-E) on the same chain (K = 1): --steps iterations of
        pds_loglik_grad (two adjoints) and pds_svgd_step, multipliers from 0.

    python -m paper_2109_08815_gb300.profile_cases svgd [--n 16384] [--m 10] [--steps 3]
        pds_svgd_step on N particles in the unit box with M kernel
        coordinates: per step the median passes (median_tc_kernel for
        N >= 2048) and phi (phi_tc_kernel for N >= 256).

    python -m paper_2109_08815_gb300.profile_cases rigid2 [--n 4096] [--calls 2]
        pds_loglik_grad on the 11-parameter rigid double pendulum (T = 1000
        at 400 Hz, W = 10, K = 1, fast math): rigid2_rollout_kernel and
        window_reduce_kernel.

    python -m paper_2109_08815_gb300.profile_cases sgld [--n 16384] [--steps 3]
        pds_sgld_step on N chains of the chain5 layout (P = 200 rows) with a
        seeded gradient: sgld_kernel.

Each case runs on cuda:0 and exits 0 after a device synchronisation.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import api
from . import workloads as wlmod


def rollout_case(n: int, calls: int) -> float:
    wl = wlmod.chain5(N=n)
    dev = torch.device("cuda")
    gen = api.Problem.from_workload(wl, np.zeros((wl.T, wl.D), np.float32))
    th = torch.tensor(wl.theta_true, dtype=torch.float32, device=dev).reshape(wl.M, 1).contiguous()
    states = gen.simulate(th)
    torch.cuda.synchronize()
    obs = wlmod.observations(wl, states[:, :, 0].cpu().numpy().astype(np.float64)).astype(np.float32)
    gen.close()
    x0 = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)
    X = torch.from_numpy(np.ascontiguousarray(x0.T, dtype=np.float32)).to(dev)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=1, fast_math=1)
    logp = torch.empty(n, device=dev)
    G = torch.empty_like(X)
    for _ in range(calls):
        prob.loglik_grad(X, out=(logp, G, None))
    torch.cuda.synchronize()
    out = float(logp.sum())
    prob.close()
    return out


def csvgd_case(n: int, steps: int) -> float:
    wl = wlmod.chain5(N=n)
    dev = torch.device("cuda")
    gen = api.Problem.from_workload(wl, np.zeros((wl.T, wl.D), np.float32))
    th = torch.tensor(wl.theta_true, dtype=torch.float32, device=dev).reshape(wl.M, 1).contiguous()
    states = gen.simulate(th)
    torch.cuda.synchronize()
    obs = wlmod.observations(wl, states[:, :, 0].cpu().numpy().astype(np.float64)).astype(np.float32)
    gen.close()
    x0 = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=1, fast_math=1)
    prob.set_csvgd(True, 1.0)
    sv = api.Svgd(n, wl.M, prob.P, wl.lo, wl.hi, lr=wl.lr)
    sv.set_csvgd(wl.W - 1)
    xa = np.concatenate([np.ascontiguousarray(x0.T, dtype=np.float32), np.zeros((prob.P - wl.P, n), np.float32)])
    X = torch.from_numpy(np.ascontiguousarray(xa)).to(dev)
    G = torch.empty((prob.grad_rows, n), device=dev)
    logp = torch.empty(n, device=dev)
    bw = None
    for _ in range(steps):
        prob.loglik_grad(X, out=(logp, G, None))
        bw, _ = sv.step(X, G)
    torch.cuda.synchronize()
    out = float(bw.item())
    sv.close()
    prob.close()
    return out


def rigid2_case(n: int, calls: int) -> float:
    wl = wlmod.rigid_double_pendulum(N=n)
    dev = torch.device("cuda")
    gen = api.Problem.from_workload(wl, np.zeros((wl.T, wl.D), np.float32))
    th = torch.tensor(wl.theta_true, dtype=torch.float32, device=dev).reshape(wl.M, 1).contiguous()
    states = gen.simulate(th)
    torch.cuda.synchronize()
    obs = wlmod.observations(wl, states[:, :, 0].cpu().numpy().astype(np.float64)).astype(np.float32)
    gen.close()
    x0 = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=1)
    X = torch.from_numpy(np.ascontiguousarray(x0.T, dtype=np.float32)).to(dev)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=1, fast_math=1)
    logp = torch.empty(n, device=dev)
    G = torch.empty_like(X)
    for _ in range(calls):
        prob.loglik_grad(X, out=(logp, G, None))
    torch.cuda.synchronize()
    out = float(logp.sum())
    prob.close()
    return out


def sgld_case(n: int, steps: int) -> float:
    wl = wlmod.chain5(N=8)
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.uniform(size=(wl.P, n)).astype(np.float32)).cuda()
    G = torch.from_numpy(rng.normal(size=(wl.P, n)).astype(np.float32)).cuda()
    sg = api.Sgld(n, wl.M, wl.P, wl.lo, wl.hi, a=1e-4, seed=1)
    for _ in range(steps):
        sg.step(X, G)
    torch.cuda.synchronize()
    out = float(X.sum())
    sg.close()
    return out


def svgd_case(n: int, m: int, steps: int) -> float:
    P = 200 if m <= 200 else m
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.uniform(size=(P, n)).astype(np.float32)).cuda()
    G = torch.from_numpy((1e3 * rng.normal(size=(P, n))).astype(np.float32)).cuda()
    sv = api.Svgd(n, m, P, np.zeros(m), np.ones(m))
    bw = None
    for _ in range(steps):
        bw, _ = sv.step(X, G)
    torch.cuda.synchronize()
    out = float(bw.item())
    sv.close()
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["rollout", "svgd", "csvgd", "rigid2", "sgld"])
    ap.add_argument("--n", type=int, default=None, help="particles (rollout 4096, svgd 16384 by default)")
    ap.add_argument("--m", type=int, default=10, help="kernel coordinates (svgd)")
    ap.add_argument("--calls", type=int, default=2, help="pds_loglik_grad calls (rollout)")
    ap.add_argument("--steps", type=int, default=3, help="pds_svgd_step calls (svgd)")
    a = ap.parse_args(argv)
    if a.case == "rollout":
        v = rollout_case(a.n or 4096, a.calls)
        print(f"rollout ok: sum log p = {v:.6e}")
    elif a.case == "rigid2":
        v = rigid2_case(a.n or 4096, a.calls)
        print(f"rigid2 ok: sum log p = {v:.6e}")
    elif a.case == "sgld":
        v = sgld_case(a.n or 16384, a.steps)
        print(f"sgld ok: sum x = {v:.6e}")
    elif a.case == "csvgd":
        v = csvgd_case(a.n or 16384, a.steps)
        print(f"csvgd ok: bandwidth = {v:.6e}")
    else:
        v = svgd_case(a.n or 16384, a.m, a.steps)
        print(f"svgd ok: bandwidth = {v:.6e}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
