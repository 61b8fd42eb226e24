"""Shared test helpers: build the same seeded problem for the oracle and the
CUDA library, and compare their results with the stated tolerances.

Tolerances (FP32 GPU path vs FP64 oracle on identical FP32-representable
inputs):
  * log p: |dlogp| <= 1e-4 * |logp_ref| per particle.
  * gradient: per particle and per block (theta rows; shooting-state rows),
    max_k |g_k - g_ref_k| <= 1e-3 * max_k |g_ref_k|.
"""
from __future__ import annotations

import numpy as np

from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import workloads as wlmod

LOGP_RTOL = 1e-4
GRAD_RTOL = 1e-3


def physical(wl, theta):
    m, l, b = wl.mass.copy(), wl.length.copy(), wl.damping.copy()
    for k, (kind, i) in enumerate(zip(wl.theta_kind, wl.theta_link)):
        {0: m, 1: l, 2: b}[int(kind)][i] = theta[k]
    return m, l, b


def observations(wl):
    m, l, b = physical(wl, wl.theta_true)
    return wlmod.observations(wl, orc.simulate(m, l, b, wl.s0, wl.dt, wl.T, g=wl.g)).astype(np.float32)


def oracle_problem(wl, obs):
    return orc.Problem(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                       theta_link=wl.theta_link, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64),
                       obs_index=wl.obs_index, sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0,
                       lo=wl.lo, hi=wl.hi, g=wl.g, c_lim=wl.c_lim)


def f32_workload(wl):
    """Round every real input to float32 so both sides see the same numbers."""
    for name in ("mass", "length", "damping", "lo", "hi", "s0", "theta_true", "theta_init"):
        setattr(wl, name, getattr(wl, name).astype(np.float32).astype(np.float64))
    wl.dt = float(np.float32(wl.dt))
    wl.g = float(np.float32(wl.g))
    return wl


def particles(wl, obs, seed=7):
    return wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=seed).astype(np.float32).astype(np.float64)


def assert_logp_close(lp, lp_ref, rtol=LOGP_RTOL):
    rel = np.abs(lp - lp_ref) / np.abs(lp_ref)
    assert np.all(rel <= rtol), f"max rel logp err {rel.max():.3e} at particle {int(rel.argmax())}"
    return rel.max()


def assert_grad_close(g, g_ref, M, rtol=GRAD_RTOL):
    worst = 0.0
    blocks = [slice(0, M)] + ([slice(M, g.shape[1])] if g.shape[1] > M else [])
    for blk in blocks:
        a, r = g[:, blk], g_ref[:, blk]
        scale = np.max(np.abs(r), axis=1)
        err = np.max(np.abs(a - r), axis=1) / np.maximum(scale, 1e-30)
        worst = max(worst, err.max())
        assert np.all(err <= rtol), f"max grad err {err.max():.3e} (block {blk}) at particle {int(err.argmax())}"
    return worst
