"""Shared test helpers: build the same seeded problem for the oracle and the
CUDA library, and compare their results with the stated tolerances.

Tolerances (FP32 GPU path vs FP64 oracle on identical FP32-representable
inputs):
  * log p: |dlogp| <= 1e-4 * |logp_ref| per particle.  Where log p passes
    near zero (its Gaussian normalising constants and the box density
    cancel against the residual terms), a bound relative to log p itself
    is not one that any rounding of the sum can meet; callers that may meet
    such particles pass the constant part C (logp_constant) and the bound
    is 1e-4 * max(|logp_ref|, |C|), relative to the larger of the two
    terms that cancel.
  * gradient, per component k of a particle:
        |g_k - g_ref_k| <= 1e-3 * |g_ref_k| + GRAD_FLOOR * max_{k' in B} |g_ref_k'|,
    B the component's block (theta rows, or shooting-state rows).  The
    floor is the absolute error of FP32 arithmetic: the adjoint sums
    O(h) products whose magnitudes are those of the block's largest
    component, each carrying relative rounding of 2^-24 times the growth of
    a window's rollout, so a component far below the block's largest one is
    known to that absolute accuracy only.
  * phi (Eq. 1): |phi - phi_ref| <= PHI_TOL * max |phi_ref| per entry.
"""
from __future__ import annotations

import numpy as np

from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import workloads as wlmod

LOGP_RTOL = 1e-4
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-5
PHI_TOL = 5e-4


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


def logp_constant(wl):
    """The part of log p that no particle changes: the Gaussian normalising
    constants of the T observation terms (Eq. 2) and of the W - 1 defect
    terms (Eq. 4), and the log density of the uniform prior box."""
    D = len(wl.obs_index)
    c = -0.5 * D * wl.T * np.log(2.0 * np.pi * wl.sigma_obs ** 2)
    c += -0.5 * wl.S * (wl.W - 1) * np.log(2.0 * np.pi * wl.sigma_def ** 2)
    return c - float(np.sum(np.log(np.asarray(wl.hi, np.float64) - np.asarray(wl.lo, np.float64))))


def assert_logp_close(lp, lp_ref, rtol=LOGP_RTOL, const=None):
    scale = np.abs(lp_ref) if const is None else np.maximum(np.abs(lp_ref), abs(const))
    rel = np.abs(lp - lp_ref) / scale
    assert np.all(rel <= rtol), f"max rel logp err {rel.max():.3e} at particle {int(rel.argmax())}"
    return rel.max()


def grad_tolerance(g_ref, M, rtol=GRAD_RTOL, floor=GRAD_FLOOR):
    """Per-entry tolerance of a gradient [N][P] (see the module docstring)."""
    tol = np.empty_like(g_ref)
    blocks = [slice(0, M)] + ([slice(M, g_ref.shape[1])] if g_ref.shape[1] > M else [])
    for blk in blocks:
        r = np.abs(g_ref[:, blk])
        tol[:, blk] = rtol * r + floor * np.max(r, axis=1, keepdims=True)
    return tol


def assert_grad_close(g, g_ref, M, rtol=GRAD_RTOL, floor=GRAD_FLOOR):
    """Every component within its tolerance; returns the largest error in
    units of the tolerance."""
    tol = grad_tolerance(g_ref, M, rtol, floor)
    ratio = np.abs(g - g_ref) / np.maximum(tol, 1e-300)
    i, k = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert ratio[i, k] <= 1.0, (f"grad component {k} of particle {i}: {g[i, k]:.7g} vs {g_ref[i, k]:.7g} "
                                f"({ratio[i, k]:.2f} x its tolerance)")
    return float(ratio.max())


def phi_tolerance(u, g_u, bw, g_tol_u):
    """Per-entry tolerance [N][M] of phi (Eq. 1) computed from a gradient
    that is itself known to g_tol_u (unit-box coordinates, e.g. the GPU's
    FP32 gradient against the oracle's): PHI_TOL * max |phi| for phi's own
    arithmetic, plus (1/N) sum_j k_ij g_tol_j, the most the gradient error
    can move the kernel-weighted sum (the repulsion term does not involve
    the gradient)."""
    phi = orc.svgd_phi(u, g_u, bw)
    rep = orc.svgd_phi(u, np.zeros_like(g_u), bw)
    carried = orc.svgd_phi(u, g_tol_u, bw) - rep
    return PHI_TOL * np.max(np.abs(phi)) + carried


def update_tolerance(x, width):
    """FP32 Adam update of an entry against the FP64 update with the same
    directions: x (and, for theta, u = (theta - lo) / w and back) rounded to
    2^-24 relative a few times, the step lr m^/(sqrt(v^) + eps) to a few ulp."""
    return 4e-7 * (np.abs(x) + width)
