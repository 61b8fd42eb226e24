"""log p as a differentiable torch op (api.loglik, a torch.autograd.Function
around pds_loglik_grad): its backward pass returns the hand-written adjoint's
gradient (Appendix B-A) scaled by the incoming gradient, grad_out[i] times
d log p_i / d particles_i, in the particles' [P][N] layout.  Checked against
the FP64 oracle's gradient at the gradient tolerance."""
import numpy as np
import pytest
import torch

from helpers import assert_logp_close, f32_workload, grad_tolerance, observations, oracle_problem, particles
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _setup(N=64):
    wl = f32_workload(wlmod.double_pendulum(N=N))
    obs = observations(wl)
    x = particles(wl, obs)
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x, threads=8)
    return wl, obs, x, lp_ref, g_ref


def test_backward_of_the_sum_is_the_gradient():
    wl, obs, x, lp_ref, g_ref = _setup()
    prob = api.Problem.from_workload(wl, obs)
    X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).cuda().requires_grad_(True)
    lp = api.loglik(X, prob)
    assert lp.shape == (wl.N,) and lp.requires_grad
    lp.sum().backward()
    assert X.grad.shape == X.shape
    assert_logp_close(lp.detach().cpu().numpy().astype(np.float64), lp_ref)
    g = X.grad.cpu().numpy().T.astype(np.float64)
    tol = grad_tolerance(g_ref, wl.M)
    assert np.all(np.abs(g - g_ref) <= tol), np.max(np.abs(g - g_ref) / tol)
    prob.close()


def test_backward_of_a_weighted_sum_scales_each_particle():
    wl, obs, x, lp_ref, g_ref = _setup()
    prob = api.Problem.from_workload(wl, obs)
    X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(3).normal(size=wl.N).astype(np.float32)).cuda()
    (w * api.loglik(X, prob)).sum().backward()
    g = X.grad.cpu().numpy().T.astype(np.float64)
    wn = w.cpu().numpy().astype(np.float64)[:, None]
    ref = wn * g_ref
    tol = np.abs(wn) * grad_tolerance(g_ref, wl.M) + 1e-7 * np.abs(ref)
    assert np.all(np.abs(g - ref) <= tol), np.max(np.abs(g - ref) / tol)
    # composes with other torch ops and with torch.autograd.grad
    X2 = X.detach().clone().requires_grad_(True)
    (gx,) = torch.autograd.grad(api.loglik(X2, prob).mean(), X2)
    np.testing.assert_allclose(gx.cpu().numpy().T, g_ref / wl.N,
                               atol=float(np.max(grad_tolerance(g_ref, wl.M))) / wl.N, rtol=0)
    prob.close()
