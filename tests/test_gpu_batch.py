"""Batched execution (pds_batch_*): several problems of uneven chain length,
trajectory length, window count and particle count iterated together from a
captured CUDA graph.

Each problem's result in the batch must equal the same problem run alone with
the same settings (the kernels and reductions are deterministic; the batched
rollout is a different kernel, so the comparison allows FP32 rounding), and
one batched iteration must match the FP64 oracle's log p and SVGD step within
the tolerances of the single-problem tests.
"""
import numpy as np
import pytest
import torch

from helpers import LOGP_RTOL, f32_workload, grad_tolerance, observations, oracle_problem, particles, phi_tolerance
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _mix(n_jobs, seed, **kw):
    wls = [f32_workload(w) for w in wlmod.batched_problems(n_jobs=n_jobs, seed=seed, **kw)]
    obs = [observations(w) for w in wls]
    xs = [particles(w, o, seed=3) for w, o in zip(wls, obs)]
    return wls, obs, xs


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _objects(wls, obs, K, fast):
    probs = [api.Problem.from_workload(w, o, checkpoint_stride=K, fast_math=fast) for w, o in zip(wls, obs)]
    svgds = [api.Svgd(w.N, w.M, w.P, w.lo, w.hi, lr=w.lr) for w in wls]
    return probs, svgds


@pytest.mark.parametrize("fast", [0, 1])
def test_batch_equals_each_problem_alone(fast):
    wls, obs, xs = _mix(7, seed=77, T_range=(30, 160), W_range=(2, 9), N_range=(40, 900))
    iters = 3
    # alone
    alone_x, alone_lp = [], []
    probs, svgds = _objects(wls, obs, K=5, fast=fast)
    for w, p, s, x in zip(wls, probs, svgds, xs):
        X = _gpu(x)
        lp = torch.empty(w.N, device="cuda")
        api.iterate(p, s, X, iters, lp)
        torch.cuda.synchronize()
        alone_x.append(X.cpu().numpy())
        alone_lp.append(lp.cpu().numpy())
    # batched
    probs, svgds = _objects(wls, obs, K=5, fast=fast)
    Xs = [_gpu(x) for x in xs]
    lps = [torch.empty(w.N, device="cuda") for w in wls]
    b = api.Batch(probs, svgds, Xs, lps)
    b.iterate(iters)
    torch.cuda.synchronize()
    ng, lpi = b.info()
    assert ng == len({w.n for w in wls})
    for j, w in enumerate(wls):
        width = np.concatenate([w.hi - w.lo, np.ones(w.P - w.M)])[:, None]
        dx = np.max(np.abs(Xs[j].cpu().numpy() - alone_x[j]) / width)
        assert dx <= 1e-5, (j, dx)
        rel = np.max(np.abs(lps[j].cpu().numpy() - alone_lp[j]) / np.abs(alone_lp[j]))
        assert rel <= 1e-6, (j, rel)
    b.close()


def test_batch_with_more_problems_than_branches():
    """70 small problems: the per-problem step branches (at most 64) wrap
    around, and the chain-length groups' rollouts run on branches of their
    own; each problem still equals itself run alone."""
    wls, obs, xs = _mix(70, seed=707, T_range=(20, 40), W_range=(2, 4), N_range=(32, 96))
    iters = 2
    alone_x = []
    probs, svgds = _objects(wls, obs, K=1, fast=1)
    for w, p, s, x in zip(wls, probs, svgds, xs):
        X = _gpu(x)
        api.iterate(p, s, X, iters)
        torch.cuda.synchronize()
        alone_x.append(X.cpu().numpy())
    probs, svgds = _objects(wls, obs, K=1, fast=1)
    Xs = [_gpu(x) for x in xs]
    b = api.Batch(probs, svgds, Xs)
    b.iterate(iters)
    torch.cuda.synchronize()
    for j, w in enumerate(wls):
        width = np.concatenate([w.hi - w.lo, np.ones(w.P - w.M)])[:, None]
        dx = np.max(np.abs(Xs[j].cpu().numpy() - alone_x[j]) / width)
        assert dx <= 1e-5, (j, dx)
    b.close()


def test_batch_autotuned_iteration_matches_oracle():
    wls, obs, xs = _mix(5, seed=91, T_range=(40, 200), W_range=(2, 10), N_range=(30, 400))
    probs, svgds = _objects(wls, obs, K=10, fast=0)
    Xs = [_gpu(x) for x in xs]
    lps = [torch.empty(w.N, device="cuda") for w in wls]
    b = api.Batch(probs, svgds, Xs, lps)
    choices = b.autotune(allow_fast_math=True)
    assert len(choices) == len({w.n for w in wls})
    for links, K, fast, blocks, upt in choices:
        assert K in (1, 5, 10, 25, 50) and fast in (0, 1) and blocks > 0
        assert upt == 1 or (upt == 2 and K == 1)
    b.iterate(1)
    torch.cuda.synchronize()
    for j, w in enumerate(wls):
        lp_ref, g_ref = oracle_problem(w, obs[j]).loglik_grad(xs[j], threads=8)
        lp = lps[j].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(lp - lp_ref) <= LOGP_RTOL * np.abs(lp_ref)), j
        x_ref = np.ascontiguousarray(xs[j].copy())
        phi_ref, bw_ref = orc.SvgdState(w.N, w.P, w.lo, w.hi, lr=w.lr).step(x_ref, g_ref)
        width = np.concatenate([w.hi - w.lo, np.ones(w.P - w.M)])
        dx = np.abs(Xs[j].cpu().numpy().T - x_ref) / width
        # Adam's first step moves each entry by lr * sign(direction): entries
        # agree to rounding except where the oracle's direction is within
        # the GPU direction's tolerance of zero (phi from the FP32 gradient
        # for theta, the gradient itself for the shooting states)
        u = (xs[j][:, :w.M] - w.lo) / (w.hi - w.lo)
        gtol = grad_tolerance(g_ref, w.M)
        near0 = np.zeros_like(dx, dtype=bool)
        near0[:, :w.M] = np.abs(phi_ref) <= phi_tolerance(u, g_ref[:, :w.M] * (w.hi - w.lo), bw_ref,
                                                          gtol[:, :w.M] * (w.hi - w.lo))
        near0[:, w.M:] = np.abs(g_ref[:, w.M:]) <= gtol[:, w.M:]
        assert np.all(dx[~near0] <= 1e-4), (j, np.max(dx[~near0]))
        assert dx.max() <= 2.5 * w.lr, (j, dx.max())
        assert np.mean(near0) <= 2e-2, (j, np.mean(near0))
    b.close()


def test_batch_rejects_mismatched_svgd():
    wls, obs, xs = _mix(2, seed=5, T_range=(30, 60), W_range=(2, 4), N_range=(20, 40))
    probs, svgds = _objects(wls, obs, K=5, fast=0)
    wrong = [svgds[1], svgds[0]] if wls[0].P != wls[1].P else None
    if wrong is None:
        pytest.skip("both problems have the same layout")
    with pytest.raises(api.PdsError):
        api.Batch(probs, wrong, [_gpu(x) for x in xs])


def test_batched_two_units_per_thread_equal_one_unit_alone():
    """Chain-length groups whose problems all allow it (K = 1, every state
    component observed, even N) run the batched launch with two particles
    per thread; each problem's log p equals its one-unit single-problem
    evaluation bit for bit."""
    wls = [f32_workload(wlmod.random_chain(n, N, seed=500 + n + N, T=T, W=W))
           for n, N, T, W in ((2, 64, 40, 4), (2, 130, 33, 3), (4, 96, 50, 5), (5, 200, 41, 4), (3, 58, 30, 3))]
    obs = [observations(w) for w in wls]
    xs = [particles(w, o, seed=3) for w, o in zip(wls, obs)]
    alone = []
    for w, o, x in zip(wls, obs, xs):
        p = api.Problem.from_workload(w, o, checkpoint_stride=1, fast_math=1)
        p.set_option(api.OPT_UNITS_PER_THREAD, 1)
        lp, _, _ = p.loglik_grad(_gpu(x))
        torch.cuda.synchronize()
        alone.append(lp.cpu().numpy())
        p.close()
    probs, svgds = _objects(wls, obs, K=1, fast=1)
    for p in probs:
        p.set_option(api.OPT_UNITS_PER_THREAD, 2)
    Xs = [_gpu(x) for x in xs]
    lps = [torch.empty(w.N, device="cuda") for w in wls]
    b = api.Batch(probs, svgds, Xs, lps)
    b.iterate(1)
    torch.cuda.synchronize()
    for j in range(len(wls)):
        np.testing.assert_array_equal(lps[j].cpu().numpy(), alone[j])
    b.close()
