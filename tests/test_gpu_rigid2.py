"""GPU parity of the rigid double pendulum (the 11-parameter physical double
pendulum of Sec. V, App. Table params-ibm-pendulum) against the FP64 oracle,
through the C ABI.

Covers: f_sim; log p and its gradient (hand-written reverse sweep against
the oracle's dual numbers) for all 11 parameters and for an unordered subset,
with particles partly outside the box, several checkpoint strides, exact and
fast math, ragged N; an SVGD iteration on the problem; batched execution and
the server with rigid pendulum jobs beside chains (equal to each job run
alone); the configurations the system does not support.
"""
import numpy as np
import pytest
import torch

from helpers import assert_grad_close, f32_workload, observations, particles
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api, serve
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _workload(N, T=200, W=5, theta_param=tuple(range(11)), seed=7000):
    wl = wlmod.rigid_double_pendulum(N=N, seed=seed, T=T, W=W, theta_param=theta_param)
    wl.p11, wl.lo, wl.hi, wl.s0 = _f32(wl.p11), _f32(wl.lo), _f32(wl.hi), _f32(wl.s0)
    wl.theta_true = wl.p11[wl.theta_param]
    wl.dt = float(np.float32(wl.dt))
    wl.g = float(np.float32(wl.g))
    st = orc.rigid2_simulate(wl.p11, wl.g, wl.dt, wl.T, wl.s0)
    obs = wlmod.observations(wl, st).astype(np.float32)
    return wl, obs


def _oracle(wl, obs):
    return orc.Rigid2Problem(p11=wl.p11, g=wl.g, theta_param=wl.theta_param, dt=wl.dt, T=wl.T, W=wl.W,
                             obs=obs.astype(np.float64), obs_index=wl.obs_index, sigma_obs=wl.sigma_obs,
                             sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo, hi=wl.hi, c_lim=wl.c_lim)


def _particles(wl, obs, seed=3):
    x = wlmod.initial_particles(wl, obs.astype(np.float64), rng_seed=seed)
    width = wl.hi - wl.lo
    x[0, 0] = wl.hi[0] + 0.05 * width[0]
    x[1 % len(x), wl.M - 1] = wl.lo[wl.M - 1] - 0.02 * width[wl.M - 1]
    return _f32(x)


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def test_simulate_matches_oracle():
    wl, obs = _workload(N=5, T=400)
    th = _f32(wl.theta_init)
    prob = api.Problem.from_workload(wl, obs)
    states = prob.simulate(_gpu(th))
    torch.cuda.synchronize()
    got = states.cpu().numpy()  # [T+1][4][N]
    for i in range(len(th)):
        p = wl.p11.copy()
        p[wl.theta_param] = th[i]
        ref = orc.rigid2_simulate(p, wl.g, wl.dt, wl.T, wl.s0)
        np.testing.assert_allclose(got[:, :, i], ref, rtol=0, atol=2e-4 * (1 + np.abs(ref).max()))
    prob.close()


@pytest.mark.parametrize("theta_param", [tuple(range(11)), (5, 0, 6, 9)])
@pytest.mark.parametrize("K,fast", [(5, 0), (1, 0), (10, 1), (7, 1)])
def test_loglik_grad_matches_oracle(theta_param, K, fast):
    wl, obs = _workload(N=300, theta_param=theta_param)
    x = _particles(wl, obs)
    lp_ref, g_ref = _oracle(wl, obs).loglik_grad(x, threads=8)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=K, fast_math=fast)
    assert prob.P == x.shape[1] and prob.M == len(theta_param)
    logp, g, status = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    # log p sums terms of both signs: Gaussian constants (+12 per observed
    # step here) and residuals; fp32 rounding scales with their magnitude, so
    # the tolerance is relative to max(|log p|, the constants' total)
    const = wl.T * 0.5 * wl.D * abs(np.log(2 * np.pi * wl.sigma_obs ** 2))
    lp = logp.cpu().numpy().astype(np.float64)
    err = np.abs(lp - lp_ref) / np.maximum(np.abs(lp_ref), const)
    assert np.all(err <= 1e-4), f"max logp err {err.max():.3e} at particle {int(err.argmax())}"
    assert_grad_close(g.cpu().numpy().T.astype(np.float64), g_ref, wl.M)
    assert int(status.sum()) == 0
    prob.close()


def test_svgd_iterations_on_the_rigid_pendulum():
    wl, obs = _workload(N=256, T=200, W=5)
    x = _particles(wl, obs)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=5)
    sv = api.Svgd(x.shape[0], wl.M, prob.P, wl.lo, wl.hi, lr=1e-3)
    X = _gpu(x)
    lp0, _, _ = prob.loglik_grad(X)
    api.iterate(prob, sv, X, 20)
    lp1, _, _ = prob.loglik_grad(X)
    torch.cuda.synchronize()
    a, b = lp0.cpu().numpy(), lp1.cpu().numpy()
    assert np.all(np.isfinite(b))
    assert np.median(b) > np.median(a)
    sv.close()
    prob.close()


def test_unsupported_configurations_are_rejected():
    wl, obs = _workload(N=16, T=40, W=2)
    prob = api.Problem.from_workload(wl, obs)
    with pytest.raises(api.PdsError):
        prob.set_csvgd(True, 1.0)
    with pytest.raises(api.PdsError):
        prob.set_trajectories(np.stack([obs, obs]), np.stack([wl.s0, wl.s0]).astype(np.float32))
    prob.close()
    bad = wlmod.rigid_double_pendulum(N=4, T=40, W=2, theta_param=(1, 1))
    with pytest.raises(api.PdsError):
        api.Problem.from_workload(bad, obs)


def _mixed_jobs():
    """Two rigid pendulum problems (all 11 and 4 parameters) beside two chains."""
    out = []
    for tp, N, seed in ((tuple(range(11)), 300, 7000), ((5, 0, 6, 9), 200, 7001)):
        wl, obs = _workload(N=N, T=120, W=4, theta_param=tp, seed=seed)
        wl.lr = 1e-3
        out.append((wl, obs, _particles(wl, obs)))
    for wl in wlmod.batched_problems(n_jobs=2, seed=91, T_range=(40, 90), W_range=(2, 5), N_range=(100, 300)):
        wl = f32_workload(wl)
        o = observations(wl)
        out.append((wl, o, particles(wl, o, seed=3)))
    return out


def test_batch_with_rigid_pendulums_equals_alone():
    jobs = _mixed_jobs()
    iters = 3
    alone = []
    for wl, obs, x in jobs:
        prob = api.Problem.from_workload(wl, obs, checkpoint_stride=5, fast_math=0)
        sv = api.Svgd(x.shape[0], wl.M, prob.P, wl.lo, wl.hi, lr=wl.lr)
        X = _gpu(x)
        api.iterate(prob, sv, X, iters)
        torch.cuda.synchronize()
        alone.append(X.cpu().numpy())
        sv.close()
        prob.close()
    probs = [api.Problem.from_workload(wl, obs, checkpoint_stride=5, fast_math=0) for wl, obs, _ in jobs]
    svgds = [api.Svgd(x.shape[0], wl.M, p.P, wl.lo, wl.hi, lr=wl.lr) for (wl, _, x), p in zip(jobs, probs)]
    Xs = [_gpu(x) for _, _, x in jobs]
    b = api.Batch(probs, svgds, Xs)
    b.iterate(iters)
    torch.cuda.synchronize()
    for j, (wl, _, _) in enumerate(jobs):
        width = np.concatenate([wl.hi - wl.lo, np.ones(wl.P - wl.M)])[:, None]
        dx = np.max(np.abs(Xs[j].cpu().numpy() - alone[j]) / width)
        assert dx <= 1e-5, (j, dx)
    b.close()


def test_server_runs_rigid_pendulum_jobs():
    jobs = [(wl, obs, x, 4) for wl, obs, x in _mixed_jobs()]
    lat, res, _ = serve.run_server(jobs, np.array([0.0, 0.0, 0.01, 0.02]), mem_budget=8 << 30, fast_math=False)
    _, ref, _ = serve.run_plain(jobs, np.zeros(len(jobs)), fast_math=False)
    for k, (wl, _, _, _) in enumerate(jobs):
        width = np.concatenate([wl.hi - wl.lo, np.ones(wl.P - wl.M)])
        assert np.max(np.abs(res[k][0] - ref[k][0]) / width) <= 1e-5, k
    assert np.all(lat >= 0)
