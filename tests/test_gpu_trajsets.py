"""GPU parity of the likelihood of a set of trajectories (Sec. IV-C: Eq.
traj_likelihood_sum, the equally weighted mixture, and Eq.
traj_likelihood_prod) against the FP64 oracle, through the C ABI: log p and
the gradient of theta and of every trajectory's shooting states, for 2-4
trajectories of double pendulums and chains, both combinations, several
checkpoint strides; one trajectory reproduces the plain problem; the SVGD
iteration runs on the set.
"""
import numpy as np
import pytest
import torch

from helpers import assert_grad_close, assert_logp_close, f32_workload, physical
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _set(wl, R, seed):
    """R trajectories from R parameter draws and start states (float32 data)."""
    rng = np.random.default_rng(seed)
    obs, s0s = [], []
    for r in range(R):
        th = wl.theta_true if r == 0 else rng.uniform(wl.lo, wl.hi)
        s0 = wl.s0 if r == 0 else np.concatenate([rng.uniform(-1.2, 1.2, wl.n), np.zeros(wl.n)])
        s0 = s0.astype(np.float32).astype(np.float64)
        m, l, b = physical(wl, th)
        roll = orc.simulate(m, l, b, s0, wl.dt, wl.T, g=wl.g)
        o = roll[1:, wl.obs_index] + wl.sigma_obs * rng.normal(size=(wl.T, len(wl.obs_index)))
        obs.append(o.astype(np.float32))
        s0s.append(s0)
    return np.stack(obs), np.stack(s0s)


def _particles(wl, obs, seed, N):
    R = obs.shape[0]
    parts = [wlmod.initial_particles(wl, obs[r].astype(np.float64), rng_seed=seed + r)[:N] for r in range(R)]
    x = np.concatenate([parts[0][:, :wl.M]] + [p[:, wl.M:] for p in parts], axis=1)
    return np.ascontiguousarray(x.astype(np.float32).astype(np.float64))


def _oracle(wl, obs, s0s, combine):
    return orc.Problem(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                       theta_link=wl.theta_link, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64),
                       obs_index=wl.obs_index, sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=s0s, lo=wl.lo,
                       hi=wl.hi, g=wl.g, c_lim=wl.c_lim, combine=combine)


def _check(wl, R, combine, seed, N=64, K=None, fast=None):
    obs, s0s = _set(wl, R, seed)
    prob = api.Problem.from_workload(wl, obs[0], checkpoint_stride=K, fast_math=fast)
    prob.set_trajectories(obs, s0s, combine)
    x = _particles(wl, obs, seed, N)
    assert prob.P == x.shape[1]
    logp, g, status = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    lp_ref, g_ref = _oracle(wl, obs, s0s, combine).loglik_grad(x, threads=8)
    assert_logp_close(logp.cpu().numpy().astype(np.float64), lp_ref)
    assert_grad_close(g.cpu().numpy().T.astype(np.float64), g_ref, wl.M)
    prob.close()


@pytest.mark.parametrize("combine", ["sum", "product"])
@pytest.mark.parametrize("R", [2, 4])
def test_double_pendulum_sets(R, combine):
    wl = f32_workload(wlmod.double_pendulum(N=64))
    _check(wl, R, combine, seed=100 + R)


@pytest.mark.parametrize("combine", ["sum", "product"])
@pytest.mark.parametrize("K", [1, 7])
def test_chain_sets(K, combine):
    wl = f32_workload(wlmod.chain5(N=32, T=120, W=4))
    _check(wl, 3, combine, seed=200 + K, N=32, K=K, fast=1)


def test_one_trajectory_set_is_the_plain_problem():
    wl = f32_workload(wlmod.double_pendulum(N=64))
    obs, s0s = _set(wl, 1, 300)
    x = _particles(wl, obs, 300, 64)
    out = []
    for combine in ("sum", "product"):
        prob = api.Problem.from_workload(wl, obs[0])
        prob.set_trajectories(obs, s0s, combine)
        lp, g, _ = prob.loglik_grad(_gpu(x))
        torch.cuda.synchronize()
        out.append((lp.cpu().numpy(), g.cpu().numpy()))
        prob.close()
    # the plain problem (its own observations and start state are trajectory 0's)
    plain = api.Problem.from_workload(wl, obs[0])
    lp, g, _ = plain.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    out.append((lp.cpu().numpy(), g.cpu().numpy()))
    plain.close()
    for lp, g in out[1:]:
        np.testing.assert_array_equal(lp, out[0][0])
        np.testing.assert_array_equal(g, out[0][1])


def test_svgd_iterates_on_a_set_and_batches_refuse_it():
    wl = f32_workload(wlmod.double_pendulum(N=64))
    obs, s0s = _set(wl, 2, 400)
    prob = api.Problem.from_workload(wl, obs[0])
    prob.set_trajectories(obs, s0s, "sum")
    x = _particles(wl, obs, 400, 64)
    X = _gpu(x)
    sv = api.Svgd(64, wl.M, prob.P, wl.lo, wl.hi, lr=1e-2)
    lp = torch.empty(64, device="cuda")
    api.iterate(prob, sv, X, 5, lp)
    torch.cuda.synchronize()
    assert torch.isfinite(X).all() and torch.isfinite(lp).all()
    with pytest.raises(api.PdsError):
        api.Batch([prob], [sv], [X])
    with pytest.raises(api.PdsError):
        prob.set_csvgd(True, 1.0)
    sv.close()
    prob.close()


def test_sum_keeps_the_modes_and_product_averages_them():
    """The paper's combination experiment, synthetically: two double-pendulum
    trajectories from two link-length settings.  After 1000 iterations the
    mixture (sum) leaves most particles at one of the two true settings,
    while the product concentrates them at a compromise near neither."""
    N = 200
    wl, thetas, noises = wlmod.two_mode_pendulums(N=N)
    dev = torch.device("cuda")
    obs = []
    for th, nz in zip(thetas, noises):
        m, l, b = physical(wl, th)
        roll = orc.simulate(m, l, b, wl.s0, wl.dt, wl.T, g=wl.g)
        obs.append((roll[1:, wl.obs_index] + wl.sigma_obs * nz).astype(np.float32))
    obs = np.stack(obs)
    s0s = np.stack([wl.s0, wl.s0])
    near = {}
    for combine in ("sum", "product"):
        prob = api.Problem.from_workload(wl, obs[0])
        prob.set_trajectories(obs, s0s, combine)
        parts = [wlmod.initial_particles(wl, obs[r].astype(np.float64), rng_seed=1) for r in range(2)]
        x = np.concatenate([parts[0][:, :2], parts[0][:, 2:], parts[1][:, 2:]], axis=1)
        X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).to(dev)
        sv = api.Svgd(N, 2, prob.P, wl.lo, wl.hi, lr=1e-2)
        api.iterate(prob, sv, X, 1000)
        torch.cuda.synchronize()
        th = X[:2].cpu().numpy().T
        near[combine] = sum(float(np.mean(np.linalg.norm(th - t, axis=1) < 0.05)) for t in thetas)
        if combine == "product":
            assert np.all(th.std(axis=0) < 0.08), th.std(axis=0)
        sv.close()
        prob.close()
    assert near["sum"] >= 0.5, near
    assert near["product"] <= 0.05, near
