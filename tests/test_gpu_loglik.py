"""GPU parity of the rollout + adjoint path (pds_loglik_grad, pds_simulate)
against the FP64 oracle, through the C ABI.

Covers Sec. IV-C's multiple-shooting likelihood (Eqs. 2, 4, 5), Sec. IV-D's
limit prior, and the gradient the adjoint computes (Appendix B-A), on seeded
workloads shaped like the paper's double pendulum and on a 5-link chain at
full size (sampled particles), plus edge cases: one window, one step per
window, uneven windows, ragged particle counts, checkpoint strides 1..h+,
non-finite inputs.
"""
import numpy as np
import pytest
import torch

from helpers import (assert_grad_close, assert_logp_close, f32_workload, observations, oracle_problem, particles,
                     physical)
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _run(wl, obs, x, K=None, grad=True, fast=None):
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=K, fast_math=fast)
    logp, g, status = prob.loglik_grad(_gpu(x), grad=grad)
    torch.cuda.synchronize()
    out = (logp.cpu().numpy().astype(np.float64), None if g is None else g.cpu().numpy().T.astype(np.float64),
           status.cpu().numpy())
    prob.close()
    return out


def _check(wl, obs, x, K=None, threads=8, fast=None):
    lp, g, st = _run(wl, obs, x, K, fast=fast)
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x, threads=threads)
    assert np.all(st == 0)
    e1 = assert_logp_close(lp, lp_ref)
    e2 = assert_grad_close(g, g_ref, wl.M)
    return e1, e2


@pytest.mark.parametrize("fast", [0, 1])
def test_double_pendulum_full_trajectory(fast):
    wl = f32_workload(wlmod.double_pendulum(N=100))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs), fast=fast)


@pytest.mark.parametrize("K", [1, 3, 10, 50, 4096])
def test_checkpoint_strides_agree(K):
    wl = f32_workload(wlmod.chain5(N=64, T=200, W=4))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs), K=K)
    _check(wl, obs, particles(wl, obs), K=K, fast=1)


@pytest.mark.parametrize("fast", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 7, 8])
def test_chain_lengths_all_parameter_kinds(n, fast):
    # at most 16 theta entries: all three kinds up to 5 links, masses and damping beyond
    kinds = (0, 1, 2) if n <= 5 else (0, 2)
    wl = f32_workload(wlmod.random_chain(n, 37, seed=300 + n, T=45, W=4, kinds=kinds))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs), K=7, fast=fast)


def test_angles_only_observations_and_uneven_windows():
    wl = f32_workload(wlmod.random_chain(3, 130, seed=41, T=53, W=7, observe_velocity=False))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs), K=4)


def test_one_window_and_one_step_windows():
    wl = f32_workload(wlmod.random_chain(2, 20, seed=42, T=12, W=1))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs))
    wl = f32_workload(wlmod.random_chain(2, 20, seed=43, T=12, W=12))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs))


def test_single_particle_and_ragged_counts():
    for N in (1, 127, 129):
        wl = f32_workload(wlmod.double_pendulum(N=N))
        wl.T, wl.W, wl.noise = 80, 4, wl.noise[:80]
        obs = observations(wl)
        _check(wl, obs, particles(wl, obs))


@pytest.mark.parametrize("case", ["pendulum", "chain5_every_fast", "angles_only_fast"])
def test_logp_only_matches_logp_with_gradient(case):
    """log p alone runs a kernel of its own (the forward sweep, fewer
    registers); it must give the same bits as the forward sweep of the
    kernel that also computes the gradient."""
    if case == "pendulum":
        wl, K, fast = f32_workload(wlmod.double_pendulum(N=50)), None, None
    elif case == "chain5_every_fast":
        wl, K, fast = f32_workload(wlmod.chain5(N=300, T=200, W=4)), 1, 1
    else:
        wl, K, fast = f32_workload(wlmod.random_chain(4, 131, seed=8, T=60, W=5, observe_velocity=False)), 1, 1
    obs = observations(wl)
    x = particles(wl, obs)
    lp1, _, st1 = _run(wl, obs, x, K=K, grad=False, fast=fast)
    lp2, _, st2 = _run(wl, obs, x, K=K, grad=True, fast=fast)
    np.testing.assert_array_equal(lp1, lp2)
    np.testing.assert_array_equal(st1, st2)
    assert_logp_close(lp1, oracle_problem(wl, obs).loglik_grad(x, grad=False, threads=8))


def test_gradient_matches_fp64_central_differences():
    """The FP32 adjoint against central differences (h = 1e-4) of the
    oracle's FP64 log p, checkpoint strides 10 and 50."""
    wl = f32_workload(wlmod.chain5(N=3, T=100, W=2))
    obs = observations(wl)
    x = particles(wl, obs)
    op = oracle_problem(wl, obs)
    for K in (10, 50):
        _, g, _ = _run(wl, obs, x, K=K)
        for i in range(x.shape[0]):
            fd = np.zeros(wl.P)
            for k in range(wl.P):
                xp, xm = x[i].copy(), x[i].copy()
                xp[k] += 1e-4
                xm[k] -= 1e-4
                fd[k] = (op.loglik_grad(xp[None], grad=False)[0] - op.loglik_grad(xm[None], grad=False)[0]) / 2e-4
            assert_grad_close(g[i:i + 1], fd[None], wl.M, rtol=2e-3)


@pytest.mark.parametrize("fast", [0, 1])
def test_full_size_chain5_sampled_particles(fast):
    """N = 16384, T = 1000, W = 20, K = 1 (the benchmark configuration):
    all particles computed on the GPU, 16 sampled particles checked."""
    wl = f32_workload(wlmod.chain5(N=16384))
    obs = observations(wl)
    x = particles(wl, obs)
    lp, g, st = _run(wl, obs, x, K=1, fast=fast)
    assert np.all(st == 0)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(wl.N, 16, replace=False))
    idx[0], idx[-1] = 0, wl.N - 1
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x[idx], threads=16)
    assert_logp_close(lp[idx], lp_ref)
    assert_grad_close(g[idx], g_ref, wl.M)


def test_maximum_particle_count_and_window_length():
    """The largest call the API accepts: N = 2^20 particles (2-link chain,
    T = 24, W = 3; 64 sampled particles, the first and last included), and a
    window of PDS_MAX_WINDOW_STEPS = 4096 steps (W = 1, 8 particles of a
    damped single pendulum, whose FP32 and FP64 rollouts stay close over
    4096 steps, unlike a chaotic double pendulum)."""
    N = 1 << 20
    wl = f32_workload(wlmod.random_chain(2, N, seed=77, T=24, W=3))
    obs = observations(wl)
    x = particles(wl, obs)
    lp, g, st = _run(wl, obs, x, K=5)
    assert np.all(st == 0)
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(N, 64, replace=False))
    idx[0], idx[-1] = 0, N - 1
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x[idx], threads=16)
    assert_logp_close(lp[idx], lp_ref)
    assert_grad_close(g[idx], g_ref, wl.M)
    wl = f32_workload(wlmod.random_chain(1, 8, seed=78, T=4096, W=1, dt=0.001))
    obs = observations(wl)
    _check(wl, obs, particles(wl, obs), K=64)
    bad = f32_workload(wlmod.random_chain(1, 8, seed=78, T=4097, W=1, dt=0.001))
    with pytest.raises(api.PdsError):
        api.Problem.from_workload(bad, np.zeros((bad.T, bad.D), np.float32))


def test_deterministic_bitwise():
    wl = f32_workload(wlmod.chain5(N=300, T=100, W=5))
    obs = observations(wl)
    x = particles(wl, obs)
    a = _run(wl, obs, x)
    b = _run(wl, obs, x)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_nonfinite_particle_flagged_and_isolated():
    wl = f32_workload(wlmod.double_pendulum(N=40))
    obs = observations(wl)
    x = particles(wl, obs)
    x_bad = x.copy()
    x_bad[3, 0] = np.nan
    lp, g, st = _run(wl, obs, x)
    lp2, g2, st2 = _run(wl, obs, x_bad)
    assert st2[3] == 1 and np.sum(st2) == 1
    keep = np.arange(wl.N) != 3
    np.testing.assert_array_equal(lp[keep], lp2[keep])
    np.testing.assert_array_equal(g[keep], g2[keep])


def test_simulate_matches_oracle_rollout():
    wl = f32_workload(wlmod.chain5(N=8, T=400, W=4))
    theta = wl.theta_init.astype(np.float32).astype(np.float64)
    obs = observations(wl)
    prob = api.Problem.from_workload(wl, obs)
    states = prob.simulate(_gpu(theta)).cpu().numpy()  # [T+1][S][N]
    for i in range(theta.shape[0]):
        m, l, b = physical(wl, theta[i])
        ref = orc.simulate(m, l, b, wl.s0, wl.dt, wl.T, g=wl.g)
        # FP32 vs FP64 rollout of a chaotic chain: the first 100 steps (0.5 s)
        # agree to 1e-4 of the state's scale.
        err = np.max(np.abs(states[:, :, i] - ref), axis=1)
        scale = np.max(np.abs(ref), axis=1) + 1.0
        assert np.all(err[:100] <= 1e-4 * scale[:100]), err[:100].max()


def test_invalid_arguments_are_rejected():
    wl = f32_workload(wlmod.double_pendulum(N=4))
    obs = observations(wl)
    with pytest.raises(api.PdsError):
        api.Problem.from_workload(wl, obs[:, :1].repeat(5, axis=1))  # D > 2n
    prob = api.Problem.from_workload(wl, obs)
    with pytest.raises(api.PdsError):
        prob.set_checkpoint_stride(0)
    bad = wlmod.double_pendulum(N=4)
    bad.theta_link = np.array([0, 0, 0, 7], dtype=np.int32)
    with pytest.raises(api.PdsError):
        api.Problem.from_workload(bad, obs)
