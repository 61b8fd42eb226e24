"""GPU parity of the arm-shaking-a-box system (pds_problem_create_armbox)
against the FP64 oracle: log p, gradient (forward tangents through each
window), f_sim, the weight-swap symmetry of the posterior, the full-size
problem (N = 2048, T = 2000, W = 40) on sampled particles, and batching
together with chain problems."""
import numpy as np
import pytest
import torch

from helpers import assert_grad_close, assert_logp_close, f32_workload
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _f32(wl):
    for name in ("arm_len", "amp", "freq", "phase", "lo", "hi", "s0", "theta_true", "theta_init"):
        setattr(wl, name, getattr(wl, name).astype(np.float32).astype(np.float64))
    wl.dt = float(np.float32(wl.dt))
    return wl


def _setup(N=64, T=300, W=6, seed=3000):
    wl = _f32(wlmod.arm_box(N=N, seed=seed, T=T, W=W))
    ab = orc.ArmBox.from_workload(wl)
    st = ab.simulate(wl.theta_true, wl.dt, wl.T, wl.s0)
    obs = (st[1:, wl.obs_index] + wl.sigma_obs * wl.noise[:wl.T]).astype(np.float32)
    op = orc.ArmBoxProblem(ab, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64), obs_index=wl.obs_index,
                           sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo, hi=wl.hi,
                           c_lim=wl.c_lim)
    rng = np.random.default_rng(seed + 1)
    shoot = st[[wl.window_start(w) for w in range(1, wl.W)]].ravel()
    x = np.concatenate([wl.theta_init, np.tile(shoot, (wl.N, 1)) + 0.02 * rng.normal(size=(wl.N, wl.P - 4))], 1)
    return wl, obs, op, x.astype(np.float32).astype(np.float64), st


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


@pytest.mark.parametrize("fast", [0, 1])
def test_armbox_logp_and_gradient_match_oracle(fast):
    wl, obs, op, x, _ = _setup()
    prob = api.Problem.armbox(wl, obs, fast_math=fast)
    lp, g, st = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    lp_ref, g_ref = op.loglik_grad(x, threads=8)
    assert np.all(st.cpu().numpy() == 0)
    assert_logp_close(lp.cpu().numpy().astype(np.float64), lp_ref)
    assert_grad_close(g.cpu().numpy().T.astype(np.float64), g_ref, 4)


def test_armbox_simulate_matches_oracle():
    wl, obs, op, x, st_ref = _setup(N=4, T=400, W=4)
    prob = api.Problem.armbox(wl, obs)
    states = prob.simulate(_gpu(wl.theta_true[None, :]))[:, :, 0].cpu().numpy()
    err = np.max(np.abs(states - st_ref), axis=1)
    assert np.all(err[:200] <= 1e-4 * (np.max(np.abs(st_ref[:200]), axis=1) + 1.0)), err[:200].max()


def test_armbox_weight_swap_symmetry_on_gpu():
    wl, obs, op, x, _ = _setup(N=50)
    xs = x.copy()
    xs[:, :4] = x[:, [2, 3, 0, 1]]
    prob = api.Problem.armbox(wl, obs)
    a, ga, _ = prob.loglik_grad(_gpu(x))
    b, gb, _ = prob.loglik_grad(_gpu(xs))
    torch.cuda.synchronize()
    a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(a - b) <= 1e-5 * np.abs(a))
    ga, gb = ga.cpu().numpy().T, gb.cpu().numpy().T
    np.testing.assert_allclose(gb[:, [2, 3, 0, 1]], ga[:, :4], rtol=1e-3, atol=1e-3 * np.abs(ga[:, :4]).max())


def test_armbox_full_size_sampled_particles():
    wl, obs, op, x, _ = _setup(N=2048, T=2000, W=40)
    prob = api.Problem.armbox(wl, obs, fast_math=1)
    lp, g, st = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    idx = np.array([0, 17, 511, 1024, 1999, 2047])
    lp_ref, g_ref = op.loglik_grad(x[idx], threads=8)
    assert_logp_close(lp.cpu().numpy()[idx].astype(np.float64), lp_ref)
    assert_grad_close(g.cpu().numpy().T[idx].astype(np.float64), g_ref, 4)


def test_armbox_in_a_batch_equals_alone():
    wl, obs, op, x, _ = _setup(N=300, T=200, W=5)
    chains = [f32_workload(w) for w in wlmod.batched_problems(n_jobs=2, seed=8, T_range=(40, 80), W_range=(2, 4),
                                                              N_range=(50, 100))]
    from helpers import observations, particles
    c_obs = [observations(w) for w in chains]
    c_x = [particles(w, o) for w, o in zip(chains, c_obs)]
    # alone
    p = api.Problem.armbox(wl, obs, checkpoint_stride=5, fast_math=1)
    s = api.Svgd(wl.N, 4, wl.P, wl.lo, wl.hi, lr=wl.lr)
    X = _gpu(x)
    api.iterate(p, s, X, 2)
    torch.cuda.synchronize()
    alone = X.cpu().numpy()
    # in a batch with two chain problems
    probs = [api.Problem.armbox(wl, obs, checkpoint_stride=5, fast_math=1)] + \
            [api.Problem.from_workload(w, o, checkpoint_stride=5, fast_math=1) for w, o in zip(chains, c_obs)]
    svgds = [api.Svgd(wl.N, 4, wl.P, wl.lo, wl.hi, lr=wl.lr)] + \
            [api.Svgd(w.N, w.M, w.P, w.lo, w.hi, lr=w.lr) for w in chains]
    Xs = [_gpu(x)] + [_gpu(cx) for cx in c_x]
    b = api.Batch(probs, svgds, Xs)
    b.iterate(2)
    torch.cuda.synchronize()
    width = np.concatenate([wl.hi - wl.lo, np.ones(wl.P - 4)])[:, None]
    assert np.max(np.abs(Xs[0].cpu().numpy() - alone) / width) <= 1e-5
    b.close()
