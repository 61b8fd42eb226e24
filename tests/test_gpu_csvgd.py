"""GPU parity of constrained SVGD (Sec. IV-E, Eq. mdmm-loss, Algorithm 1)
against the FP64 oracle, through the C ABI.

Covers:
  * the observation log-likelihood;
  * the defect and limit constraint values;
  * the observation gradient, the shooting-state gradient and the MDMM
    constraint gradient of theta, which the rollout's second adjoint
    produces (seeded at each window's end);
  * the update: phi plus the constraint direction for theta, Adam for the
    shooting states, lam += lr g for the multipliers;
on seeded chains of 1 to 8 links, with particles partly outside the box,
exact and fast math, and several checkpoint strides.
"""
import numpy as np
import pytest
import torch

from helpers import GRAD_FLOOR, LOGP_RTOL, PHI_TOL, f32_workload, observations, oracle_problem, particles
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _augmented(wl, obs, seed, N, outside=True):
    """Particles [N][Pc]: theta, shooting states (with defects), multipliers."""
    rng = np.random.default_rng(seed)
    x = particles(wl, obs, seed)[:N].copy()
    M, W = wl.M, wl.W
    x[:, M:] += 0.02 * rng.normal(size=(N, x.shape[1] - M))
    if outside:
        # the last parameter (a damping or a length, never a mass that
        # would make the dynamics stiff) leaves the box on both sides
        width = wl.hi - wl.lo
        x[0, M - 1] = wl.hi[M - 1] + 0.05 * width[M - 1]
        x[1 % N, M - 1] = wl.lo[M - 1] - 0.03 * width[M - 1]
    lam = np.concatenate([rng.uniform(-1, 1, (N, W - 1)), rng.uniform(-1, 1, (N, M))], axis=1)
    xa = np.concatenate([x, lam], axis=1)
    return np.ascontiguousarray(xa.astype(np.float32).astype(np.float64))


def _blocks(prob):
    M, S, W, P = prob.M, prob.S, prob.W, prob.P
    Pms = M + (W - 1) * S
    return {"theta": slice(0, M), "shoot": slice(M, Pms), "gdef": slice(Pms, Pms + W - 1),
            "glim": slice(Pms + W - 1, P), "con": slice(P, P + M)}


def _check(wl, obs, x, c, K=None, fast=None, rtol=1e-3):
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=K, fast_math=fast)
    prob.set_csvgd(True, c)
    assert prob.P == x.shape[1]
    logp, g, status = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    lp = logp.cpu().numpy().astype(np.float64)
    g = g.cpu().numpy().T.astype(np.float64)
    assert np.all(status.cpu().numpy() == 0)
    oprob = oracle_problem(wl, obs)
    lp_ref, g_ref = oprob.csvgd_loglik_grad(x, c=c, threads=8)
    # log p_obs adds positive Gaussian constants to negative residual terms;
    # the FP32 error scales with the magnitude of the terms summed
    so2 = wl.sigma_obs ** 2
    const = wl.T * 0.5 * len(wl.obs_index) * abs(np.log(2 * np.pi * so2))
    rel = np.abs(lp - lp_ref) / (np.abs(lp_ref) + const)
    assert rel.max() <= LOGP_RTOL, rel.max()
    worst = {}
    for name, blk in _blocks(prob).items():
        a, r = g[:, blk], g_ref[:, blk]
        if a.shape[1] == 0:
            continue
        if name == "glim":
            err = np.max(np.abs(a - r))
            assert err <= 1e-6, (name, err)
        else:
            # per component, as the unconstrained gradient (helpers)
            tol = rtol * np.abs(r) + GRAD_FLOOR * np.max(np.abs(r), axis=1, keepdims=True)
            ratio = np.abs(a - r) / np.maximum(tol, 1e-300)
            err = ratio.max()
            assert err <= 1.0, (name, err, np.unravel_index(int(ratio.argmax()), ratio.shape))
        worst[name] = float(np.max(err))
    prob.close()
    return worst


@pytest.mark.parametrize("fast", [0, 1])
@pytest.mark.parametrize("c", [0.0, 0.7])
def test_double_pendulum(fast, c):
    wl = f32_workload(wlmod.double_pendulum(N=100))
    obs = observations(wl)
    _check(wl, obs, _augmented(wl, obs, 11, 64), c, fast=fast)


@pytest.mark.parametrize("K", [1, 5, 17])
def test_chain5_checkpoint_strides(K):
    wl = f32_workload(wlmod.chain5(N=64, T=200, W=4))
    obs = observations(wl)
    _check(wl, obs, _augmented(wl, obs, 12, 64), 1.0, K=K, fast=1)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_random_chains(n):
    kinds = (wlmod.PARAM_MASS, wlmod.PARAM_DAMPING) if n > 5 else (wlmod.PARAM_MASS, wlmod.PARAM_LENGTH,
                                                                   wlmod.PARAM_DAMPING)
    wl = f32_workload(wlmod.random_chain(n, 48, seed=20 + n, T=60, W=5, kinds=kinds))
    obs = observations(wl)
    _check(wl, obs, _augmented(wl, obs, 13 + n, 48), 0.5, K=4)


def test_zero_multipliers_and_damping_leave_only_the_observation_gradient():
    wl = f32_workload(wlmod.chain5(N=32, T=100, W=5))
    obs = observations(wl)
    x = _augmented(wl, obs, 14, 32, outside=False)
    x[:, -(wl.W - 1 + wl.M):] = 0.0
    prob = api.Problem.from_workload(wl, obs)
    prob.set_csvgd(True, 0.0)
    _, g, _ = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    g = g.cpu().numpy().T
    assert np.all(g[:, _blocks(prob)["con"]] == 0.0)
    prob.close()


def test_update_matches_oracle():
    wl = f32_workload(wlmod.double_pendulum(N=100))
    obs = observations(wl)
    x = _augmented(wl, obs, 15, 100)
    N = x.shape[0]
    prob = api.Problem.from_workload(wl, obs)
    prob.set_csvgd(True, 1.0)
    X = _gpu(x)
    _, G, _ = prob.loglik_grad(X)
    torch.cuda.synchronize()
    g64 = G.cpu().numpy().T.astype(np.float64)
    sv = api.Svgd(N, wl.M, prob.P, wl.lo, wl.hi, lr=1e-2)
    sv.set_csvgd(wl.W - 1)
    bw, phi = sv.step(X, G, return_phi=True)
    torch.cuda.synchronize()
    xo = x.copy()
    st = orc.CsvgdState(N, prob.P, wl.W - 1, wl.lo, wl.hi, lr=1e-2)
    phi_ref, bw_ref = st.step(xo, g64)
    assert abs(bw.item() - bw_ref) <= 1e-5 * bw_ref
    phi = phi.cpu().numpy().T
    assert np.max(np.abs(phi - phi_ref)) <= PHI_TOL * np.max(np.abs(phi_ref))
    xg = X.cpu().numpy().T.astype(np.float64)
    lam0 = wl.M + (wl.W - 1) * 2 * wl.n
    # multipliers: lam + lr g (float32 arithmetic against float64)
    np.testing.assert_allclose(xg[:, lam0:], xo[:, lam0:], rtol=1e-6, atol=1e-7)
    # theta and shooting states: the first Adam step moves each entry by
    # lr * sign(direction).  Both sides have the same gradient, so the
    # shooting states agree to rounding; a theta entry may take the other
    # sign only where its direction, phi plus the constraint direction, lies
    # within phi's tolerance of zero
    width = np.concatenate([wl.hi - wl.lo, np.ones(lam0 - wl.M)])
    dx = np.abs(xg[:, :lam0] - xo[:, :lam0]) / width
    direction = phi_ref + g64[:, prob.P:prob.P + wl.M] * (wl.hi - wl.lo)
    near0 = np.zeros_like(dx, dtype=bool)
    near0[:, :wl.M] = np.abs(direction) <= PHI_TOL * np.max(np.abs(phi_ref))
    assert np.all(dx[~near0] <= 1e-4), np.max(dx[~near0])
    assert dx.max() <= 2.5e-2
    assert np.mean(near0) <= 2e-2
    # theta is not clipped to the box in the constrained method
    assert np.any(xg[:, wl.M - 1] > wl.hi[wl.M - 1])
    sv.close()
    prob.close()


def test_iterate_requires_both_sides_constrained():
    wl = f32_workload(wlmod.double_pendulum(N=32))
    obs = observations(wl)
    x = _augmented(wl, obs, 16, 32)
    prob = api.Problem.from_workload(wl, obs)
    prob.set_csvgd(True, 1.0)
    sv = api.Svgd(32, wl.M, prob.P, wl.lo, wl.hi)
    X = _gpu(x)
    with pytest.raises(api.PdsError):
        api.iterate(prob, sv, X, 1)
    sv.set_csvgd(wl.W - 1)
    # iterate == loglik + step by hand, bit for bit
    X2 = X.clone()
    api.iterate(prob, sv, X, 2)
    sv2 = api.Svgd(32, wl.M, prob.P, wl.lo, wl.hi)
    sv2.set_csvgd(wl.W - 1)
    for _ in range(2):
        _, G, _ = prob.loglik_grad(X2)
        sv2.step(X2, G)
    torch.cuda.synchronize()
    assert torch.equal(X, X2)
    # switching back restores the multiple-shooting layout
    prob.set_csvgd(False)
    assert prob.P == wl.M + (wl.W - 1) * 2 * wl.n
    sv.close()
    sv2.close()
    prob.close()


def test_constrained_problems_are_not_batched():
    wl = f32_workload(wlmod.double_pendulum(N=32))
    obs = observations(wl)
    prob = api.Problem.from_workload(wl, obs)
    prob.set_csvgd(True, 1.0)
    sv = api.Svgd(32, wl.M, prob.P, wl.lo, wl.hi)
    X = _gpu(_augmented(wl, obs, 17, 32))
    with pytest.raises(api.PdsError):
        api.Batch([prob], [sv], [X])
    sv.close()
    prob.close()
