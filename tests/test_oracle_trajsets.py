"""Pins of the oracle's likelihood for a set of trajectories (Sec. IV-C:
Eq. traj_likelihood_sum, the equally weighted Gaussian mixture, and Eq.
traj_likelihood_prod, the product) on the CPU.

Each trajectory r has its own start state and shooting states; the
parameter-limit prior is counted once.  What fixes the oracle:
  * with one window (single shooting) both combinations follow from scipy's
    Gaussian densities of independent rollouts (logsumexp - log R for the sum);
  * R copies of one trajectory give the single-trajectory likelihood
    (sum) or R times its data term (product), with the same theta gradient
    (sum) or R times it (product);
  * one trajectory in a set is the plain problem;
  * the gradient matches central differences in both modes.
"""
import numpy as np
import pytest
from scipy import special, stats

from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import workloads as wlmod

from test_oracle_likelihood import _physical


def _set(wl, thetas, s0s, W, combine, T=None):
    T = T or wl.T
    rng = np.random.default_rng(77)
    obs = []
    for th, s0 in zip(thetas, s0s):
        m, l, b = _physical(wl, th)
        roll = orc.simulate(m, l, b, s0, wl.dt, T, g=wl.g)
        obs.append(roll[1:, wl.obs_index] + wl.sigma_obs * rng.normal(size=(T, len(wl.obs_index))))
    obs = np.stack(obs)
    prob = orc.Problem(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                       theta_link=wl.theta_link, dt=wl.dt, T=T, W=W, obs=obs, obs_index=wl.obs_index,
                       sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=np.stack(s0s), lo=wl.lo, hi=wl.hi,
                       g=wl.g, c_lim=wl.c_lim, combine=combine)
    return prob, obs


def _two_trajectories(seed=4):
    wl = wlmod.double_pendulum(N=4)
    rng = np.random.default_rng(seed)
    thetas = [wl.theta_true, rng.uniform(wl.lo, wl.hi)]
    s0s = [wl.s0, np.array([0.8, -0.4, 0.0, 0.0])]
    return wl, thetas, s0s


@pytest.mark.parametrize("combine", ["sum", "product"])
def test_single_shooting_against_scipy(combine):
    wl, thetas, s0s = _two_trajectories()
    prob, obs = _set(wl, thetas, s0s, W=1, combine=combine, T=60)
    for theta in wl.theta_init[:3]:
        m, l, b = _physical(wl, theta)
        terms = []
        for r in range(2):
            pred = orc.simulate(m, l, b, s0s[r], wl.dt, 60, g=wl.g)[1:, wl.obs_index]
            terms.append(stats.norm.logpdf(obs[r], loc=pred, scale=wl.sigma_obs).sum())
        prior = stats.uniform.logpdf(theta, loc=wl.lo, scale=wl.hi - wl.lo).sum()
        ref = (special.logsumexp(terms) - np.log(2) if combine == "sum" else sum(terms)) + prior
        got = prob.loglik_grad(theta[None, :], grad=False)[0]
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)


def test_copies_of_one_trajectory():
    wl = wlmod.double_pendulum(N=4)
    R = 3
    single, obs = _set(wl, [wl.theta_true], [wl.s0], W=5, combine="sum", T=50)
    kw = dict(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
              theta_link=wl.theta_link, dt=wl.dt, T=50, W=5, obs=np.repeat(obs, R, axis=0), obs_index=wl.obs_index,
              sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=np.stack([wl.s0] * R), lo=wl.lo, hi=wl.hi,
              g=wl.g, c_lim=wl.c_lim)
    psum = orc.Problem(combine="sum", **kw)
    pprod = orc.Problem(combine="product", **kw)
    rng = np.random.default_rng(1)
    x1 = np.concatenate([wl.theta_init[0], rng.normal(scale=0.3, size=single.P - single.M)])
    xR = np.concatenate([x1[:single.M]] + [x1[single.M:]] * R)
    lp1, g1 = single.loglik_grad(x1[None, :])
    lps, gs = psum.loglik_grad(xR[None, :])
    lpp, gp = pprod.loglik_grad(xR[None, :])
    prior = -np.log(wl.hi - wl.lo).sum()  # theta inside the box
    assert abs(lps[0] - lp1[0]) <= 1e-9 * abs(lp1[0])
    assert abs(lpp[0] - (R * (lp1[0] - prior) + prior)) <= 1e-9 * abs(lpp[0])
    M, Ps = single.M, single.P - single.M
    np.testing.assert_allclose(gs[0, :M], g1[0, :M], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gp[0, :M], R * g1[0, :M], rtol=1e-9, atol=1e-9)
    for r in range(R):
        np.testing.assert_allclose(gs[0, M + r * Ps:M + (r + 1) * Ps], g1[0, M:] / R, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(gp[0, M + r * Ps:M + (r + 1) * Ps], g1[0, M:], rtol=1e-9, atol=1e-9)


def test_one_trajectory_set_is_the_plain_problem():
    wl = wlmod.random_chain(3, 4, seed=9)
    m, l, b = _physical(wl, wl.theta_true)
    obs = wlmod.observations(wl, orc.simulate(m, l, b, wl.s0, wl.dt, wl.T, g=wl.g))
    kw = dict(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind, theta_link=wl.theta_link,
              dt=wl.dt, T=wl.T, W=wl.W, obs_index=wl.obs_index, sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def,
              lo=wl.lo, hi=wl.hi, g=wl.g, c_lim=wl.c_lim)
    plain = orc.Problem(obs=obs, s0=wl.s0, **kw)
    x = wlmod.initial_particles(wl, obs, rng_seed=3)
    lp, g = plain.loglik_grad(x)
    for combine in ("sum", "product"):
        one = orc.Problem(obs=obs[None], s0=wl.s0[None], combine=combine, **kw)
        lp1, g1 = one.loglik_grad(x)
        np.testing.assert_allclose(lp1, lp, rtol=1e-12)
        np.testing.assert_allclose(g1, g, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("combine", ["sum", "product"])
def test_gradient_matches_central_differences(combine):
    wl, thetas, s0s = _two_trajectories(seed=6)
    prob, _ = _set(wl, thetas, s0s, W=3, combine=combine, T=30)
    rng = np.random.default_rng(2)
    x = np.concatenate([wl.theta_init[1], rng.normal(scale=0.3, size=prob.P - prob.M)])
    _, g = prob.loglik_grad(x[None, :])
    fd = np.zeros(prob.P)
    for k in range(prob.P):
        h = 1e-6 * max(1.0, abs(x[k]))
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd[k] = (prob.loglik_grad(xp[None, :], grad=False)[0] - prob.loglik_grad(xm[None, :], grad=False)[0]) / (2 * h)
    assert np.max(np.abs(g[0] - fd)) <= 1e-5 * max(1.0, np.max(np.abs(fd)))
