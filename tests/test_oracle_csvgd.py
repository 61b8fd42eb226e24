"""Pins of the oracle's constrained SVGD (Sec. IV-E, Eq. mdmm-loss,
Algorithm 1) on the CPU.

CSVGD keeps only the observation term in the likelihood and turns the
defect and limit terms into equality constraints with per-particle MDMM
multipliers.  What fixes the oracle:
  * with lambda_def = 1/2 and c = 0 the MDMM gradient of the defect
    constraints g = ||d||^2 / sigma_def^2 is exactly the gradient of the
    Gaussian defect terms log N(d | 0, sigma_def^2) (Eq. 4), so the
    constrained gradient must reproduce the already pinned multiple-shooting
    gradient, and log p_obs must be log p_ms minus the defect and prior terms;
  * the constraint values follow from an independent rollout of each window;
  * -dPsi/dx matches central differences of Psi built from those values;
  * the update moves the multipliers by lr * g and, for one particle, moves
    u by lr * sign of the summed direction on the first Adam step;
  * on a one-dimensional toy, the MDMM iteration settles on the constrained
    optimum and its multiplier (an approximate pin, stated as such).
"""
import numpy as np
import pytest

from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import workloads as wlmod

from test_oracle_likelihood import _obs, _physical, _problem


def _case(seed=3, n=3, W=4, T=40):
    wl = wlmod.random_chain(n, 4, seed=seed, T=T, W=W)
    obs = _obs(wl)
    return wl, obs, _problem(wl, obs)


def _augment(wl, prob, x_ms, lam_def, lam_lim):
    N = x_ms.shape[0]
    lam_def = np.broadcast_to(np.asarray(lam_def, float), (N, wl.W - 1))
    lam_lim = np.broadcast_to(np.asarray(lam_lim, float), (N, prob.M))
    return np.ascontiguousarray(np.concatenate([x_ms, lam_def, lam_lim], axis=1))


def _particles(wl, prob, rng, N=3):
    x = wlmod.initial_particles(wl, _obs(wl), rng_seed=int(rng.integers(1 << 30)))[:N].copy()
    x[:, prob.M:] += 0.05 * rng.normal(size=(N, prob.P - prob.M))  # non-zero defects
    return x


def test_half_multiplier_reproduces_multiple_shooting():
    wl, obs, prob = _case()
    rng = np.random.default_rng(0)
    x = _particles(wl, prob, rng)
    lp_ms, g_ms = prob.loglik_grad(x)
    xa = _augment(wl, prob, x, 0.5, 0.0)
    lp_obs, out = prob.csvgd_loglik_grad(xa, c=0.0)
    M, S, W, P, Pc = prob.M, prob.S, prob.W, prob.P, prob.Pc
    gdef = out[:, P:P + W - 1]
    sd2 = wl.sigma_def ** 2
    def_terms = (-0.5 * gdef - 0.5 * S * np.log(2 * np.pi * sd2)).sum(axis=1)
    prior = -np.log(wl.hi - wl.lo).sum()  # theta inside the box: no penalty
    np.testing.assert_allclose(lp_obs + def_terms + prior, lp_ms, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(out[:, M:P], g_ms[:, M:P], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(out[:, :M] + out[:, Pc:Pc + M], g_ms[:, :M], rtol=1e-9, atol=1e-9)


def test_defect_values_from_independent_rollouts():
    wl, obs, prob = _case(seed=7, n=2, W=5, T=50)
    rng = np.random.default_rng(1)
    x = _particles(wl, prob, rng, N=2)
    _, out = prob.csvgd_loglik_grad(_augment(wl, prob, x, 0.3, 0.0), c=2.0)
    M, S, W, P = prob.M, prob.S, prob.W, prob.P
    for i in range(x.shape[0]):
        m, l, b = _physical(wl, x[i, :M])
        for w in range(W - 1):
            t0, t1 = (w * wl.T) // W, ((w + 1) * wl.T) // W
            s_start = wl.s0 if w == 0 else x[i, M + (w - 1) * S:M + w * S]
            s_end = orc.simulate(m, l, b, s_start, wl.dt, t1 - t0, g=wl.g)[-1]
            d = x[i, M + w * S:M + (w + 1) * S] - s_end
            assert abs(out[i, P + w] - d @ d / wl.sigma_def ** 2) <= 1e-9 * max(1.0, out[i, P + w])


def test_zero_defects_give_no_constraint_gradient():
    wl, obs, prob = _case(seed=11, n=2, W=4, T=40)
    M, S, W, P, Pc = prob.M, prob.S, prob.W, prob.P, prob.Pc
    theta = wl.theta_init[0]
    m, l, b = _physical(wl, theta)
    st = orc.simulate(m, l, b, wl.s0, wl.dt, wl.T, g=wl.g)
    x = np.concatenate([theta] + [st[(w * wl.T) // W] for w in range(1, W)])[None, :]
    _, out0 = prob.csvgd_loglik_grad(_augment(wl, prob, x, 0.0, 0.0), c=0.0)
    _, out = prob.csvgd_loglik_grad(_augment(wl, prob, x, 3.0, 0.0), c=5.0)
    assert np.max(np.abs(out[:, P:P + W - 1])) <= 1e-20
    np.testing.assert_allclose(out[:, Pc:], 0.0, atol=1e-12)
    np.testing.assert_allclose(out[:, :P], out0[:, :P], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("c", [0.0, 0.7])
def test_constraint_gradient_matches_central_differences(c):
    wl, obs, prob = _case(seed=5, n=2, W=3, T=24)
    rng = np.random.default_rng(2)
    M, S, W, P, Pc = prob.M, prob.S, prob.W, prob.P, prob.Pc
    x = _particles(wl, prob, rng, N=1)[0]
    # two theta components outside the box to exercise the limit constraint
    width = wl.hi - wl.lo
    x[0] = wl.hi[0] + 0.1 * width[0]
    x[1] = wl.lo[1] - 0.07 * width[1]
    lam_def = rng.uniform(-1, 1, W - 1)
    lam_lim = rng.uniform(-1, 1, M)
    xa = _augment(wl, prob, x[None, :], lam_def, lam_lim)

    def psi(xv):
        _, o = prob.csvgd_loglik_grad(_augment(wl, prob, xv[None, :], lam_def, lam_lim), c=c)
        gd, gl = o[0, P:P + W - 1], o[0, P + W - 1:Pc]
        return float(lam_def @ gd + 0.5 * c * gd @ gd + lam_lim @ gl + 0.5 * c * gl @ gl)

    _, out = prob.csvgd_loglik_grad(xa, c=c)
    _, out_obs = prob.csvgd_loglik_grad(_augment(wl, prob, x[None, :], 0.0, 0.0), c=0.0)
    fd = np.zeros(P)
    for k in range(P):
        h = 1e-6 * max(1.0, abs(x[k]))
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd[k] = (psi(xp) - psi(xm)) / (2 * h)
    scale = max(1.0, np.max(np.abs(fd)))
    assert np.max(np.abs(-out[0, Pc:] - fd[:M])) <= 1e-6 * scale
    assert np.max(np.abs(-(out[0, M:P] - out_obs[0, M:P]) - fd[M:P])) <= 1e-6 * scale
    u = (x[:M] - wl.lo) / width
    np.testing.assert_allclose(out[0, P + W - 1:Pc], np.clip(u, 0, 1) - u, atol=1e-15)


def test_step_moves_multipliers_by_lr_g_and_theta_by_sign():
    rng = np.random.default_rng(4)
    M, n_shoot, n_def = 3, 4, 2
    Pc = M + n_shoot + n_def + M
    lo, hi = np.zeros(M), np.array([1.0, 2.0, 4.0])
    x = np.ascontiguousarray(np.concatenate([rng.uniform(0.2, 0.8, M) * hi, rng.normal(size=n_shoot),
                                             rng.normal(size=n_def), rng.normal(size=M)])[None, :])
    out = rng.normal(size=(1, Pc + M))
    st = orc.CsvgdState(1, Pc, n_def, lo, hi, lr=1e-2)
    x0 = x.copy()
    st.step(x, out)
    lam0 = M + n_shoot
    np.testing.assert_allclose(x[0, lam0:], x0[0, lam0:] + 1e-2 * out[0, lam0:Pc], rtol=0, atol=1e-15)
    # N = 1: phi = gradient in u (k = 1, no repulsion); first Adam step = lr * sign
    direction = out[0, :M] * hi + out[0, Pc:] * hi
    np.testing.assert_allclose((x[0, :M] - x0[0, :M]) / hi, 1e-2 * np.sign(direction), rtol=1e-6)
    np.testing.assert_allclose(x[0, M:lam0] - x0[0, M:lam0], 1e-2 * np.sign(out[0, M:lam0]), rtol=1e-6)


def test_mdmm_settles_on_the_constrained_optimum():
    """Maximise -(theta - a)^2 / 2 on [0, 1] with a = 1.5: the constrained
    optimum is theta = 1 with multiplier 1 - a = -0.5 (approximate pin)."""
    a, c = 1.5, 1.0
    lo, hi = np.zeros(1), np.ones(1)
    x = np.array([[0.5, 0.0]])  # theta, lambda_lim
    st = orc.CsvgdState(1, 2, 0, lo, hi, lr=1e-2)
    hist = []
    for _ in range(20000):
        th, lam = x[0]
        g = min(1.0, max(0.0, th)) - th
        dg = -1.0 if (th < 0 or th > 1) else 0.0
        out = np.array([[-(th - a), g, -(lam + c * g) * dg]])
        st.step(x, out)
        hist.append(x[0].copy())
    tail = np.array(hist[-1000:])
    assert abs(tail[:, 0].mean() - 1.0) < 1e-3, tail[:, 0].mean()
    assert abs(tail[:, 1].mean() - (1.0 - a)) < 1e-3, tail[:, 1].mean()
