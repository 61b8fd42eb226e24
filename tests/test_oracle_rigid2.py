"""Pins of the oracle's rigid double pendulum (the 11-parameter model of the
physical double pendulum, Sec. V; 6-D articulated-body algorithm), on the CPU:
  * Euler-Lagrange equations derived by sympy from the links' COM positions,
    masses, rotational inertias and joint friction (1e-10);
  * point masses at the link tips reduce it to the planar point-mass chain,
    whose ABA and CRBA are pinned elsewhere (1e-12);
  * with parallel joint axes the motion does not depend on the inertia
    entries other than I_zz nor on the COM's z offset (1e-12);
  * without friction the energy stays bounded with no secular drift and its
    error shrinks with dt; with friction it decays;
  * the multiple-shooting log-likelihood with W = 1 equals scipy's Gaussian
    log density of the rollout plus the uniform prior; its dual-number
    gradient equals central differences for all 11 parameters and the
    shooting states (1e-6).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import pds_oracle as orc

sympy = pytest.importorskip("sympy")

G = 9.81


def _random_params(rng):
    lo = np.array([0.05, 0.002, -0.2, -0.2, 0.0, 0.08, 0.05, 0.002, -0.2, -0.2, 0.0])
    hi = np.array([0.5, 1.0, 0.2, 0.2, 0.5, 0.3, 0.5, 1.0, 0.2, 0.2, 0.5])
    return rng.uniform(lo, hi)


def _lagrange_qdd():
    q1, q2, v1, v2 = sympy.symbols("q1 q2 v1 v2")
    m1, I1, ax1, ay1, b1, l, m2, I2, ax2, ay2, b2 = sympy.symbols("m1 I1 ax1 ay1 b1 l m2 I2 ax2 ay2 b2")
    t = sympy.symbols("t")
    Q1, Q2 = sympy.Function("Q1")(t), sympy.Function("Q2")(t)

    def rot(a):
        return sympy.Matrix([[sympy.cos(a), -sympy.sin(a)], [sympy.sin(a), sympy.cos(a)]])

    c1 = rot(Q1) * sympy.Matrix([ax1, ay1])
    j2 = rot(Q1) * sympy.Matrix([0, -l])
    c2 = j2 + rot(Q1 + Q2) * sympy.Matrix([ax2, ay2])
    dc1, dc2 = c1.diff(t), c2.diff(t)
    w1, w2 = Q1.diff(t), Q1.diff(t) + Q2.diff(t)
    Tk = (m1 * dc1.dot(dc1) + m2 * dc2.dot(dc2) + I1 * w1 ** 2 + I2 * w2 ** 2) / 2
    V = G * (m1 * c1[1] + m2 * c2[1])
    L = Tk - V
    eqs = []
    for Q, b in ((Q1, b1), (Q2, b2)):
        e = sympy.diff(L.diff(Q.diff(t)), t) - L.diff(Q) + b * Q.diff(t)
        eqs.append(e)
    a1, a2 = sympy.symbols("a1 a2")
    subs = {Q1.diff(t, 2): a1, Q2.diff(t, 2): a2}
    eqs = [e.subs(subs) for e in eqs]
    subs = {Q1.diff(t): v1, Q2.diff(t): v2}
    eqs = [e.subs(subs) for e in eqs]
    subs = {Q1: q1, Q2: q2}
    eqs = [e.subs(subs) for e in eqs]
    # the equations are linear in the accelerations: M a + h = 0
    Mrows = [[e.diff(a1), e.diff(a2)] for e in eqs]
    h = [e.subs({a1: 0, a2: 0}) for e in eqs]
    args = (q1, q2, v1, v2, m1, I1, ax1, ay1, b1, l, m2, I2, ax2, ay2, b2)
    fM = sympy.lambdify(args, Mrows, "numpy")
    fh = sympy.lambdify(args, h, "numpy")

    def qdd(*a):
        return np.linalg.solve(np.array(fM(*a), dtype=np.float64), -np.array(fh(*a), dtype=np.float64))

    return qdd


def test_matches_euler_lagrange():
    f = _lagrange_qdd()
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = _random_params(rng)
        s = np.concatenate([rng.uniform(-3, 3, 2), rng.uniform(-4, 4, 2)])
        ref = np.array(f(*s, *p), dtype=np.float64)
        got = orc.rigid2_qdd(p, G, s)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_point_masses_reduce_to_the_chain():
    rng = np.random.default_rng(2)
    for _ in range(10):
        m = rng.uniform(0.2, 2.0, 2)
        L = rng.uniform(0.3, 1.5, 2)
        b = rng.uniform(0.0, 0.5, 2)
        q, qd = rng.uniform(-2, 2, 2), rng.uniform(-3, 3, 2)
        got = orc.rigid2_qdd_full(m, [[0, -L[0], 0], [0, -L[1], 0]], np.zeros((2, 3, 3)), b, L[0], G,
                                  np.concatenate([q, qd]))
        ref = orc.aba(m, L, np.zeros(2), q, qd, -b * qd, g=G)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got, orc.fd_crba(m, L, np.zeros(2), q, qd, -b * qd, g=G), rtol=1e-10,
                                   atol=1e-10)


def test_planar_motion_ignores_off_axis_inertia_and_com_z():
    rng = np.random.default_rng(3)
    for _ in range(10):
        p = _random_params(rng)
        s = np.concatenate([rng.uniform(-3, 3, 2), rng.uniform(-4, 4, 2)])
        base = orc.rigid2_qdd(p, G, s)
        Ic = np.zeros((2, 3, 3))
        c = np.zeros((2, 3))
        for k, (mi, Ii, cx, cy) in enumerate(((0, 1, 2, 3), (6, 7, 8, 9))):
            A = rng.normal(size=(3, 3))
            S = 0.05 * (A @ A.T)
            S[2, 2] = p[Ii]  # keep the axis component
            Ic[k] = S
            c[k] = [p[cx], p[cy], rng.uniform(-0.3, 0.3)]
        got = orc.rigid2_qdd_full([p[0], p[6]], c, Ic, [p[4], p[10]], p[5], G, s)
        np.testing.assert_allclose(got, base, rtol=1e-12, atol=1e-12)


def _energy(p, s):
    m1, I1, ax1, ay1, _, l, m2, I2, ax2, ay2, _ = p
    q1, q2, v1, v2 = s

    def rot(a, v):
        return np.array([np.cos(a) * v[0] - np.sin(a) * v[1], np.sin(a) * v[0] + np.cos(a) * v[1]])

    def perp(v):
        return np.array([-v[1], v[0]])

    c1 = rot(q1, (ax1, ay1))
    j2 = rot(q1, (0.0, -l))
    r2 = rot(q1 + q2, (ax2, ay2))
    dc1 = v1 * perp(c1)
    dc2 = v1 * perp(j2) + (v1 + v2) * perp(r2)
    T = 0.5 * (m1 * dc1 @ dc1 + m2 * dc2 @ dc2 + I1 * v1 ** 2 + I2 * (v1 + v2) ** 2)
    return T + G * (m1 * c1[1] + m2 * (j2[1] + r2[1]))


def test_energy_without_and_with_friction():
    rng = np.random.default_rng(4)
    p = _random_params(rng)
    p[1], p[7] = 0.01, 0.008
    p[4] = p[10] = 0.0
    s0 = np.array([1.2, -0.7, 0.0, 0.0])
    drift = []
    for dt in (2e-3, 1e-3):
        T = int(round(4.0 / dt))
        st = orc.rigid2_simulate(p, G, dt, T, s0)
        E = np.array([_energy(p, x) for x in st[:: max(1, T // 400)]])
        drift.append(np.max(np.abs(E - E[0])))
        # no secular drift: the last quarter does not sit further from E0 than the first
        q = len(E) // 4
        assert np.mean(np.abs(E[-q:] - E[0])) < 3.0 * np.mean(np.abs(E[1:q + 1] - E[0])) + 1e-12
    assert drift[1] < 0.7 * drift[0]
    p[4], p[10] = 0.2, 0.1
    st = orc.rigid2_simulate(p, G, 1e-3, 4000, s0)
    E = np.array([_energy(p, x) for x in st[::200]])
    assert E[-1] < E[0] - 1e-3


def _problem(rng, T=60, W=3, theta_param=tuple(range(11))):
    p = _random_params(rng)
    p[1], p[7] = rng.uniform(0.005, 0.05, 2)
    s0 = np.array([0.8, -0.4, 0.0, 0.3])
    dt = 0.005
    st = orc.rigid2_simulate(p, G, dt, T, s0)
    obs = st[1:] + 0.01 * rng.standard_normal((T, 4))
    tp = np.asarray(theta_param, dtype=np.int32)
    lo = np.array([0.05, 0.002, -0.2, -0.2, 0.0, 0.08, 0.05, 0.002, -0.2, -0.2, 0.0])[tp]
    hi = np.array([0.5, 1.0, 0.2, 0.2, 0.5, 0.3, 0.5, 1.0, 0.2, 0.2, 0.5])[tp]
    prob = orc.Rigid2Problem(p11=p, g=G, theta_param=tp, dt=dt, T=T, W=W, obs=obs, obs_index=np.arange(4),
                             sigma_obs=0.05, sigma_def=0.1, s0=s0, lo=lo, hi=hi)
    return prob, p, st, obs, lo, hi


def test_single_window_equals_scipy_densities():
    rng = np.random.default_rng(5)
    prob, p, st, obs, lo, hi = _problem(rng, W=1)
    lp = prob.loglik_grad(p[None, :], grad=False)[0]
    ref = stats.norm.logpdf(obs, loc=st[1:], scale=0.05).sum() + stats.uniform.logpdf(p, lo, hi - lo).sum()
    assert abs(lp - ref) < 1e-9 * abs(ref)


def test_gradient_equals_central_differences():
    rng = np.random.default_rng(6)
    prob, p, st, obs, lo, hi = _problem(rng, W=3)
    x = np.concatenate([p, st[20] + 0.01, st[40] - 0.02])
    x[3] = hi[3] + 0.01  # one parameter outside the box: the limit penalty acts
    lp, g = prob.loglik_grad(x[None, :])
    fd = np.zeros_like(x)
    for k in range(len(x)):
        h = 1e-6 * max(1.0, abs(x[k]))
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd[k] = (prob.loglik_grad(xp[None, :], grad=False)[0] - prob.loglik_grad(xm[None, :], grad=False)[0]) / (2 * h)
    np.testing.assert_allclose(g[0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
