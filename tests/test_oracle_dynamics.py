"""Pins of the oracle's dynamics against textbook mechanics (CPU only).

The forward dynamics the paper uses is the ABA with semi-implicit Euler
(Appendix B-A, Eq. dynamics).  These tests check the oracle's ABA against
results fixed by mechanics itself, not against the oracle's own formulas:
the closed-form double-pendulum equations of motion, an Euler-Lagrange
derivation done symbolically by sympy, a second forward-dynamics algorithm
(CRBA + Cholesky), the small-angle pendulum period and energy behaviour.
"""
import math

import numpy as np
import pytest

from oracle import pds_oracle as orc

G = 9.81


def textbook_double_pendulum_qdd(m1, m2, l1, l2, q, qd, tau, g=G):
    """Point masses at the link tips, relative angles, q = 0 hanging down.

    M(q) qdd + c(q, qd) + G(q) = tau with the standard closed forms.
    """
    q1, q2 = q
    d1, d2 = qd
    M = np.array([
        [(m1 + m2) * l1 ** 2 + m2 * l2 ** 2 + 2 * m2 * l1 * l2 * math.cos(q2),
         m2 * l2 ** 2 + m2 * l1 * l2 * math.cos(q2)],
        [m2 * l2 ** 2 + m2 * l1 * l2 * math.cos(q2), m2 * l2 ** 2]])
    h = m2 * l1 * l2 * math.sin(q2)
    c = np.array([-h * (2 * d1 * d2 + d2 ** 2), h * d1 ** 2])
    Gv = np.array([(m1 + m2) * g * l1 * math.sin(q1) + m2 * g * l2 * math.sin(q1 + q2),
                   m2 * g * l2 * math.sin(q1 + q2)])
    return np.linalg.solve(M, np.asarray(tau) - c - Gv)


def test_aba_matches_textbook_double_pendulum():
    rng = np.random.default_rng(1)
    for _ in range(50):
        m = rng.uniform(0.2, 3.0, 2)
        l = rng.uniform(0.2, 2.0, 2)
        b = rng.uniform(0.0, 1.0, 2)
        q = rng.uniform(-3, 3, 2)
        qd = rng.uniform(-4, 4, 2)
        tau = -b * qd
        ref = textbook_double_pendulum_qdd(m[0], m[1], l[0], l[1], q, qd, tau)
        got = orc.aba(m, l, b, q, qd, tau)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def _lagrange_qdd_fn(n):
    """Euler-Lagrange equations of a planar point-mass chain, derived by sympy."""
    sp = pytest.importorskip("sympy")
    q = sp.symbols(f"q0:{n}")
    qd = sp.symbols(f"qd0:{n}")
    m = sp.symbols(f"m0:{n}")
    l = sp.symbols(f"l0:{n}")
    g = sp.Symbol("g")
    x = y = 0
    phi = 0
    vx = vy = 0
    T = 0
    V = 0
    for i in range(n):
        phi = phi + q[i]
        x = x + l[i] * sp.sin(phi)
        y = y - l[i] * sp.cos(phi)
        # velocity of the point by the chain rule over all joint angles
        vx = sum(sp.diff(x, q[j]) * qd[j] for j in range(n))
        vy = sum(sp.diff(y, q[j]) * qd[j] for j in range(n))
        T = T + sp.Rational(1, 2) * m[i] * (vx ** 2 + vy ** 2)
        V = V + m[i] * g * y
    L = T - V
    Mmat = sp.Matrix(n, n, lambda i, j: sp.diff(L, qd[i], qd[j]))
    # d/dt dL/dqd = M qdd + sum_j d^2L/(dqd_i dq_j) qd_j
    rest = sp.Matrix([sum(sp.diff(L, qd[i], q[j]) * qd[j] for j in range(n)) - sp.diff(L, q[i]) for i in range(n)])
    args = list(q) + list(qd) + list(m) + list(l) + [g]
    fM = sp.lambdify(args, Mmat, "numpy")
    fr = sp.lambdify(args, rest, "numpy")

    def qdd(mv, lv, qv, qdv, tau, gv=G):
        a = list(qv) + list(qdv) + list(mv) + list(lv) + [gv]
        return np.linalg.solve(np.array(fM(*a), dtype=float), np.asarray(tau) - np.array(fr(*a), dtype=float).ravel())

    return qdd


@pytest.mark.parametrize("n", [1, 3, 4])
def test_aba_matches_euler_lagrange(n):
    f = _lagrange_qdd_fn(n)
    rng = np.random.default_rng(10 + n)
    for _ in range(10):
        m = rng.uniform(0.2, 3.0, n)
        l = rng.uniform(0.2, 1.5, n)
        b = rng.uniform(0.0, 1.0, n)
        q = rng.uniform(-3, 3, n)
        qd = rng.uniform(-3, 3, n)
        tau = -b * qd
        np.testing.assert_allclose(orc.aba(m, l, b, q, qd, tau), f(m, l, q, qd, tau), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n", range(1, 9))
def test_aba_matches_crba_cholesky(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(20):
        m = rng.uniform(0.1, 3.0, n)
        l = rng.uniform(0.1, 1.5, n)
        b = rng.uniform(0.0, 2.0, n)
        q = rng.uniform(-3.5, 3.5, n)
        qd = rng.uniform(-5, 5, n)
        tau = -b * qd
        np.testing.assert_allclose(orc.aba(m, l, b, q, qd, tau), orc.fd_crba(m, l, b, q, qd, tau),
                                   rtol=1e-9, atol=1e-9)


def test_crba_mass_matrix_matches_jacobians():
    """H = sum_k m_k J_k^T J_k for point masses (J_k = d p_k / d q)."""
    rng = np.random.default_rng(7)
    n = 5
    m = rng.uniform(0.1, 3.0, n)
    l = rng.uniform(0.1, 1.5, n)
    q = rng.uniform(-3, 3, n)
    H, _ = orc.crba(m, l, np.zeros(n), q, np.zeros(n))
    phi = np.cumsum(q)
    ref = np.zeros((n, n))
    for k in range(n):
        J = np.zeros((2, n))
        for i in range(k + 1):
            # d p_k / d q_i: rotation about joint i moves every link j >= i
            J[0, i] = sum(l[j] * math.cos(phi[j]) for j in range(i, k + 1))
            J[1, i] = sum(l[j] * math.sin(phi[j]) for j in range(i, k + 1))
        ref += m[k] * J.T @ J
    np.testing.assert_allclose(H, ref, rtol=1e-12, atol=1e-12)


def _upward_crossings(t, x):
    idx = np.nonzero((x[:-1] < 0) & (x[1:] >= 0))[0]
    return t[idx] - x[idx] * (t[idx + 1] - t[idx]) / (x[idx + 1] - x[idx])


def test_small_angle_pendulum_period():
    l, dt, q0 = 1.3, 1e-4, 0.01
    T0 = 2 * math.pi * math.sqrt(l / G)
    steps = int(4 * T0 / dt)
    st = orc.simulate([1.0], [l], [0.0], [q0, 0.0], dt, steps)
    t = np.arange(steps + 1) * dt
    zc = _upward_crossings(t, st[:, 0])
    period = np.mean(np.diff(zc))
    # finite-amplitude correction (1 + q0^2/16) is 6e-6; the integrator's
    # phase error is O((omega dt)^2): both far below the tolerance.
    assert abs(period - T0) / T0 < 1e-4


def test_energy_bounded_single_pendulum():
    m, l, dt = [1.2], [0.8], 1e-3
    st = orc.simulate(m, l, [0.0], [1.0, 0.0], dt, 100_000)
    E = np.array([orc.energy(m, l, s[:1], s[1:]) for s in st[::50]])
    rel = np.abs(E - E[0]) / abs(E[0])
    assert rel.max() < 5e-3
    k = len(E) // 10
    # symplectic Euler: bounded oscillation, no secular trend
    assert abs(np.mean(E[-k:]) - np.mean(E[:k])) / abs(E[0]) < 1e-4


def test_energy_drift_first_order_in_dt_double_pendulum():
    m, l = [1.0, 0.7], [0.9, 0.6]
    s0 = [1.2, -0.5, 0.0, 0.0]

    def max_drift(dt):
        st = orc.simulate(m, l, [0.0, 0.0], s0, dt, int(round(1.0 / dt)))
        E = np.array([orc.energy(m, l, s[:2], s[2:]) for s in st])
        return np.max(np.abs(E - E[0]))

    d1, d2, d3 = max_drift(1e-3), max_drift(5e-4), max_drift(2.5e-4)
    assert 1.6 < d1 / d2 < 2.5 and 1.6 < d2 / d3 < 2.5


def test_damping_dissipates_energy():
    n = 3
    m, l, b = [1.0, 0.5, 0.8], [0.7, 0.5, 0.4], [0.3, 0.2, 0.4]
    dt = 1e-3
    st = orc.simulate(m, l, b, [1.0, -0.7, 0.4, 0.0, 0.0, 0.0], dt, 5000)
    E = np.array([orc.energy(m, l, s[:n], s[n:]) for s in st])
    assert E[-1] < E[0] - 0.1 * abs(E[0] - E.min())
    # non-increasing up to the integrator's O(dt) energy oscillation
    running_min = np.minimum.accumulate(E)
    assert np.max(E - running_min) < 5e-2 * abs(E[0] - E.min()) + 1e-3


def test_step_is_semi_implicit_euler():
    """q_{t+1} uses the new velocity (Eq. dynamics), not the old one."""
    rng = np.random.default_rng(3)
    n = 3
    m, l, b = rng.uniform(0.3, 2, n), rng.uniform(0.3, 1, n), rng.uniform(0, 1, n)
    s = rng.uniform(-1, 1, 2 * n)
    dt = 0.01
    qdd = orc.fd_crba(m, l, b, s[:n], s[n:], -b * s[n:])
    v1 = s[n:] + qdd * dt
    q1 = s[:n] + v1 * dt
    np.testing.assert_allclose(orc.step(m, l, b, s, dt), np.concatenate([q1, v1]), rtol=1e-12, atol=1e-12)
