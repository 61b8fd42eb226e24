"""Pins of the oracle's SVGD step (Sec. IV-A, Eq. 1) (CPU only).

* N = 1: the kernel is 1 and the repulsion vanishes, so phi is the gradient.
* The median heuristic's median equals a brute-force sort of all pairwise
  squared distances (lower middle element for an even count).
* On a linear-Gaussian target N(mu, Sigma), iterating SVGD + Adam recovers
  the closed-form mean and covariance (an approximate pin: SVGD's particle
  approximation with N = 400 particles, stated tolerance).
"""
import numpy as np
import pytest

from oracle import pds_oracle as orc


def test_single_particle_phi_is_gradient():
    rng = np.random.default_rng(0)
    u = rng.uniform(size=(1, 6))
    g = rng.normal(size=(1, 6))
    assert orc.bandwidth(1, orc.median_sqdist(u)) == 1.0
    np.testing.assert_array_equal(orc.svgd_phi(u, g, 0.37), g)


@pytest.mark.parametrize("N,M", [(2, 3), (3, 1), (4, 2), (17, 5), (64, 10)])
def test_median_is_lower_middle_of_sorted_pairs(N, M):
    rng = np.random.default_rng(N * 31 + M)
    u = rng.uniform(size=(N, M))
    d = np.sort([np.sum((u[i] - u[j]) ** 2) for i in range(N) for j in range(i + 1, N)])
    assert orc.median_sqdist(u) == d[(len(d) - 1) // 2]


def test_bandwidth_rule():
    assert orc.bandwidth(100, 0.5) == pytest.approx(0.5 / np.log(100), rel=1e-15)
    assert orc.bandwidth(50, 0.0) == 1.0
    assert orc.bandwidth(1, 3.0) == 1.0


def test_two_particles_repel_symmetrically():
    """With zero gradient, two particles move apart along their difference."""
    u = np.array([[0.4, 0.5], [0.6, 0.5]])
    g = np.zeros_like(u)
    bw = 0.3
    phi = orc.svgd_phi(u, g, bw)
    k = np.exp(-0.04 / bw)
    # (1/N) * (2/bw) * (u_i - u_j) * k for the one other particle
    np.testing.assert_allclose(phi[0], 0.5 * (2 / bw) * (u[0] - u[1]) * k, rtol=1e-14)
    np.testing.assert_allclose(phi[1], -phi[0], rtol=1e-14)


@pytest.mark.slow
def test_linear_gaussian_posterior_recovered():
    mu = np.array([0.3, -0.2])
    Sig = np.array([[0.04, 0.018], [0.018, 0.025]])
    Prec = np.linalg.inv(Sig)
    lo, hi = np.array([-2.0, -2.0]), np.array([2.0, 2.0])
    N = 400
    rng = np.random.default_rng(42)
    x = np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(N, 2)))
    st = orc.SvgdState(N, 2, lo, hi, lr=2e-2, clamp=False)
    for _ in range(1500):
        grad = -(x - mu) @ Prec          # closed-form d log N(x | mu, Sigma) / dx
        st.step(x, grad)
    sd = np.sqrt(np.diag(Sig))
    assert np.all(np.abs(x.mean(0) - mu) < 0.05 * sd)
    C = np.cov(x.T)
    assert np.all(np.abs(np.diag(C) - np.diag(Sig)) < 0.1 * np.diag(Sig))
    assert abs(C[0, 1] - Sig[0, 1]) < 0.1 * np.sqrt(Sig[0, 0] * Sig[1, 1])


def test_adam_step_on_shooting_states_and_clamp():
    """Shooting rows follow plain Adam ascent on their own gradient; theta
    rows are clamped to the box after the update."""
    N, M, P = 3, 2, 4
    lo, hi = np.array([0.0, 1.0]), np.array([1.0, 3.0])
    x = np.ascontiguousarray([[0.999, 2.0, 0.1, 0.2], [0.5, 1.5, -0.3, 0.0], [0.2, 2.9, 1.0, 1.0]], dtype=float)
    g = np.array([[50.0, 0.0, 1.0, -2.0], [0.0, 0.0, 0.5, 0.0], [0.0, 80.0, -1.0, 3.0]])
    st = orc.SvgdState(N, P, lo, hi, lr=0.1)
    x_before = x.copy()
    st.step(x, g)
    # first Adam step moves by lr * sign(g) (|g| >> eps)
    np.testing.assert_allclose(x[:, 2:], x_before[:, 2:] + 0.1 * np.sign(g[:, 2:]), atol=1e-7)
    assert np.all(x[:, :M] >= lo) and np.all(x[:, :M] <= hi)


def test_particles_that_are_not_finite_sit_out_the_step():
    """A particle whose gradient or coordinates are not finite takes no part
    in the step: the others move exactly as in a step over the live subset
    alone (median, bandwidth and the 1/N of Eq. 1 over the live particles),
    and its own direction is NaN."""
    rng = np.random.default_rng(31)
    N, M, P = 40, 3, 5
    lo, hi = np.zeros(M), np.ones(M)
    x = rng.uniform(0.1, 0.9, size=(N, P))
    g = rng.normal(size=(N, P))
    dead = [3, 17, 29]
    g[3, 0] = np.inf
    g[17, 2] = np.nan
    x[29, 1] = np.nan
    live = np.setdiff1d(np.arange(N), dead)
    st = orc.SvgdState(N, P, lo, hi, lr=1e-2)
    xa = x.copy()
    phi, bw = st.step(xa, g)
    sl = orc.SvgdState(len(live), P, lo, hi, lr=1e-2)
    xl = np.ascontiguousarray(x[live])
    phi_l, bw_l = sl.step(xl, np.ascontiguousarray(g[live]))
    assert bw == bw_l
    np.testing.assert_array_equal(phi[live], phi_l)
    np.testing.assert_array_equal(xa[live], xl)
    assert np.all(np.isnan(phi[dead]))


def test_update_with_given_directions_is_the_update_half_of_a_step():
    """The update alone, fed the step's own phi and gradient, moves the
    particles and the Adam moments exactly as the whole step does (Algorithm
    1: the direction, then the Adam ascent); and its Adam arithmetic is the
    textbook one: after two steps with directions d1, d2 the move of an entry
    is lr (m2 / (1 - b1^2)) / (sqrt(v2 / (1 - b2^2)) + eps) on top of the
    first step's lr sign(d1)."""
    rng = np.random.default_rng(8)
    N, M, P = 30, 3, 7
    lo, hi = rng.uniform(-1, 0, M), rng.uniform(1, 2, M)
    x0 = np.ascontiguousarray(np.concatenate([rng.uniform(lo, hi, (N, M)), rng.normal(size=(N, P - M))], 1))
    g1, g2 = rng.normal(size=(N, P)), rng.normal(size=(N, P))
    lr, b1, b2, eps = 0.05, 0.9, 0.999, 1e-8
    whole = orc.SvgdState(N, P, lo, hi, lr=lr, clamp=False)
    half = orc.SvgdState(N, P, lo, hi, lr=lr, clamp=False)
    xw, xh = x0.copy(), x0.copy()
    phis = []
    for g in (g1, g2):
        phi, _ = whole.step(xw, g)
        half.update(xh, phi, g)
        phis.append(phi)
    np.testing.assert_array_equal(xh, xw)
    np.testing.assert_array_equal(half.m, whole.m)
    np.testing.assert_array_equal(half.v, whole.v)
    # Kingma and Ba's bias-corrected update, written out, on the shooting rows
    d1, d2 = g1[:, M:], g2[:, M:]
    m2 = b1 * (1 - b1) * d1 + (1 - b1) * d2
    v2 = b2 * (1 - b2) * d1 ** 2 + (1 - b2) * d2 ** 2
    step1 = lr * ((1 - b1) * d1 / (1 - b1)) / (np.sqrt((1 - b2) * d1 ** 2 / (1 - b2)) + eps)
    step2 = lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    np.testing.assert_allclose(xh[:, M:], x0[:, M:] + step1 + step2, rtol=0, atol=1e-13)
    # theta rows: the same two moves in unit-box coordinates, on phi
    p1, p2 = phis
    m2u = b1 * (1 - b1) * p1 + (1 - b1) * p2
    v2u = b2 * (1 - b2) * p1 ** 2 + (1 - b2) * p2 ** 2
    u0 = (x0[:, :M] - lo) / (hi - lo)
    u2 = u0 + lr * np.sign(p1) * np.abs(p1) / (np.abs(p1) + eps) + lr * (m2u / (1 - b1 ** 2)) / (
        np.sqrt(v2u / (1 - b2 ** 2)) + eps)
    np.testing.assert_allclose(xh[:, :M], lo + u2 * (hi - lo), rtol=0, atol=1e-12)
