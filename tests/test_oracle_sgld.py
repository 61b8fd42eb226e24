"""Pins of the oracle's SGLD estimator (Welling and Teh 2011) with the
multiple-shooting likelihood, on the CPU:
  * the noise generator's SplitMix64 stream reproduces the published test
    vector of the reference implementation (seed 1234567);
  * its Box-Muller normals are standard normal (Kolmogorov-Smirnov) and
    uncorrelated between neighbouring indices;
  * with a constant step on a Gaussian target the chains sample the target's
    mean and variance (the eps/2 drift against sqrt(eps) noise: a factor 2 in
    either would double or halve the variance); approximate pin;
  * a step moves theta in unit-box coordinates and clips it to the box.
"""
import numpy as np
from scipy import stats

from oracle import pds_oracle as orc


def test_splitmix64_reference_vector():
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    assert [orc.splitmix64(1234567, i) for i in range(1, 6)] == ref


def test_normals_are_standard_and_uncorrelated():
    z = np.array([orc.langevin_normal(99, k) for k in range(60000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 0.02


def test_chains_sample_a_gaussian_target():
    # target N(mu, diag(s^2)) on two unbounded rows (no theta rows: M = 0 box)
    N, P = 400, 2
    mu, s = np.array([1.0, -2.0]), np.array([0.5, 2.0])
    x = np.ascontiguousarray(np.zeros((N, P)))
    st = orc.SgldState(N, P, np.zeros(0), np.zeros(0), a=2e-2, b=1.0, gamma=0.0, seed=5, clamp=False)
    samples = []
    for it in range(3000):
        g = -(x - mu) / s ** 2
        st.step(x, g)
        if it >= 1000 and it % 10 == 0:
            samples.append(x.copy())
    smp = np.concatenate(samples)
    assert np.all(np.abs(smp.mean(0) - mu) < 0.05 * np.maximum(1.0, s)), smp.mean(0)
    assert np.all(np.abs(smp.std(0) / s - 1.0) < 0.06), smp.std(0) / s


def test_theta_moves_in_unit_coordinates_and_is_clipped():
    lo, hi = np.array([1.0]), np.array([3.0])
    x = np.ascontiguousarray([[2.0, 0.5]])
    g = np.array([[1.5, -1.0]])
    st = orc.SgldState(1, 2, lo, hi, a=1e-2, b=2.0, gamma=0.5, seed=7, clamp=True)
    st.step(x, g)
    eps = 1e-2 * (2.0 + 1) ** -0.5
    xi0, xi1 = orc.langevin_normal(7, 0), orc.langevin_normal(7, 1)
    u = 0.5 + 0.5 * eps * 1.5 * 2.0 + np.sqrt(eps) * xi0
    assert abs(x[0, 0] - (1.0 + 2.0 * np.clip(u, 0, 1))) < 1e-12
    assert abs(x[0, 1] - (0.5 + 0.5 * eps * -1.0 + np.sqrt(eps) * xi1)) < 1e-12
    y = np.ascontiguousarray([[2.999, 0.0]])
    st2 = orc.SgldState(1, 2, lo, hi, a=10.0, b=0.0, gamma=0.0, seed=1, clamp=True)
    st2.step(y, np.array([[1e3, 0.0]]))
    assert y[0, 0] == 3.0
