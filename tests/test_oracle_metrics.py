"""Pins of the metric references (CPU only): the KNN-KL estimate converges to
the closed-form KL divergence of two Gaussians, is 0-centred for two samples
of one distribution, and scales with the dimension as the closed form does;
the unbiased MMD^2 converges to its closed form for Gaussian samples under
the RBF kernel and has zero mean under equal distributions (approximate
pins, with tolerances from the estimators' spread)."""
import numpy as np

from oracle import metrics_oracle as mo


def _kl_gauss(mu0, s0, mu1, s1):
    """KL(N(mu0, s0^2 I) || N(mu1, s1^2 I)) in d dimensions (closed form)."""
    d = len(mu0)
    return 0.5 * (d * s0 ** 2 / s1 ** 2 + np.sum((mu1 - mu0) ** 2) / s1 ** 2 - d + 2 * d * np.log(s1 / s0))


def test_knn_kl_converges_to_the_gaussian_closed_form():
    rng = np.random.default_rng(0)
    for d, mu, s1 in [(2, 1.0, 1.0), (3, 0.5, 1.5)]:
        mu1 = np.full(d, mu)
        p = rng.normal(size=(2500, d))            # unequal set sizes exercise log(m / (n - 1))
        q = mu1 + s1 * rng.normal(size=(6000, d))
        ref = _kl_gauss(np.zeros(d), 1.0, mu1, s1)
        est = mo.knn_kl(p, q, k=3)
        assert abs(est - ref) <= 0.08 + 0.05 * ref, (d, est, ref)


def test_knn_kl_of_one_distribution_is_near_zero():
    rng = np.random.default_rng(1)
    est = [mo.knn_kl(rng.normal(size=(1500, 2)), rng.normal(size=(1500, 2))) for _ in range(4)]
    assert abs(np.mean(est)) <= 0.05, est


def test_mmd_matches_the_gaussian_closed_form():
    """E k(x, x') = (1 + 4 s^2 / h)^(-d/2) for x, x' ~ N(mu, s^2 I); across two
    Gaussians E k(x, y) = (1 + 2(s1^2 + s2^2)/h)^(-d/2) exp(-|mu1 - mu2|^2 / (h + 2(s1^2 + s2^2)))."""
    rng = np.random.default_rng(2)
    d, h = 2, 1.5
    mu1, s1, mu2, s2 = np.zeros(d), 1.0, np.array([0.8, -0.3]), 0.7
    exx = (1 + 4 * s1 ** 2 / h) ** (-d / 2)
    eyy = (1 + 4 * s2 ** 2 / h) ** (-d / 2)
    v = s1 ** 2 + s2 ** 2
    exy = (1 + 2 * v / h) ** (-d / 2) * np.exp(-np.sum((mu1 - mu2) ** 2) / (h + 2 * v))
    ref = exx + eyy - 2 * exy
    est = [mo.mmd2_unbiased(mu1 + s1 * rng.normal(size=(1500, d)), mu2 + s2 * rng.normal(size=(1500, d)), h)
           for _ in range(4)]
    assert abs(np.mean(est) - ref) <= 0.05 * ref + 2e-3, (np.mean(est), ref)


def test_mmd_has_zero_mean_under_equal_distributions():
    rng = np.random.default_rng(3)
    est = [mo.mmd2_unbiased(rng.normal(size=(800, 3)), rng.normal(size=(800, 3)), 2.0) for _ in range(6)]
    assert abs(np.mean(est)) <= 2e-3, est
