"""GPU parity of the Sobol initialisation (App. A-A) against the reference
(scipy's unscrambled Sobol sequence), through the C ABI:
  * bit for bit in the unit box (the points have at most 24 significant bits
    below index 2^24, so fp32 holds them exactly), 1 to 16 dimensions, ragged
    N, with and without a skip;
  * in a general box within fp32 rounding of lo + x (hi - lo);
  * the stratification and (0, m, 2)-net properties on the GPU's own output;
  * writing the first M rows of a particle array leaves the other rows alone;
  * argument checks.
"""
import numpy as np
import pytest
import torch

from oracle import sobol_oracle as so
from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,M,skip", [(1, 1, 0), (4099, 16, 0), (1000, 10, 12345), (65536, 3, 0), (300, 5, 2 ** 24 - 100)])
def test_unit_box_bit_exact(N, M, skip):
    th = torch.empty((M, N), device="cuda")
    api.sobol_box(th, np.zeros(M), np.ones(M), skip=skip)
    ref = so.sobol_unit(N, M, skip).astype(np.float32).T
    got = th.cpu().numpy()
    if skip + N <= 2 ** 24:
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).max() <= 2 ** -24


def test_general_box():
    rng = np.random.default_rng(4)
    M, N = 11, 5000
    lo = rng.uniform(-3, 3, M).astype(np.float32)
    hi = (lo + rng.uniform(0.01, 5, M)).astype(np.float32)
    th = torch.empty((M, N), device="cuda")
    api.sobol_box(th, lo, hi, skip=7)
    ref = so.sobol_box(N, lo.astype(np.float64), hi.astype(np.float64), skip=7).T
    tol = 2.0 ** -22 * (np.abs(lo) + np.abs(hi))[:, None]
    assert np.all(np.abs(th.cpu().numpy() - ref) <= tol)


def test_net_properties_of_gpu_points():
    m = 12
    th = torch.empty((16, 2 ** m), device="cuda")
    api.sobol_box(th, np.zeros(16), np.ones(16))
    x = th.cpu().numpy().astype(np.float64)
    for k in range(16):
        assert np.array_equal(np.sort(np.floor(x[k] * 2 ** m)), np.arange(2 ** m))
    for p in range(m + 1):
        a = np.floor(x[0] * 2 ** p).astype(np.int64)
        b = np.floor(x[1] * 2 ** (m - p)).astype(np.int64)
        assert np.all(np.bincount(a * 2 ** (m - p) + b, minlength=2 ** m) == 1)


def test_fills_theta_rows_of_particles_only():
    P, M, N = 40, 4, 777
    X = torch.full((P, N), 7.0, device="cuda")
    api.sobol_box(X[:M], np.zeros(M), np.ones(M) * 2)
    assert torch.all(X[M:] == 7.0)
    assert torch.all((X[:M] >= 0) & (X[:M] < 2))


def test_sobol_rejects_bad_arguments():
    th = torch.empty((17, 10), device="cuda")
    with pytest.raises(api.PdsError):
        api.sobol_box(th, np.zeros(17), np.ones(17))
    th = torch.empty((2, 10), device="cuda")
    with pytest.raises(api.PdsError):
        api.sobol_box(th, np.zeros(2), np.array([1.0, 0.0]))
    with pytest.raises(api.PdsError):
        api.sobol_box(th, np.zeros(2), np.ones(2), skip=2 ** 32 - 5)
    with pytest.raises(api.PdsError):
        api.sobol_box(th, np.zeros(2), np.ones(2), skip=-1)
