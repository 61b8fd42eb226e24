"""GPU parity of the posterior metrics (pds_knn_kl, pds_mmd2) against the
FP64 references on the same float32 samples: KNN-KL (Eq. knn-kl, k = 1..8)
and the unbiased RBF MMD^2, for dimensions 1-64, set sizes that span
several 128-point tiles with ragged tails, and the argument checks."""
import numpy as np
import pytest
import torch

from oracle import metrics_oracle as mo
from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float32).T)).cuda()


@pytest.mark.parametrize("n,m,d,k", [(300, 400, 2, 3), (129, 1000, 10, 3), (1000, 257, 4, 1), (200, 200, 33, 5),
                                     (64, 90, 64, 8)])
def test_knn_kl_matches_reference(n, m, d, k):
    rng = np.random.default_rng(n + m + d)
    p = rng.normal(size=(n, d)).astype(np.float32).astype(np.float64)
    q = (0.4 + 1.3 * rng.normal(size=(m, d))).astype(np.float32).astype(np.float64)
    got = api.knn_kl(_gpu(p), _gpu(q), k=k)
    ref = mo.knn_kl(p, q, k=k)
    assert abs(got - ref) <= 1e-4 * max(1.0, abs(ref)), (got, ref)


@pytest.mark.parametrize("n,m,d,h", [(300, 400, 2, 1.0), (129, 1000, 10, 5.0), (1000, 257, 4, 0.3),
                                     (200, 200, 33, 20.0)])
def test_mmd2_matches_reference(n, m, d, h):
    rng = np.random.default_rng(n * m + d)
    x = rng.normal(size=(n, d)).astype(np.float32).astype(np.float64)
    y = (0.3 + rng.normal(size=(m, d))).astype(np.float32).astype(np.float64)
    got = api.mmd2(_gpu(x), _gpu(y), h)
    ref = mo.mmd2_unbiased(x, y, h)
    assert abs(got - ref) <= 1e-5 + 1e-4 * abs(ref), (got, ref)


def test_metric_arguments_are_checked():
    x = _gpu(np.zeros((4, 2)))
    with pytest.raises(api.PdsError):
        api.knn_kl(x, x, k=9)
    with pytest.raises(api.PdsError):
        api.knn_kl(x, x, k=4)  # n must exceed k
    with pytest.raises(api.PdsError):
        api.mmd2(x, x, 0.0)
    big = _gpu(np.zeros((4, 65)))
    with pytest.raises(api.PdsError):
        api.mmd2(big, big, 1.0)
