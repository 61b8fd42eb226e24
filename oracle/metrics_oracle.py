"""FP64 reference of the posterior metrics (test infrastructure only: only
the test suite, the smoke check and the benchmark's CPU legs may import it).

  * KNN-based KL divergence estimate between two sample sets (the paper's
    Eq. knn-kl, after Wang, Kulkarni and Verdu 2009), with k_i = l_i = k:
        D(P || Q) ~ (d / n) sum_i log( nu_k(i) / rho_k(i) )
                    + (1 / n) sum_i [psi(k) - psi(k)] + log( m / (n - 1) )
    nu_k(i): Euclidean distance from p_i to its k-th nearest neighbour in Q;
    rho_k(i): distance from p_i to its k-th nearest neighbour in P without p_i;
    n = |P|, m = |Q|, d = dimension.
  * Squared maximum mean discrepancy with the RBF kernel
    k(x, y) = exp(-||x - y||^2 / h), unbiased estimate (Gretton et al. 2012):
        MMD^2_u = 1/(n(n-1)) sum_{i != j} k(x_i, x_j)
                + 1/(m(m-1)) sum_{i != j} k(y_i, y_j)
                - 2/(n m) sum_{i, j} k(x_i, y_j).
Both written out from the definitions with numpy, brute force.
"""
from __future__ import annotations

import numpy as np


def _sqdist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return ((a[:, None, :] - b[None, :, :]) ** 2).sum(axis=-1)


def knn_kl(p: np.ndarray, q: np.ndarray, k: int = 3) -> float:
    """D(P || Q) estimate; p [n][d], q [m][d]."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n, d = p.shape
    m = q.shape[0]
    dpq = np.sqrt(_sqdist(p, q))
    dpp = np.sqrt(_sqdist(p, p))
    np.fill_diagonal(dpp, np.inf)  # p_i itself is not a neighbour
    nu = np.sort(dpq, axis=1)[:, k - 1]
    rho = np.sort(dpp, axis=1)[:, k - 1]
    return float(d / n * np.sum(np.log(nu / rho)) + np.log(m / (n - 1)))


def mmd2_unbiased(x: np.ndarray, y: np.ndarray, h: float) -> float:
    """MMD^2_u with k(a, b) = exp(-||a - b||^2 / h); x [n][d], y [m][d]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, m = x.shape[0], y.shape[0]
    kxx = np.exp(-_sqdist(x, x) / h)
    kyy = np.exp(-_sqdist(y, y) / h)
    kxy = np.exp(-_sqdist(x, y) / h)
    sxx = (kxx.sum() - np.trace(kxx)) / (n * (n - 1))
    syy = (kyy.sum() - np.trace(kyy)) / (m * (m - 1))
    return float(sxx + syy - 2.0 * kxy.mean())
