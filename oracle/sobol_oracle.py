"""FP64 reference of the Sobol initialisation (test infrastructure only: only
the test suite, the smoke check and the benchmark's CPU legs may import it).

App. A-A: the estimators' particles start from the deterministic Sobol
sequence over the parameter limits.  The reference takes the sequence from a
library routine, scipy's unscrambled Sobol generator (Gray-code order, point 0
the origin, direction numbers of Joe and Kuo 2008), and scales it to the box:
    theta_k(n) = lo_k + x_k(n) (hi_k - lo_k),  n = skip, ..., skip + N - 1.
"""
from __future__ import annotations

import warnings

import numpy as np
from scipy.stats import qmc


def sobol_unit(N: int, d: int, skip: int = 0) -> np.ndarray:
    """Points skip .. skip + N - 1 of the d-dimensional Sobol sequence, [N][d]."""
    eng = qmc.Sobol(d, scramble=False)
    if skip:
        eng.fast_forward(int(skip))
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")  # balance warning for N not a power of 2
        return eng.random(int(N))


def sobol_box(N: int, lo, hi, skip: int = 0) -> np.ndarray:
    """Sobol points scaled to the box [lo, hi], [N][M]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + sobol_unit(N, lo.size, skip) * (hi - lo)
