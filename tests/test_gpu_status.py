"""Errors that the device finds while an SVGD step runs reach the host.

Every mbarrier wait of the tensor-core passes (the median's distance tiles,
phi's kernel-matrix products) is bounded.  A pass that runs out of polls lets
its copies and products in flight finish, frees its tensor memory, flags the
step, and returns; the host then sees PDS_ERR_TIMEOUT from pds_svgd_status or
from the next step.  The test makes the waits run out by setting the poll
limit to 0 (test each barrier once, never wait): the first product of every
CTA has not landed when it is first tested.  It then checks that the GPU is
still usable by running a step with the default limit against the oracle.
A step in which no particle is finite reports PDS_ERR_NONFINITE the same way.
"""
import numpy as np
import pytest
import torch

from helpers import PHI_TOL
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _case(N, M, P, seed):
    rng = np.random.default_rng(seed)
    lo = np.zeros(M)
    hi = np.ones(M)
    x = np.concatenate([rng.uniform(0.05, 0.95, (N, M)), rng.normal(size=(N, P - M))], 1)
    g = rng.normal(size=(N, P))
    return lo, hi, x.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("N,M", [(4096, 10), (700, 4)])
def test_tensor_core_pass_that_gives_up_reports_timeout(N, M):
    """N = 4096: both tensor-core passes (median tiles and phi); N = 700: phi
    alone (the median runs on the CUDA cores below N = 2048)."""
    P = M + 4
    lo, hi, x, g = _case(N, M, P, seed=N)
    sv = api.Svgd(N, M, P, lo, hi)
    sv.set_option(api.OPT_WAIT_LIMIT, 0)
    X, G = _gpu(x), _gpu(g)
    sv.step(X, G)
    assert sv.status() == api.ERR_TIMEOUT
    assert sv.status() == 0  # reading clears it
    # reported by the next step call as well, which then queues nothing
    sv.step(X, G)
    torch.cuda.synchronize()
    with pytest.raises(api.PdsError) as e:
        sv.step(X, G)
    assert e.value.code == api.ERR_TIMEOUT
    # the context is intact: the default limit gives the oracle's step
    sv.set_option(api.OPT_WAIT_LIMIT, 1 << 24)
    sv.reset()
    X = _gpu(x)
    bw, phi = sv.step(X, G, return_phi=True)
    assert sv.status() == 0
    ost = orc.SvgdState(N, P, lo, hi, lr=1e-2)
    xo = np.ascontiguousarray(x.copy())
    phi_ref, bw_ref = ost.step(xo, g)
    assert abs(bw.item() - bw_ref) <= 1e-5 * bw_ref
    phi = phi.cpu().numpy().T
    assert np.max(np.abs(phi - phi_ref)) <= PHI_TOL * np.max(np.abs(phi_ref))
    sv.close()


def test_step_with_no_finite_particle_reports_nonfinite():
    N, M, P = 300, 3, 5
    lo, hi, x, g = _case(N, M, P, seed=4)
    x[:, 1] = np.nan
    sv = api.Svgd(N, M, P, lo, hi)
    X = _gpu(x)
    sv.step(X, _gpu(g))
    assert sv.status() == api.ERR_NONFINITE
    # one finite particle is enough
    x[5, 1] = 0.5
    sv.step(_gpu(x), _gpu(g))
    assert sv.status() == 0
    sv.close()


def test_wait_limit_option_rejects_negative_values():
    sv = api.Svgd(10, 2, 2, [0, 0], [1, 1])
    with pytest.raises(api.PdsError) as e:
        sv.set_option(api.OPT_WAIT_LIMIT, -1)
    assert e.value.code == api.ERR_ARG
    sv.close()
