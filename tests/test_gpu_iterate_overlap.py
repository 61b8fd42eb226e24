"""pds_iterate with the SVGD step's median beside the likelihood.

On a stream that can be captured, pds_iterate runs each iteration as one
graph: the median bandwidth of the step (Sec. IV-A's median heuristic, which
reads only the particles' coordinates) on a side stream while the rollout
and its adjoint run, then the rest of the step (Eq. 1's phi and the Adam
update of Algorithm 1).  A particle whose coordinates are finite but whose
gradient is not is then taken out after the median was computed, and the
full radix passes compute the median again over the particles that remain.

Covers:
  * several iterations give the same particles and log p, bit for bit, as
    pds_loglik_grad followed by pds_svgd_step on the same stream;
  * the same with a particle whose gradient is not finite (a shooting state
    far outside the trajectory) and one whose coordinates are not;
  * the first two calls (direct launches, then the capture) and the replays
    agree.
"""
import numpy as np
import pytest
import torch

from helpers import f32_workload, observations, particles
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _setup(wl, obs, x, stream):
    prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=1, fast_math=1)
    sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
    with torch.cuda.stream(stream):
        X = torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).cuda()
    return prob, sv, X


@pytest.mark.parametrize("divergent", [False, True])
def test_overlapped_iteration_equals_loglik_then_step(divergent):
    wl = f32_workload(wlmod.chain5(N=4096, T=200, W=4))
    obs = observations(wl)
    x = particles(wl, obs)
    if divergent:
        x[17, wl.M + 7] = 1e30      # a shooting velocity: finite coordinates, gradient not finite
        x[4000, 3] = np.nan         # a coordinate that is not finite
    iters = 4
    s1 = torch.cuda.Stream()
    prob, sv, X = _setup(wl, obs, x, s1)
    lp1 = torch.empty(wl.N, device="cuda")
    for _ in range(iters):
        with torch.cuda.stream(s1):
            api.iterate(prob, sv, X, 1, lp1)
    s1.synchronize()
    xa, lpa = X.cpu().numpy(), lp1.cpu().numpy()
    prob.close()
    sv.close()

    s2 = torch.cuda.Stream()
    prob, sv, X = _setup(wl, obs, x, s2)
    lp2 = torch.empty(wl.N, device="cuda")
    G = torch.empty((prob.grad_rows, wl.N), device="cuda")
    L = api.lib()
    for _ in range(iters):
        with torch.cuda.stream(s2):
            assert L.pds_loglik_grad(prob.handle, api._ptr(X), wl.N, api._ptr(lp2), api._ptr(G), None) == 0
            assert L.pds_svgd_step(sv.handle, api._ptr(X), api._ptr(G), None, None) == 0
    s2.synchronize()
    xb, lpb = X.cpu().numpy(), lp2.cpu().numpy()
    prob.close()
    sv.close()

    np.testing.assert_array_equal(lpa, lpb)
    np.testing.assert_array_equal(xa, xb)
    if divergent:
        assert not np.isfinite(lpa[17]) and not np.isfinite(lpa[4000])
        assert np.isfinite(np.delete(lpa, [17, 4000])).all()
