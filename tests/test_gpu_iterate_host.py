"""pds_iterate_host (Algorithm 1 on host-resident particles) equals
pds_iterate on device buffers bit for bit.  For a single planar-chain
trajectory the host path copies the particle rows in groups of windows and
starts each group's rollout as its rows land (the copy overlaps the
rollout); the kernels and their arithmetic are the same.  Covered: one and
several iterations, window counts below and above the number of copy
groups, uneven windows, and the paths that copy in one piece (the
arm-and-box system, constrained SVGD)."""
import numpy as np
import pytest
import torch

from helpers import f32_workload, observations, particles
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _pair(make_problem, make_svgd, x, iters):
    host = np.ascontiguousarray(x.T, dtype=np.float32)
    lp_h = np.empty(host.shape[1], np.float32)
    p1, s1 = make_problem(), make_svgd()
    xh = host.copy()
    api.iterate_host(p1, s1, xh, iters, lp_h)
    p2, s2 = make_problem(), make_svgd()
    X = torch.from_numpy(host.copy()).cuda()
    lp_d = torch.empty(host.shape[1], device="cuda")
    api.iterate(p2, s2, X, iters, lp_d)
    torch.cuda.synchronize()
    for o in (p1, s1, p2, s2):
        o.close()
    return xh, lp_h, X.cpu().numpy(), lp_d.cpu().numpy()


@pytest.mark.parametrize("N,T,W,iters,fast", [(700, 140, 7, 1, 1), (300, 200, 20, 3, 1), (129, 97, 11, 2, 0),
                                              (2100, 60, 3, 1, 1), (64, 50, 1, 2, 0)])
def test_host_iterations_equal_device_iterations(N, T, W, iters, fast):
    wl = f32_workload(wlmod.chain5(N=N, T=T, W=W))
    obs = observations(wl)
    x = particles(wl, obs)
    xh, lph, xd, lpd = _pair(lambda: api.Problem.from_workload(wl, obs, checkpoint_stride=1, fast_math=fast),
                             lambda: api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr), x, iters)
    np.testing.assert_array_equal(xh, xd)
    np.testing.assert_array_equal(lph, lpd)


def test_host_iterations_of_the_arm_box_and_of_constrained_svgd():
    import test_gpu_armbox as ta
    wl, obs, _, x, _ = ta._setup(N=96, T=120, W=4)
    xh, lph, xd, lpd = _pair(lambda: api.Problem.armbox(wl, obs),
                             lambda: api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr), x, 2)
    np.testing.assert_array_equal(xh, xd)
    np.testing.assert_array_equal(lph, lpd)

    wl = f32_workload(wlmod.double_pendulum(N=80))
    obs = observations(wl)
    x = particles(wl, obs)
    xa = np.concatenate([x, np.zeros((x.shape[0], wl.W - 1 + wl.M))], 1)

    def prob():
        p = api.Problem.from_workload(wl, obs)
        p.set_csvgd(True, 1.0)
        return p

    def svgd():
        s = api.Svgd(wl.N, wl.M, xa.shape[1], wl.lo, wl.hi, lr=wl.lr)
        s.set_csvgd(wl.W - 1)
        return s

    xh, lph, xd, lpd = _pair(prob, svgd, xa, 2)
    np.testing.assert_array_equal(xh, xd)
    np.testing.assert_array_equal(lph, lpd)
