"""The paper's single- versus multiple-shooting landscape (Fig. 2), on the
device: the log-likelihood of a double pendulum's link lengths on a 40 x 40
grid (400 steps; the multiple-shooting variant with 10 windows and shooting
states on the true trajectory).  Single shooting is rugged (several local
maxima); multiple shooting keeps one maximum; both peak at the true
lengths."""
import dataclasses

import numpy as np
import pytest
import torch

from helpers import physical
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _landscape(wl, obs, states, W, grid):
    w2 = dataclasses.replace(wl, W=W)
    prob = api.Problem.from_workload(w2, obs)
    shoot = [states[(w * wl.T) // W] for w in range(1, W)]
    x = np.concatenate([grid] + [np.tile(s, (len(grid), 1)) for s in shoot], axis=1)
    lp, _, _ = prob.loglik_grad(torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)).cuda(), grad=False)
    torch.cuda.synchronize()
    prob.close()
    return lp.cpu().numpy().astype(np.float64)


def _local_maxima(L):
    c = L[1:-1, 1:-1]
    return int(np.sum((c > L[:-2, 1:-1]) & (c > L[2:, 1:-1]) & (c > L[1:-1, :-2]) & (c > L[1:-1, 2:])))


def test_multiple_shooting_smooths_the_landscape():
    wl0, thetas, _ = wlmod.two_mode_pendulums(N=4)
    T, G = 400, 40
    wl = dataclasses.replace(wl0, T=T, noise=np.random.default_rng(1).standard_normal((T, 2)))
    m, l, b = physical(wl, thetas[0])
    states = orc.simulate(m, l, b, wl.s0, wl.dt, T, g=wl.g)
    obs = (states[1:, wl.obs_index] + wl.sigma_obs * wl.noise).astype(np.float32)
    l1, l2 = np.meshgrid(np.linspace(0.5, 1.5, G), np.linspace(0.5, 1.5, G), indexing="ij")
    grid = np.stack([l1.ravel(), l2.ravel()], axis=1)
    ss = _landscape(wl, obs, states, 1, grid).reshape(G, G)
    ms = _landscape(wl, obs, states, 10, grid).reshape(G, G)
    assert _local_maxima(ss) >= 3, _local_maxima(ss)
    assert _local_maxima(ms) <= 1, _local_maxima(ms)
    step = 1.0 / (G - 1)
    for L in (ss, ms):
        am = np.unravel_index(np.argmax(L), L.shape)
        assert np.all(np.abs(np.array([l1[am], l2[am]]) - thetas[0]) <= 1.5 * step)
