"""Observations in state order (Eq. 2's observation term): the rollout reads
a problem's observations from a copy in state order that the library builds
from the [T][D] rows and obs_index. A problem that observes every state
component reads it with no per-component lookup.

Covers:
  * observation columns given in any order yield the same log p and
    gradient, bit for bit (the state-ordered copy is the same);
  * a partial, unordered observation set (velocities before angles,
    components skipped) matches the FP64 oracle;
  * both math modes and checkpoint strides 1 and 4.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import assert_grad_close, assert_logp_close, f32_workload, observations, oracle_problem, particles
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _run(wl, obs, x, K, fast):
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=K, fast_math=fast)
    logp, g, status = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    out = logp.cpu().numpy(), g.cpu().numpy(), status.cpu().numpy()
    prob.close()
    return out


@pytest.mark.parametrize("fast,K", [(0, 1), (1, 1), (1, 4)])
def test_permuted_observation_columns_are_bit_identical(fast, K):
    wl = f32_workload(wlmod.random_chain(3, 200, seed=61, T=48, W=4))
    assert list(wl.obs_index) == list(range(6))
    obs = observations(wl)
    x = particles(wl, obs)
    lp0, g0, st0 = _run(wl, obs, x, K, fast)
    perm = np.array([4, 0, 5, 2, 1, 3])
    wl2 = copy.copy(wl)
    wl2.obs_index = np.ascontiguousarray(wl.obs_index[perm]).astype(np.int32)
    lp1, g1, st1 = _run(wl2, np.ascontiguousarray(obs[:, perm]), x, K, fast)
    assert np.all(st0 == 0) and np.all(st1 == 0)
    assert np.array_equal(lp0, lp1)
    assert np.array_equal(g0, g1)


@pytest.mark.parametrize("fast,K", [(0, 1), (1, 1), (1, 4)])
def test_partial_unordered_observations_match_oracle(fast, K):
    wl = f32_workload(wlmod.random_chain(4, 150, seed=62, T=40, W=4))
    # velocity 1, angles 0, 3, 2 (the shooting states' velocities come from
    # the observed angles' differences)
    idx = np.array([5, 0, 3, 2], dtype=np.int32)
    wl.noise = np.ascontiguousarray(wl.noise[:, idx])  # the noise drawn for those components
    wl.obs_index = idx
    obs = observations(wl)
    x = particles(wl, obs)
    lp, g, st = _run(wl, obs, x, K, fast)
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x, threads=8)
    assert np.all(st == 0)
    assert_logp_close(lp.astype(np.float64), lp_ref)
    assert_grad_close(g.T.astype(np.float64), g_ref, wl.M)
