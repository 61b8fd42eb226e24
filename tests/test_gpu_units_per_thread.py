"""Two rollout units per thread (PDS_OPT_UNITS_PER_THREAD).

The two-unit kernel steps particles i and i + 1 of a window together, each
quantity held as a float2, so that the step's FP32 arithmetic (Appendix B-A's
forward dynamics, semi-implicit Euler, the observation and defect terms of
Eqs. 2, 4, 5 and the adjoint) issues as paired instructions.  Each pair
component rounds exactly as the one-unit kernel's scalar operation, so:

  * forcing one or two units per thread gives the same log p and gradient
    bit for bit, for 1..8 links, both math modes, windows of uneven length
    and sets of two trajectories;
  * the two-unit result also matches the FP64 oracle within the tolerances
    of the other parity tests;
  * where two units do not apply (an odd particle count, K > 1, a partial
    observation set) the option falls back to one unit per thread with the
    same results;
  * the option rejects values outside 0..2.
"""
import numpy as np
import pytest
import torch

from helpers import (assert_grad_close, assert_logp_close, f32_workload, logp_constant, observations, oracle_problem,
                     particles)
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _run(wl, obs, x, upt, fast, K=1, R=1):
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=K, fast_math=fast)
    prob.set_option(api.OPT_UNITS_PER_THREAD, upt)
    assert prob.get_option(api.OPT_UNITS_PER_THREAD) == upt
    if R > 1:
        # the second trajectory: the same observations with a small offset
        obs2 = np.stack([obs, obs + np.float32(0.01)]).astype(np.float32)
        s02 = np.stack([wl.s0, wl.s0]).astype(np.float32)
        prob.set_trajectories(obs2, s02, "sum")
        x = np.concatenate([x, x[:, wl.M:]], axis=1)
    logp, g, status = prob.loglik_grad(_gpu(x))
    torch.cuda.synchronize()
    out = logp.cpu().numpy(), g.cpu().numpy(), status.cpu().numpy()
    prob.close()
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("fast", [0, 1])
def test_two_units_per_thread_are_bit_identical_to_one(n, fast):
    # T / W not an integer: windows differ in length by one step
    # at most 16 estimated parameters: longer chains estimate masses and dampings
    kinds = (wlmod.PARAM_MASS, wlmod.PARAM_LENGTH, wlmod.PARAM_DAMPING) if n <= 5 else (wlmod.PARAM_MASS, wlmod.PARAM_DAMPING)
    wl = f32_workload(wlmod.random_chain(n, 258, seed=300 + n, T=47, W=5, kinds=kinds))
    obs = observations(wl)
    x = particles(wl, obs)
    lp1, g1, st1 = _run(wl, obs, x, 1, fast)
    lp2, g2, st2 = _run(wl, obs, x, 2, fast)
    assert np.all(st1 == 0) and np.all(st2 == 0)
    assert np.array_equal(lp1, lp2)
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_without_length_parameters_both_kernels_match_the_oracle(n):
    # masses and dampings only: the adjoint step leaves out the length
    # adjoint (the kernels specialised for it, fast math, K = 1)
    wl = f32_workload(wlmod.random_chain(n, 130, seed=330 + n, T=47, W=5,
                                         kinds=(wlmod.PARAM_MASS, wlmod.PARAM_DAMPING)))
    assert not np.any(wl.theta_kind == wlmod.PARAM_LENGTH)
    obs = observations(wl)
    x = particles(wl, obs)
    lp1, g1, st1 = _run(wl, obs, x, 1, 1)
    lp2, g2, st2 = _run(wl, obs, x, 2, 1)
    assert np.all(st1 == 0) and np.all(st2 == 0)
    assert np.array_equal(lp1, lp2)
    assert np.array_equal(g1, g2)
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x.astype(np.float32).astype(np.float64))
    # some of these 130 random particles have log p near zero (their residual
    # terms cancel the normalising constants): log p is compared relative to
    # the larger of |log p| and the constants' sum
    assert_logp_close(lp1.astype(np.float64), lp_ref, const=logp_constant(wl))
    assert_grad_close(g1.T.astype(np.float64), g_ref, wl.M)


@pytest.mark.parametrize("fast", [0, 1])
def test_two_units_per_thread_match_the_oracle(fast):
    wl = f32_workload(wlmod.random_chain(5, 130, seed=311, T=60, W=6))
    obs = observations(wl)
    x = particles(wl, obs)
    lp, g, st = _run(wl, obs, x, 2, fast)
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x.astype(np.float32).astype(np.float64))
    assert np.all(st == 0)
    assert_logp_close(lp.astype(np.float64), lp_ref)
    assert_grad_close(g.T.astype(np.float64), g_ref, wl.M)


def test_two_units_per_thread_with_two_trajectories():
    wl = f32_workload(wlmod.random_chain(4, 66, seed=312, T=40, W=4))
    obs = observations(wl)
    x = particles(wl, obs)
    lp1, g1, _ = _run(wl, obs, x, 1, 1, R=2)
    lp2, g2, _ = _run(wl, obs, x, 2, 1, R=2)
    assert np.array_equal(lp1, lp2)
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("case", ["odd_N", "K4", "partial_obs"])
def test_where_two_units_do_not_apply_the_results_are_unchanged(case):
    N = 131 if case == "odd_N" else 130
    wl = f32_workload(wlmod.random_chain(5, N, seed=313, T=40, W=4, observe_velocity=(case != "partial_obs")))
    K = 4 if case == "K4" else 1
    obs = observations(wl)
    x = particles(wl, obs)
    lp1, g1, _ = _run(wl, obs, x, 1, 1, K=K)
    lp2, g2, _ = _run(wl, obs, x, 2, 1, K=K)
    assert np.array_equal(lp1, lp2)
    assert np.array_equal(g1, g2)


def test_units_per_thread_option_range():
    wl = f32_workload(wlmod.random_chain(2, 8, seed=314, T=10, W=2))
    prob = api.Problem.from_workload(wl, observations(wl))
    assert prob.get_option(api.OPT_UNITS_PER_THREAD) == 0
    for bad in (-1, 3):
        with pytest.raises(api.PdsError):
            prob.set_option(api.OPT_UNITS_PER_THREAD, bad)
    prob.close()


def test_autotuner_keeps_the_fastest_valid_choice():
    """pds_problem_autotune times the candidate launches, sets the fastest
    (units per thread, K), and the likelihood it then computes still matches
    the FP64 oracle."""
    wl = f32_workload(wlmod.random_chain(5, 256, seed=315, T=100, W=4))
    obs = observations(wl)
    x = particles(wl, obs)
    prob = api.Problem.from_workload(wl, obs, fast_math=1)
    X = _gpu(x)
    ch = prob.autotune(X)
    assert ch["units_per_thread"] in (1, 2)
    assert ch["K"] in (1, 5, 10, 25, 50)
    assert ch["K"] == 1 or ch["units_per_thread"] == 1
    assert ch["us_per_call"] > 0
    assert prob.get_option(api.OPT_UNITS_PER_THREAD) == ch["units_per_thread"]
    assert prob.get_option(api.OPT_CHECKPOINT_STRIDE) == ch["K"]
    lp, g, st = prob.loglik_grad(X)
    torch.cuda.synchronize()
    lp_ref, g_ref = oracle_problem(wl, obs).loglik_grad(x.astype(np.float32).astype(np.float64))
    assert np.all(st.cpu().numpy() == 0)
    assert_logp_close(lp.cpu().numpy().astype(np.float64), lp_ref)
    assert_grad_close(g.cpu().numpy().T.astype(np.float64), g_ref, wl.M)
    prob.close()
