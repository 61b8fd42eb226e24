"""GPU parity of the SGLD chains (Welling and Teh 2011, the second estimator
of Sec. V-B's multiple-shooting comparison) against the FP64 oracle, through
the C ABI.

Covers:
  * the counter-based noise: with eps = 1, zero gradient and zero start the
    step writes the generator's normals, compared element by element with the
    oracle's draws (fp32 Box-Muller against fp64: |dxi| <= 5e-6, the
    float rounding of u2 times the largest radius sqrt(-2 ln 2^-53) = 8.6);
  * several steps of the update with theta rows in unit-box coordinates
    (clipped, and not clipped), shooting rows, a polynomially decaying step
    and a ragged particle count;
  * reset repeats the draws; other seeds give other draws;
  * the chains sample a Gaussian target with the variance that constant-step
    SGLD has in closed form (an AR(1) chain: s^2 / (1 - eps / (4 s^2)));
  * two steps on the double pendulum with the GPU likelihood gradient against
    the oracle's chain with the oracle's gradient.
"""
import numpy as np
import pytest
import torch

from helpers import f32_workload, observations, oracle_problem, particles
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu

XI_ATOL = 5e-6


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("N,P", [(1, 1), (1000, 3), (4099, 2)])
def test_noise_matches_oracle(N, P):
    seed = 0x1234_5678_9ABC_DEF0
    x = torch.zeros((P, N), device="cuda")
    g = torch.zeros_like(x)
    sg = api.Sgld(N, 0, P, [], [], a=1.0, b=0.0, gamma=0.0, seed=seed, clamp=False)
    ref = np.zeros(P * N)
    for t in range(1, 3):
        assert sg.step(x, g) == 1.0
        ref += np.array([orc.langevin_normal(seed, (t - 1) * P * N + k) for k in range(P * N)])
        got = x.cpu().numpy().reshape(-1).astype(np.float64)
        err = np.abs(got - ref)
        assert err.max() <= t * XI_ATOL, f"step {t}: max |dxi| {err.max():.2e} at {int(err.argmax())}"
    sg.close()
    if N * P >= 1000:
        z = ref / np.sqrt(2.0)
        assert abs(z.mean()) < 0.1 and abs(z.std() - 1.0) < 0.1


def _box_case(N, M, S, seed):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-2.0, 1.0, M).astype(np.float32).astype(np.float64)
    hi = (lo + rng.uniform(0.5, 3.0, M)).astype(np.float32).astype(np.float64)
    th = lo + (hi - lo) * rng.uniform(0.0, 1.0, (N, M))
    th[: min(N, 5), 0] = hi[0] - 1e-3 * (hi[0] - lo[0])  # near the upper bound: clipped by the step
    th[5:10, 0] = lo[0]
    x = np.concatenate([th, rng.normal(size=(N, S))], axis=1)
    return lo, hi, x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("clamp", [True, False])
@pytest.mark.parametrize("N,M,S", [(1000, 3, 7), (257, 1, 0), (64, 16, 40)])
def test_steps_match_oracle(N, M, S, clamp):
    P = M + S
    lo, hi, x = _box_case(N, M, S, seed=N + M)
    a, b, gamma, seed = 4e-3, 1.0, 0.55, 77
    sg = api.Sgld(N, M, P, lo, hi, a=a, b=b, gamma=gamma, seed=seed, clamp=clamp)
    ost = orc.SgldState(N, P, lo, hi, a=a, b=b, gamma=gamma, seed=seed, clamp=clamp)
    X = _dev(x.T)
    xr = np.ascontiguousarray(x.copy())
    w = np.concatenate([hi - lo, np.ones(S)])
    rng = np.random.default_rng(3)
    tol = np.zeros(P)
    for t in range(1, 6):
        g = (rng.normal(size=(N, P)) * 30.0).astype(np.float32).astype(np.float64)
        g[:5, 0] = 1e4  # drives the near-bound particles out of the box
        eps = sg.step(X, _dev(g.T))
        ost.step(xr, g)
        eps_ref = a * (b + t) ** -gamma
        assert abs(eps - eps_ref) <= 1e-6 * eps_ref
        # per-step error: fp32 rounding of the unit-box round trip and of the
        # drift, and the generator's fp32 error scaled by sqrt(eps)
        tol = tol + 4e-7 * (np.abs(xr).max(axis=0) + w) + XI_ATOL * np.sqrt(eps_ref) + 1e-7 * eps_ref * 1e4 * w
        got = X.cpu().numpy().T.astype(np.float64)
        err = np.abs(got - xr).max(axis=0)
        assert np.all(err <= tol), f"step {t}: row errors {err} above {tol}"
    if clamp:
        slack = 1e-6 * (np.abs(lo) + np.abs(hi))
        assert np.all(got[:, :M] >= lo - slack) and np.all(got[:, :M] <= hi + slack)
        assert np.all(np.abs(got[:5, 0] - hi[0]) <= slack[0])
    else:
        assert np.any(got[:5, 0] > hi[0])
    sg.close()


def test_reset_repeats_draws_and_seeds_differ():
    N, P = 300, 4
    x0 = np.random.default_rng(1).normal(size=(P, N))
    g = _dev(np.zeros((P, N)))
    out = []
    for seed in (5, 5, 6):
        sg = api.Sgld(N, 0, P, [], [], a=1e-2, seed=seed, clamp=False)
        X = _dev(x0)
        sg.step(X, g)
        out.append(X.cpu().numpy())
        sg.reset()
        X2 = _dev(x0)
        sg.step(X2, g)
        assert np.array_equal(X2.cpu().numpy(), out[-1])
        sg.close()
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])


def test_chains_sample_gaussian_target():
    # constant step: x' = x + (eps/2)(-(x - mu)/s^2) + sqrt(eps) xi is AR(1)
    # with coefficient 1 - eps/(2 s^2); its stationary variance is
    # s^2 / (1 - eps / (4 s^2)).
    N, P, eps = 16384, 2, 2e-2
    mu = torch.tensor([1.0, -2.0], device="cuda").reshape(P, 1)
    s = torch.tensor([0.5, 1.5], device="cuda").reshape(P, 1)
    X = mu.expand(P, N).contiguous()
    G = torch.empty_like(X)
    sg = api.Sgld(N, 0, P, [], [], a=eps, b=0.0, gamma=0.0, seed=11, clamp=False)
    snaps = []
    for it in range(3000):
        torch.sub(X, mu, out=G)
        G.div_(-(s * s))
        sg.step(X, G)
        if it >= 1500 and it % 50 == 0:
            snaps.append(X.clone())
    smp = torch.cat(snaps, dim=1).cpu().numpy().astype(np.float64)
    sv = s.cpu().numpy().reshape(-1)
    var_ref = sv ** 2 / (1.0 - eps / (4.0 * sv ** 2))
    assert np.all(np.abs(smp.mean(axis=1) - mu.cpu().numpy().reshape(-1)) < 0.02 * sv)
    ratio = smp.var(axis=1) / var_ref
    assert np.all(np.abs(ratio - 1.0) < 0.03), ratio
    sg.close()


def test_two_steps_with_likelihood_gradient_match_oracle():
    wl = f32_workload(wlmod.double_pendulum(N=64, seed=1000))
    obs = observations(wl)
    x = particles(wl, obs, seed=3)[:64].copy()
    x = np.ascontiguousarray(x.astype(np.float32).astype(np.float64))
    N, P, M = x.shape[0], x.shape[1], wl.M
    prob = api.Problem.from_workload(wl, obs)
    oprob = oracle_problem(wl, obs)
    a, b, gamma, seed = 1e-6, 1.0, 0.55, 2024
    sg = api.Sgld(N, M, P, wl.lo, wl.hi, a=a, b=b, gamma=gamma, seed=seed)
    ost = orc.SgldState(N, P, wl.lo, wl.hi, a=a, b=b, gamma=gamma, seed=seed)
    X = _dev(x.T)
    xr = x.copy()
    for _ in range(2):
        x_prev = xr.copy()
        _, G, _ = prob.loglik_grad(X)
        _, g_ref = oprob.loglik_grad(xr)
        sg.step(X, G)
        ost.step(xr, g_ref)
        got = X.cpu().numpy().T.astype(np.float64)
        for blk in (slice(0, M), slice(M, P)):
            move = np.abs(xr[:, blk] - x_prev[:, blk]).max(axis=1)
            err = np.abs(got[:, blk] - xr[:, blk]).max(axis=1)
            scale = np.abs(xr[:, blk]).max(axis=1)
            assert np.all(err <= 5e-3 * move + 2e-6 * (1.0 + scale)), (blk, err.max(), move.min())
    assert np.all(np.isfinite(got))
    sg.close()
    prob.close()


def test_sgld_rejects_bad_arguments():
    with pytest.raises(api.PdsError):
        api.Sgld(0, 0, 1, [], [])
    with pytest.raises(api.PdsError):
        api.Sgld(10, 1, 2, [1.0], [1.0])  # empty box
    with pytest.raises(api.PdsError):
        api.Sgld(10, 0, 2, [], [], a=0.0)
    with pytest.raises(api.PdsError):
        api.Sgld(10, 2, 1, [0.0, 0.0], [1.0, 1.0])  # P < M
