"""Posterior-level parity of Algorithm 1 on the GPU against the FP64 oracle.

Every test starts the GPU and the oracle from the same FP32-representable
particles of a seeded workload and compares what the iterations produce:

* Along the GPU's own trajectory (10 iterations of the double pendulum of
  Sec. V-A's setting), every step's log p, gradient, bandwidth and phi
  against the oracle evaluated at the GPU's particles, and the GPU's Adam
  update against the oracle's update driven by the GPU's own directions
  (Algorithm 1).  This checks every component of every step element by
  element without letting an FP32 rounding difference grow over the run.
* Independent runs (pds_iterate against the oracle's own loop) after 1 and
  10 iterations, element by element: Adam's first step moves an entry by
  lr * sign(direction), so an entry may differ by up to 2 lr only where the
  oracle's direction lies within its parity tolerance of zero (there the
  FP32 direction may take the other sign); every other entry agrees within
  the bound the direction tolerances give.
* 100 iterations (the configuration's run length): per-dimension means and
  covariances of theta within relative 5e-2, and a two-sample permutation
  test on the unbiased MMD^2 that finds no difference between the GPU's and
  the oracle's particle sets.  Run with the tensor-core passes (N >= 256 for
  phi, N >= 2048 for the median's distances) and on the CUDA cores.
* The arm-shaking-a-box system of Sec. V-C (reduced to the oracle's budget):
  its posterior is symmetric under swapping the two weights, so particles
  are compared after ordering each one's weights by x, on the fraction that
  needed the swap (the mode each particle settled in) and the moments.
* The benchmark's own system (the 5-link damped chain with the fast-math
  rollout) and the 11-parameter rigid double pendulum: theta's moments and
  the MMD^2 test after 20-25 iterations.
* The linear-Gaussian toy (a target with a closed-form posterior) through
  pds_svgd_step on the device: the mean within 0.05 sigma, the covariance
  within 10 % (the oracle pin of the same toy, now on the GPU), and the
  GPU's particle set against the oracle's run from the same start.
"""
import numpy as np
import pytest
import torch

from helpers import (GRAD_RTOL, LOGP_RTOL, PHI_TOL, assert_grad_close, assert_logp_close, f32_workload,
                     grad_tolerance, observations, oracle_problem, particles)
from oracle import metrics_oracle as mo
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu

THREADS = 16


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _host(t):
    return t.cpu().numpy().T.astype(np.float64)


def _c0(N, seed=1000):
    wl = f32_workload(wlmod.double_pendulum(N=N, seed=seed))
    obs = observations(wl)
    return wl, obs, oracle_problem(wl, obs), particles(wl, obs)


def _svgd(wl, cuda_cores):
    sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr)
    sv.set_option(api.OPT_PHI_CUDA_CORES, int(cuda_cores))
    sv.set_option(api.OPT_MEDIAN_CUDA_CORES, int(cuda_cores))
    return sv


def _width(wl):
    return np.concatenate([wl.hi - wl.lo, np.ones(wl.P - wl.M)])


# Adam's FP32 update of an entry (x + lr m^/(sqrt v^ + eps), with u = (theta - lo)/w
# and back for theta rows) against the FP64 update given the same directions:
# rounding of x (2^-24 |x| twice) and of the step (a few ulp of lr).
def _update_tol(x, width):
    return 4e-7 * (np.abs(x) + width)


@pytest.mark.parametrize("N,cuda_cores", [(100, True), (512, False)])
def test_ten_iterations_along_the_gpu_trajectory(N, cuda_cores):
    wl, obs, op, x = _c0(N)
    prob = api.Problem.from_workload(wl, obs)
    sv = _svgd(wl, cuda_cores)
    ost = orc.SvgdState(wl.N, wl.P, wl.lo, wl.hi, lr=wl.lr)
    X = _gpu(x)
    width = _width(wl)
    for it in range(10):
        xk = _host(X)
        logp, G, status = prob.loglik_grad(X)
        bw, phi = sv.step(X, G, return_phi=True)
        torch.cuda.synchronize()
        assert int(status.sum()) == 0
        lp_ref, g_ref = op.loglik_grad(xk, threads=THREADS)
        assert_logp_close(logp.cpu().numpy().astype(np.float64), lp_ref)
        g = _host(G)
        assert_grad_close(g, g_ref, wl.M)
        # bandwidth and phi of the oracle at the GPU's particles and gradient
        u = (xk[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
        bw_ref = orc.bandwidth(N, orc.median_sqdist(u))
        assert abs(bw.item() - bw_ref) <= 1e-5 * bw_ref, (it, bw.item(), bw_ref)
        phi_ref = orc.svgd_phi(u, g[:, :wl.M] * (wl.hi - wl.lo), bw_ref)
        ph = _host(phi)
        assert np.max(np.abs(ph - phi_ref)) <= PHI_TOL * np.max(np.abs(phi_ref)), (it, np.max(np.abs(ph - phi_ref)))
        # the update: the oracle's Adam driven by the GPU's own directions
        xo = np.ascontiguousarray(xk.copy())
        ost.update(xo, ph, g)
        xg = _host(X)
        err = np.abs(xg - xo)
        assert np.all(err <= _update_tol(xo, width)), (it, np.max(err / _update_tol(xo, width)))
    sv.close()
    prob.close()


def _independent(wl, op, x, iters, cuda_cores, prob):
    """pds_iterate and the oracle's own loop from the same particles; returns
    both particle sets and, per entry, whether the oracle's direction came
    within its parity tolerance of zero at some step."""
    sv = _svgd(wl, cuda_cores)
    X = _gpu(x)
    api.iterate(prob, sv, X, iters)
    torch.cuda.synchronize()
    ost = orc.SvgdState(wl.N, wl.P, wl.lo, wl.hi, lr=wl.lr)
    xo = np.ascontiguousarray(x.copy())
    near0 = np.zeros(x.shape, dtype=bool)
    for _ in range(iters):
        _, g_ref = op.loglik_grad(xo, threads=THREADS)
        phi_ref, _ = ost.step(xo, g_ref)
        near0[:, :wl.M] |= np.abs(phi_ref) <= PHI_TOL * np.max(np.abs(phi_ref))
        near0[:, wl.M:] |= np.abs(g_ref[:, wl.M:]) <= grad_tolerance(g_ref, wl.M)[:, wl.M:]
    xg = _host(X)
    sv.close()
    return xg, xo, near0


@pytest.mark.parametrize("iters", [1, 10])
def test_independent_runs_agree_entry_by_entry(iters):
    wl, obs, op, x = _c0(100)
    prob = api.Problem.from_workload(wl, obs)
    xg, xo, near0 = _independent(wl, op, x, iters, True, prob)
    prob.close()
    width = _width(wl)
    # each step of an entry whose direction keeps its sign moves by lr times
    # m^/sqrt(v^), which a relative direction error e changes by at most 2e:
    # 2 lr e per step, e the gradient tolerance (phi's is tighter)
    bound = iters * (2 * wl.lr * GRAD_RTOL + 1e-6) * width
    d = np.abs(xg - xo)
    ok = d <= bound
    assert np.all(ok | near0), (np.max((d / bound)[~near0]), int(np.sum(~ok)))
    assert np.all(d[near0] <= 2.5 * wl.lr * iters * width[np.nonzero(near0)[1]])
    assert np.mean(near0) < 0.01


def _moments_agree(a, b, rel=5e-2):
    mu_a, mu_b = a.mean(0), b.mean(0)
    assert np.all(np.abs(mu_a - mu_b) <= rel * np.abs(mu_b)), (mu_a, mu_b)
    ca, cb = np.cov(a.T), np.cov(b.T)
    sd = np.sqrt(np.diag(cb))
    assert np.all(np.abs(ca - cb) <= rel * np.outer(sd, sd)), (ca, cb)


def _mmd_permutation_pvalue(a, b, h, perms=200, seed=0):
    obs = mo.mmd2_unbiased(a, b, h)
    pool = np.concatenate([a, b])
    rng = np.random.default_rng(seed)
    null = []
    for _ in range(perms):
        p = rng.permutation(len(pool))
        null.append(mo.mmd2_unbiased(pool[p[:len(a)]], pool[p[len(a):]], h))
    return obs, float(np.mean(np.asarray(null) >= obs))


@pytest.mark.slow
@pytest.mark.parametrize("N,iters,cuda_cores", [(100, 100, True), (512, 100, False), (512, 100, True),
                                                 (2048, 25, False)])
def test_posterior_moments_and_mmd(N, iters, cuda_cores):
    """N = 100 is the configuration's own particle count (CUDA-core passes);
    N = 512 takes phi on the tensor cores or the CUDA cores; N = 2048 adds
    the median's tensor-core distances (fewer iterations: the oracle's
    budget)."""
    wl, obs, op, x = _c0(N)
    prob = api.Problem.from_workload(wl, obs)
    xg, xo, _ = _independent(wl, op, x, iters, cuda_cores, prob)
    prob.close()
    ug = (xg[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    uo = (xo[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    assert np.all(np.isfinite(ug))
    _moments_agree(xg[:, :wl.M], xo[:, :wl.M])
    # MMD^2 between the sets with the median-heuristic bandwidth of the oracle's set
    h = orc.median_sqdist(uo)
    m2, p = _mmd_permutation_pvalue(ug, uo, h)
    assert p > 0.05, (m2, p)
    # the run moved the particles: the initial set is far from both
    u0 = (x[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    assert mo.mmd2_unbiased(u0, uo, h) > 10 * abs(m2)


def _armbox(N, T, W, seed=3000):
    wl = wlmod.arm_box(N=N, seed=seed, T=T, W=W)
    for name in ("arm_len", "amp", "freq", "phase", "lo", "hi", "s0", "theta_true", "theta_init"):
        setattr(wl, name, getattr(wl, name).astype(np.float32).astype(np.float64))
    wl.dt = float(np.float32(wl.dt))
    ab = orc.ArmBox.from_workload(wl)
    st = ab.simulate(wl.theta_true, wl.dt, wl.T, wl.s0)
    obs = (st[1:, wl.obs_index] + wl.sigma_obs * wl.noise[:wl.T]).astype(np.float32)
    op = orc.ArmBoxProblem(ab, dt=wl.dt, T=wl.T, W=wl.W, obs=obs.astype(np.float64), obs_index=wl.obs_index,
                           sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo, hi=wl.hi,
                           c_lim=wl.c_lim)
    shoot = st[[wl.window_start(w) for w in range(1, wl.W)]].ravel()
    x = np.concatenate([wl.theta_init, np.tile(shoot, (wl.N, 1))], 1)
    return wl, obs, op, x.astype(np.float32).astype(np.float64)


def _canonical(th):
    """Order each particle's two weights by x (the posterior is symmetric
    under swapping them); returns the ordered set and which were swapped."""
    sw = th[:, 0] > th[:, 2]
    c = th.copy()
    c[sw] = th[sw][:, [2, 3, 0, 1]]
    return c, sw


@pytest.mark.slow
def test_arm_box_symmetric_posterior_modes():
    wl, obs, op, x = _armbox(N=256, T=400, W=8)
    iters = 30
    prob = api.Problem.armbox(wl, obs)
    sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr)
    X = _gpu(x)
    api.iterate(prob, sv, X, iters)
    torch.cuda.synchronize()
    xg = _host(X)
    ost = orc.SvgdState(wl.N, wl.P, wl.lo, wl.hi, lr=wl.lr)
    xo = np.ascontiguousarray(x.copy())
    for _ in range(iters):
        _, g_ref = op.loglik_grad(xo, threads=THREADS)
        ost.step(xo, g_ref)
    cg, swg = _canonical(xg[:, :4])
    co, swo = _canonical(xo[:, :4])
    # the mode each particle settled in: the same but for particles near the
    # boundary between the modes
    assert np.mean(swg != swo) <= 0.02, np.mean(swg != swo)
    assert abs(np.mean(swg) - np.mean(swo)) <= 0.02
    # both modes are populated (the posterior is multimodal)
    assert 0.1 < np.mean(swo) < 0.9
    mu_g, mu_o = cg.mean(0), co.mean(0)
    sd = np.sqrt(np.diag(np.cov(co.T)))
    assert np.all(np.abs(mu_g - mu_o) <= 5e-2 * sd + 1e-3 * (wl.hi - wl.lo)), (mu_g, mu_o, sd)
    assert np.all(np.abs(np.sqrt(np.diag(np.cov(cg.T))) - sd) <= 5e-2 * sd + 1e-3 * (wl.hi - wl.lo))
    sv.close()
    prob.close()


def test_linear_gaussian_toy_on_the_gpu():
    """d log N(x | mu, Sigma)/dx = -Sigma^-1 (x - mu) written by the test on
    the device; the SVGD updates through pds_svgd_step (tensor-core phi at
    N = 1000)."""
    mu = np.array([0.3, -0.2])
    Sig = np.array([[0.04, 0.018], [0.018, 0.025]])
    Prec = torch.tensor(np.linalg.inv(Sig), dtype=torch.float32, device="cuda")
    mu_t = torch.tensor(mu, dtype=torch.float32, device="cuda")[:, None]
    lo, hi = np.array([-2.0, -2.0]), np.array([2.0, 2.0])
    for N, iters in ((1000, 2000), (400, 1500)):
        rng = np.random.default_rng(42)
        x0 = rng.uniform(-1.0, 1.0, size=(N, 2)).astype(np.float32).astype(np.float64)
        sv = api.Svgd(N, 2, 2, lo, hi, lr=2e-2, clamp=False)
        X = _gpu(x0)
        for _ in range(iters):
            G = -(Prec @ (X - mu_t))
            sv.step(X, G.contiguous())
        torch.cuda.synchronize()
        xg = _host(X)
        sv.close()
        sd = np.sqrt(np.diag(Sig))
        assert np.all(np.abs(xg.mean(0) - mu) < 0.05 * sd), xg.mean(0)
        C = np.cov(xg.T)
        assert np.all(np.abs(np.diag(C) - np.diag(Sig)) < 0.1 * np.diag(Sig)), C
        assert abs(C[0, 1] - Sig[0, 1]) < 0.1 * np.sqrt(Sig[0, 0] * Sig[1, 1])
        if N == 400:
            # the oracle's run of the same toy from the same start
            xo = np.ascontiguousarray(x0.copy())
            st = orc.SvgdState(N, 2, lo, hi, lr=2e-2, clamp=False)
            Pr = np.linalg.inv(Sig)
            for _ in range(iters):
                st.step(xo, -(xo - mu) @ Pr)
            _moments_agree(xg, xo)


def _run_both(prob, op, wl, x, iters, threads=THREADS):
    """pds_iterate on the GPU and the oracle's own loop from the same particles."""
    sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr)
    X = _gpu(x)
    api.iterate(prob, sv, X, iters)
    torch.cuda.synchronize()
    xg = _host(X)
    sv.close()
    ost = orc.SvgdState(wl.N, wl.P, wl.lo, wl.hi, lr=wl.lr)
    xo = np.ascontiguousarray(x.copy())
    for _ in range(iters):
        _, g_ref = op.loglik_grad(xo, threads=threads)
        ost.step(xo, g_ref)
    return xg, xo


@pytest.mark.slow
def test_chain5_posterior_with_fast_math():
    """The benchmark's system (5-link damped chain, theta = 5 masses + 5
    dampings, T = 1000 at dt = 0.005, 20 windows, angles and velocities
    observed) with the benchmark's fast-math rollout, N = 256 for 20
    iterations: theta's moments and the MMD^2 two-sample test against the
    oracle run from the same particles."""
    wl = f32_workload(wlmod.chain5(N=256))
    obs = observations(wl)
    x = particles(wl, obs)
    op = oracle_problem(wl, obs)
    prob = api.Problem.from_workload(wl, obs, checkpoint_stride=1, fast_math=1)
    xg, xo = _run_both(prob, op, wl, x, 20)
    prob.close()
    assert np.all(np.isfinite(xg)) and np.all(np.isfinite(xo))
    _moments_agree(xg[:, :wl.M], xo[:, :wl.M])
    ug = (xg[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    uo = (xo[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    h = orc.median_sqdist(uo)
    m2, p = _mmd_permutation_pvalue(ug, uo, h)
    assert p > 0.05, (m2, p)
    # the shooting states too: per-dimension means within 5e-2 of their spread
    sd = np.std(xo[:, wl.M:], axis=0) + 1e-3
    assert np.all(np.abs(xg[:, wl.M:].mean(0) - xo[:, wl.M:].mean(0)) <= 5e-2 * sd)


@pytest.mark.slow
def test_rigid_double_pendulum_posterior():
    """The 11-parameter rigid double pendulum (N = 128, T = 200, W = 5),
    25 iterations: the same comparison of theta's moments and MMD^2."""
    import test_gpu_rigid2 as tr
    wl, obs = tr._workload(N=128, T=200, W=5)
    x = tr._particles(wl, obs)
    op = tr._oracle(wl, obs)
    prob = api.Problem.from_workload(wl, obs)
    xg, xo = _run_both(prob, op, wl, x, 25)
    prob.close()
    assert np.all(np.isfinite(xg))
    _moments_agree(xg[:, :wl.M], xo[:, :wl.M])
    ug = (xg[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    uo = (xo[:, :wl.M] - wl.lo) / (wl.hi - wl.lo)
    m2, p = _mmd_permutation_pvalue(ug, uo, orc.median_sqdist(uo))
    assert p > 0.05, (m2, p)
