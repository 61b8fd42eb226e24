"""The seeded synthetic inputs (the stand-ins for the paper's datasets) have
the shapes, ranges and mix their recipes state, and are reproducible from
their seeds:
  * the 5-link chain benchmark (n = 5, M = 10, T = 1000, W = 20, D = 10,
    P = 200) and the double-pendulum stand-in (n = 2, M = 4, T = 200,
    W = 10, D = 2);
  * the arm-and-box stand-in (M = 4, T = 2000, W = 40, D = 2);
  * 64 uneven problems: n in 2..8, T in 100..2000, W in 5..50 (at most
    T / 2), N in 64..4096, the two parameter types about half each, with
    their dt and observed components;
  * the serving mix (about 10 % arm-and-box jobs at 512 particles) and
    Poisson arrivals with the stated mean gap;
  * windows t_w = floor(w T / W) that cover the trajectory once.
"""
import numpy as np

from paper_2109_08815_gb300 import serve
from paper_2109_08815_gb300 import workloads as wlmod


def _in_box(wl):
    return np.all(wl.theta_init >= wl.lo) and np.all(wl.theta_init <= wl.hi)


def test_benchmark_and_pendulum_shapes():
    wl = wlmod.chain5(N=16384)
    assert (wl.n, wl.M, wl.T, wl.W, wl.D, wl.S, wl.P, wl.N) == (5, 10, 1000, 20, 10, 10, 200, 16384)
    assert list(wl.obs_index) == list(range(10)) and _in_box(wl)
    assert wl.noise.shape == (wl.T, wl.D)
    dp = wlmod.double_pendulum(N=100)
    assert (dp.n, dp.M, dp.T, dp.W, dp.D, dp.N) == (2, 4, 200, 10, 2, 100)
    assert list(dp.obs_index) == [0, 1] and _in_box(dp)
    ab = wlmod.arm_box(N=2048)
    assert (ab.M, ab.T, ab.W, ab.D, ab.N) == (4, 2000, 40, 2, 2048)
    assert np.all(ab.theta_init >= ab.lo) and np.all(ab.theta_init <= ab.hi)


def test_generators_are_reproducible_from_their_seeds():
    a, b = wlmod.chain5(N=64, seed=3), wlmod.chain5(N=64, seed=3)
    assert np.array_equal(a.theta_init, b.theta_init) and np.array_equal(a.noise, b.noise)
    c = wlmod.chain5(N=64, seed=4)
    assert not np.array_equal(a.theta_init, c.theta_init)
    p1 = wlmod.batched_problems(n_jobs=8, seed=4000)
    p2 = wlmod.batched_problems(n_jobs=8, seed=4000)
    for x, y in zip(p1, p2):
        assert (x.n, x.T, x.W, x.N) == (y.n, y.T, y.W, y.N)
        assert np.array_equal(x.theta_init, y.theta_init) and np.array_equal(x.noise, y.noise)
    assert np.array_equal(serve.poisson_arrivals(10, 50.0, 5000), serve.poisson_arrivals(10, 50.0, 5000))


def test_uneven_problems_follow_their_recipe():
    probs = wlmod.batched_problems(n_jobs=64, seed=4000)
    assert len(probs) == 64
    pend = 0
    for wl in probs:
        assert 2 <= wl.n <= 8 and 100 <= wl.T <= 2000 and 64 <= wl.N <= 4096
        assert 5 <= wl.W <= 50 and wl.W <= wl.T // 2
        assert _in_box(wl) and wl.theta_init.shape == (wl.N, 2 * wl.n)
        if wl.name.split("_")[1].startswith("pend"):
            pend += 1
            assert wl.dt == 0.01 and list(wl.obs_index) == list(range(wl.n))
        else:
            assert wl.dt == 0.005 and list(wl.obs_index) == list(range(2 * wl.n))
    # 50/50 types: a binomial(64, 1/2) count stays within 4 standard deviations
    assert abs(pend - 32) <= 16
    # the log-uniform ranges are spread out, not collapsed on one end
    Ns = np.array([wl.N for wl in probs])
    assert Ns.min() < 256 and Ns.max() > 1024


def test_serving_mix_and_arrivals():
    jobs = wlmod.serving_mix(200, seed=5000)
    arm = [j for j in jobs if isinstance(j, wlmod.ArmBoxWorkload)]
    assert 0.03 <= len(arm) / len(jobs) <= 0.2
    assert all(j.N == 512 and j.T == 2000 and j.W == 40 for j in arm)
    t = serve.poisson_arrivals(20000, 50.0, 5000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1 / rate: the sample mean within 3 standard errors
    assert abs(gaps.mean() - 0.02) <= 3 * 0.02 / np.sqrt(len(gaps))


def test_windows_cover_the_trajectory_once():
    for T, W in ((1000, 20), (200, 10), (2000, 40), (137, 9), (5, 5)):
        wl = wlmod.chain5(N=4, T=T, W=W)
        starts = [wl.window_start(w) for w in range(W + 1)]
        assert starts[0] == 0 and starts[-1] == T
        assert all(b > a for a, b in zip(starts, starts[1:]))
        assert sum(b - a for a, b in zip(starts, starts[1:])) == T
