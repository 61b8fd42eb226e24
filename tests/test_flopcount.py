"""The roofline numerator, counted by executing the step (no GPU).

tests/flopcount.py transcribes the GPU's per-step arithmetic of the planar
chain (forward step with its observation term, reverse step with its
observation seed) on a scalar that counts operations (FMA = 2, add / sub /
mul = 1, sincos and reciprocals on the MUFU not counted).  These tests pin
that transcription to the FP64 oracle -- the forward step equals the
oracle's semi-implicit Euler step of the articulated-body dynamics, and the
reverse step equals central differences of it -- and then check that the
count per particle-step agrees with the closed form that bench.py divides
by the measured time (60n + 3D - 43 forward and 110n + 3D - 54 reverse for
n >= 2; 19 + 3D and 66 + 3D for one link; 9n less in the reverse when no
link length is a parameter), once the 2(n - 1) flops of the
two re-formed products are taken out (qdd_i and mu_i are each formed as one
fused multiply-add of a product's factors; the count credits the product
once).  Operations on values that are zero by construction are not
counted; the parameter adjoints, which the reverse step adds to over a
window's steps, are running sums and count in full.
"""
import numpy as np
import pytest

import flopcount as fc
from oracle import pds_oracle as orc

G = 9.81


def _chain(n, seed):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.3, 2.0, n)
    l = rng.uniform(0.3, 1.2, n)
    b = rng.uniform(0.0, 0.8, n)
    q = rng.uniform(-1.5, 1.5, n)
    v = rng.uniform(-1.0, 1.0, n)
    return m, l, b, q, v


def _S(xs, c):
    return [fc.S(x, c) for x in xs]


def _forward(m, l, b, q, v, dt, c):
    M, L, B = _S(m, c), _S(l, c), _S(b, c)
    IL = [fc.rcp(x) for x in L]
    MG = [x * fc.S(G, c) for x in M]  # loop-invariant: computed once per unit, not per step
    c.flops = 0
    q2, v2 = fc.chain_step(_S(q, c), _S(v, c), M, L, B, IL, MG, fc.S(dt, c))
    return q2, v2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_transcribed_forward_step_equals_the_oracle_step(n):
    m, l, b, q, v = _chain(n, 10 + n)
    dt = 0.005
    c = fc.Counter()
    q2, v2 = _forward(m, l, b, q, v, dt, c)
    ref = orc.step(m, l, b, np.concatenate([q, v]), dt, g=G)
    got = np.array([x.v for x in q2 + v2])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def _reverse(m, l, b, q, v, v2, dt, cq, cv, c, lengths=True, acc=None):
    M, L, B = _S(m, c), _S(l, c), _S(b, c)
    IL = [fc.rcp(x) for x in L]
    # the parameter adjoints are running sums over a window's steps (zero
    # only before its first reverse step, not by construction), like rss
    acc = acc if acc is not None else [[fc.S(0.0, c) for _ in m] for _ in range(3)]
    c.flops = 0
    return fc.chain_step_vjp(_S(q, c), _S(v, c), _S(v2, c), M, L, B, IL, fc.S(G, c), fc.S(dt, c),
                             fc.S(1.0 / dt, c), _S(cq, c), _S(cv, c), *acc, lengths=lengths)


@pytest.mark.parametrize("lengths", [True, False])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_transcribed_reverse_step_equals_central_differences_of_the_oracle(n, lengths):
    m, l, b, q, v = _chain(n, 20 + n)
    dt = 0.005
    rng = np.random.default_rng(30 + n)
    cq, cv = rng.standard_normal(n), rng.standard_normal(n)
    s2 = orc.step(m, l, b, np.concatenate([q, v]), dt, g=G)
    c = fc.Counter()
    acc = [[fc.S(0.0, c) for _ in range(n)] for _ in range(3)]
    qb, vb, mb, lb, bb = _reverse(m, l, b, q, v, s2[n:], dt, cq, cv, c, lengths=lengths, acc=acc)
    if not lengths:
        # the length adjoint is left out: lb comes back as the accumulators passed in
        assert all(x is y for x, y in zip(lb, acc[1]))
    got = np.array([x.v for x in qb + vb + mb + lb + bb])

    def L(m_, l_, b_, q_, v_):
        s = orc.step(m_, l_, b_, np.concatenate([q_, v_]), dt, g=G)
        return float(cq @ s[:n] + cv @ s[n:])

    args = [m, l, b, q, v]
    fd = {}
    h = 1e-6
    for k, name in enumerate(["m", "l", "b", "q", "v"]):
        d = np.zeros(n)
        for i in range(n):
            ap = [a.copy() for a in args]
            am = [a.copy() for a in args]
            ap[k][i] += h
            am[k][i] -= h
            d[i] = (L(*ap) - L(*am)) / (2 * h)
        fd[name] = d
    ref = np.concatenate([fd["q"], fd["v"], fd["m"], fd["l"] if lengths else np.zeros(n), fd["b"]])
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())


@pytest.mark.parametrize("lengths", [True, False])
@pytest.mark.parametrize("n", range(1, 9))
def test_count_per_particle_step_matches_the_roofline_numerator(n, lengths):
    from bench import flops_per_particle_step

    D = 2 * n  # the benchmark observes every state component
    m, l, b, q, v = _chain(n, 40 + n)
    dt = 0.005
    obs = np.random.default_rng(50 + n).standard_normal(D)
    c = fc.Counter()
    # forward: the step, its observation residual, the running sum of residuals
    q2, v2 = _forward(m, l, b, q, v, dt, c)
    acc = fc.obs_residual(_S(obs, c), q2, v2)
    _ = fc.S(1.0, c) + acc  # rss += acc (rss is a running sum, not a structural zero)
    fwd = c.flops
    # reverse: the observation seed at the step's output, then the step's adjoint
    c2 = fc.Counter()
    qb, vb = fc.obs_seed(_S(obs, c2), _S([x.v for x in q2], c2), _S([x.v for x in v2], c2),
                         _S(np.ones(n), c2), _S(np.ones(n), c2), fc.S(1.0, c2))
    seed = c2.flops
    _reverse(m, l, b, q, v, [x.v for x in v2], dt, [x.v for x in qb], [x.v for x in vb], c2, lengths=lengths)
    rev = seed + c2.flops
    fwd_ref, rev_ref = flops_per_particle_step(n, D, lengths=lengths)
    refs = n - 1  # one re-formed product per link after the first, in each direction
    assert fwd - refs == fwd_ref, (n, fwd, fwd_ref)
    assert rev - refs == rev_ref, (n, rev, rev_ref)


def test_benchmark_workload_counts_no_length_adjoint():
    # the benchmark's chain estimates masses and dampings only, so its
    # rollout leaves out the length adjoint and the numerator is 287 + 481
    from bench import flops_per_particle_step
    from paper_2109_08815_gb300 import workloads as wlmod

    wl = wlmod.chain5(N=4)
    assert not np.any(wl.theta_kind == wlmod.PARAM_LENGTH)
    assert flops_per_particle_step(wl.n, wl.D, lengths=False) == (287, 481)
    assert flops_per_particle_step(wl.n, wl.D) == (287, 526)
