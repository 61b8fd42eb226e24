"""GPU parity of the SVGD step (pds_svgd_step: median-heuristic bandwidth,
Eq. 1's phi, Adam update) against the FP64 oracle, through the C ABI.

Tolerances: bandwidth rel 1e-5 (the median of FP32 distances is within
rounding of the FP64 median); phi within PHI_TOL of the largest |phi| (FP32
sums of N kernel-weighted terms); the update, fed the GPU's own phi and the
gradient, within FP32 rounding of the oracle's Adam (update_tolerance); the
particles of independent runs within 1e-4 of the box width per step, except
theta entries whose phi lies within its tolerance of zero, where FP32 and
FP64 may take opposite signs and Adam's first step lr sign(phi) then differs
by 2 lr.
"""
import numpy as np
import pytest
import torch

from helpers import PHI_TOL, update_tolerance
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)).cuda()


def _case(N, M, P, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-2, 0, M).astype(np.float32).astype(np.float64)
    hi = (lo + rng.uniform(0.5, 3, M)).astype(np.float32).astype(np.float64)
    x = np.zeros((N, P))
    x[:, :M] = lo + (hi - lo) * np.clip(0.5 + spread * (rng.uniform(size=(N, M)) - 0.5), 0, 1)
    x[:, M:] = rng.normal(size=(N, P - M))
    g = rng.normal(size=(N, P)) * rng.uniform(0.1, 10, P)
    return lo, hi, x.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)


def _compare(N, M, P, seed, steps=1, spread=1.0, lr=1e-2, fast=False):
    lo, hi, x, g = _case(N, M, P, seed, spread)
    sv = api.Svgd(N, M, P, lo, hi, lr=lr, fast_math=fast)
    X, G = _gpu(x), _gpu(g)
    ost = orc.SvgdState(N, P, lo, hi, lr=lr)  # independent run
    fed = orc.SvgdState(N, P, lo, hi, lr=lr)  # driven by the GPU's phi
    xo = np.ascontiguousarray(x.copy())
    width = np.concatenate([hi - lo, np.ones(P - M)])
    near0 = np.zeros((N, P), dtype=bool)
    for _ in range(steps):
        xk = X.cpu().numpy().T.astype(np.float64)
        bw, phi = sv.step(X, G, return_phi=True)
        phi_ref, bw_ref = ost.step(xo, g)
        near0[:, :M] |= np.abs(phi_ref) <= PHI_TOL * np.max(np.abs(phi_ref))
        torch.cuda.synchronize()
        ph = phi.cpu().numpy().T.astype(np.float64)
        xf = np.ascontiguousarray(xk)
        fed.update(xf, ph, g)
        xg = X.cpu().numpy().T.astype(np.float64)
        assert np.all(np.abs(xg - xf) <= update_tolerance(xf, width)), \
            np.max(np.abs(xg - xf) / update_tolerance(xf, width))
    # after several steps the two particle sets differ by the rare sign flips
    # below, which moves the median slightly
    assert abs(bw.item() - bw_ref) <= (1e-5 if steps == 1 else 1e-3) * bw_ref, (bw.item(), bw_ref)
    scale = np.max(np.abs(phi_ref))
    if steps == 1:
        assert np.max(np.abs(ph - phi_ref)) <= PHI_TOL * scale, np.max(np.abs(ph - phi_ref)) / scale
    dx = np.abs(xg - xo) / width
    far = ~near0
    assert np.all(dx[far] <= 1e-4 * steps), np.max(dx[far])
    assert np.all(dx <= 2.5 * lr * steps), dx.max()
    assert np.mean(near0) <= 2e-2


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("N,M,P", [(2, 1, 1), (3, 2, 5), (100, 4, 76), (129, 10, 30), (1000, 7, 7), (257, 16, 40),
                                   (600, 3, 9), (1031, 9, 9), (700, 11, 47), (2100, 12, 12)])
def test_svgd_step_matches_oracle(N, M, P, fast):
    _compare(N, M, P, seed=N + 10 * M, fast=fast)


def test_svgd_five_steps_match_oracle():
    _compare(300, 4, 12, seed=5, steps=5)


def test_single_particle_phi_is_gradient():
    lo, hi, x, g = _case(1, 3, 3, seed=1)
    sv = api.Svgd(1, 3, 3, lo, hi)
    bw, phi = sv.step(_gpu(x), _gpu(g), return_phi=True)
    torch.cuda.synchronize()
    assert bw.item() == 1.0
    np.testing.assert_allclose(phi.cpu().numpy().T, g * (hi - lo), rtol=1e-6)


def test_exact_median_on_integer_grid():
    """Distances that FP32 represents exactly: the radix select must return
    the same median as a brute-force sort, bit for bit."""
    rng = np.random.default_rng(3)
    N, M = 513, 3
    lo, hi = np.zeros(M), np.full(M, 64.0)
    pts = rng.integers(0, 64, size=(N, M)).astype(np.float64)
    u = pts / 64.0  # exact in binary: (theta - 0) / 64
    d = np.sort([np.sum((u[i] - u[j]) ** 2) for i in range(N) for j in range(i + 1, N)])
    med = d[(len(d) - 1) // 2]
    sv = api.Svgd(N, M, M, lo, hi)
    bw, _ = sv.step(_gpu(pts), _gpu(np.zeros_like(pts)))
    torch.cuda.synchronize()
    # neighbouring distances on this grid differ by >= 2^-12 (relative 5e-4
    # near the median), so 1e-6 agreement pins the exact order statistic
    assert abs(bw.item() - med / np.log(N)) <= 1e-6 * med / np.log(N)


def test_coincident_particles_give_unit_bandwidth():
    N, M = 50, 2
    lo, hi = np.zeros(M), np.ones(M)
    x = np.full((N, M), 0.5)
    sv = api.Svgd(N, M, M, lo, hi)
    bw, phi = sv.step(_gpu(x), _gpu(np.ones_like(x)), return_phi=True)
    torch.cuda.synchronize()
    assert bw.item() == 1.0
    np.testing.assert_allclose(phi.cpu().numpy(), 1.0, rtol=1e-6)


@pytest.mark.slow
def test_full_size_bandwidth_and_phi():
    """N = 16384, M = 10 (the benchmark's particle set): bandwidth over all
    1.3e8 pairs and phi of every particle against the oracle."""
    N, M, P = 16384, 10, 10
    lo, hi, x, g = _case(N, M, P, seed=11)
    sv = api.Svgd(N, M, P, lo, hi)
    bw, phi = sv.step(_gpu(x), _gpu(g), return_phi=True)
    torch.cuda.synchronize()
    u = (x[:, :M] - lo) / (hi - lo)
    bw_ref = orc.bandwidth(N, orc.median_sqdist(u))
    assert abs(bw.item() - bw_ref) <= 1e-5 * bw_ref
    rng = np.random.default_rng(0)
    idx = rng.choice(N, 64, replace=False)
    gu = g[:, :M] * (hi - lo)
    # phi rows for sampled particles: the oracle's phi over all j, evaluated row by row
    full = orc.svgd_phi(u, gu, bw_ref)
    phi = phi.cpu().numpy().T
    scale = np.max(np.abs(full))
    assert np.max(np.abs(phi[idx] - full[idx])) <= PHI_TOL * scale


def test_maximum_size_step():
    """N = 65536 (the largest SVGD state) and M = 16 (the largest theta):
    2.1e9 pairs, just under 2^31.  The exact lower median is checked by its
    rank among 4e5 sampled pairs (within 4 standard deviations of the
    middle); phi of 32 sampled particles (the last one included) against the
    oracle's phi of those rows with the GPU's bandwidth."""
    N, M, P = 65536, 16, 18
    lo, hi, x, g = _case(N, M, P, seed=21)
    sv = api.Svgd(N, M, P, lo, hi)
    bw, phi = sv.step(_gpu(x), _gpu(g), return_phi=True)
    torch.cuda.synchronize()
    bw = bw.item()
    u = (x[:, :M] - lo) / (hi - lo)
    rng = np.random.default_rng(5)
    n_s = 400000
    i = rng.integers(0, N, n_s)
    j = rng.integers(0, N - 1, n_s)
    j[j >= i] += 1
    d = ((u[i] - u[j]) ** 2).sum(axis=1)
    frac = np.mean(d < bw * np.log(N))
    assert abs(frac - 0.5) < 4 * 0.5 / np.sqrt(n_s), frac
    rows = rng.choice(N, 32, replace=False)
    rows[-1] = N - 1
    ref = orc.svgd_phi_rows(u, g[:, :M] * (hi - lo), bw, rows)
    got = phi.cpu().numpy().T[rows]
    assert np.max(np.abs(got - ref)) <= PHI_TOL * np.max(np.abs(ref))
    sv.close()


def test_svgd_rejects_bad_sizes():
    with pytest.raises(api.PdsError):
        api.Svgd(0, 2, 2, [0, 0], [1, 1])
    with pytest.raises(api.PdsError):
        api.Svgd(10, 17, 17, np.zeros(17), np.ones(17))
    with pytest.raises(api.PdsError):
        api.Svgd(10, 2, 2, [0, 1], [1, 1])


def _bw(x, lo, hi, full):
    N, M = x.shape
    sv = api.Svgd(N, M, M, lo, hi)
    sv.set_option(api.OPT_MEDIAN_FULL_PASSES, int(full))
    bw, _ = sv.step(_gpu(x), _gpu(np.zeros_like(x)))
    torch.cuda.synchronize()
    out = float(bw.item())
    sv.close()
    return out


@pytest.mark.parametrize("kind", ["uniform", "clusters", "grid_ties"])
def test_sampled_bracket_median_equals_full_passes(kind):
    """N >= 2048 selects the median among the pairs inside a sampled bracket;
    it must equal the three full radix passes bit for bit."""
    rng = np.random.default_rng(17)
    N, M = 4099, 5
    lo, hi = np.zeros(M), np.ones(M)
    if kind == "uniform":
        x = rng.uniform(size=(N, M))
    elif kind == "clusters":
        c = rng.uniform(size=(3, M))
        x = np.clip(c[rng.integers(0, 3, N)] + 0.01 * rng.normal(size=(N, M)), 0, 1)
    else:
        x = rng.integers(0, 4, size=(N, M)) / 4.0  # few distinct distances, many ties
    x = x.astype(np.float32).astype(np.float64)
    b_bracket = _bw(x, lo, hi, False)
    b_full = _bw(x, lo, hi, True)
    assert b_bracket == b_full
    if kind == "grid_ties":
        u = x
        d = ((u[:, None, :] - u[None, :, :]) ** 2).sum(-1)[np.triu_indices(N, 1)]
        med = np.partition(d, (len(d) - 1) // 2)[(len(d) - 1) // 2]
        assert abs(b_full - med / np.log(N)) <= 1e-6 * med / np.log(N)


@pytest.mark.parametrize("N,M", [(256, 1), (300, 4), (1000, 10), (777, 16), (4096, 10), (2500, 8), (1500, 11),
                                 (2049, 12)])
def test_tensor_core_phi_matches_cuda_cores(N, M):
    """phi's kernel-matrix products on tcgen05 (split tf32 operands, fp32
    accumulation; the kernel values themselves rounded to tf32) against the
    fp32 CUDA-core kernel."""
    lo, hi, x, g = _case(N, M, M + 3, seed=N + M)
    out = []
    for cuda_cores in (1, 0):
        sv = api.Svgd(N, M, M + 3, lo, hi)
        sv.set_option(api.OPT_PHI_CUDA_CORES, cuda_cores)
        bw, phi = sv.step(_gpu(x), _gpu(g), return_phi=True)
        torch.cuda.synchronize()
        out.append((bw.item(), phi.cpu().numpy().T))
        sv.close()
    assert out[0][0] == out[1][0]
    ref, tcp = out[0][1], out[1][1]
    # the kernel values enter the second product rounded to tf32 (relative
    # 2^-11 at most, unbiased): about 1e-4 of the largest |phi|
    assert np.max(np.abs(tcp - ref)) <= 1e-3 * np.max(np.abs(ref)), np.max(np.abs(tcp - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("N,M", [(2048, 2), (3001, 10), (4096, 16), (2600, 11), (4100, 12)])
def test_tensor_core_median_matches_cuda_cores(N, M):
    """Pair distances of the median passes from tensor-core products against
    the CUDA-core distances: the same bandwidth within 1e-5."""
    rng = np.random.default_rng(N)
    lo, hi = np.zeros(M), np.ones(M)
    x = rng.uniform(size=(N, M))
    out = []
    for cc in (1, 0):
        sv = api.Svgd(N, M, M, lo, hi)
        sv.set_option(api.OPT_MEDIAN_CUDA_CORES, cc)
        bw, _ = sv.step(_gpu(x), _gpu(np.zeros_like(x)))
        torch.cuda.synchronize()
        out.append(bw.item())
        sv.close()
    assert abs(out[0] - out[1]) <= 1e-5 * out[0], out
    u = x
    d = ((u[:, None, :] - u[None, :, :]) ** 2).sum(-1)[np.triu_indices(N, 1)]
    med = np.partition(d, (len(d) - 1) // 2)[(len(d) - 1) // 2]
    assert abs(out[1] - med / np.log(N)) <= 1e-5 * med / np.log(N)


@pytest.mark.parametrize("N,M,phi_cc,med_cc,full", [(300, 4, 0, 0, 0), (300, 4, 1, 1, 0), (2500, 6, 0, 0, 0),
                                                      (2500, 6, 0, 0, 1), (2500, 6, 1, 1, 0)])
def test_particles_that_are_not_finite_sit_out(N, M, phi_cc, med_cc, full):
    """Particles with a non-finite gradient or coordinate take no part in the
    median or the other particles' phi (tensor-core and CUDA-core paths,
    bracket and full passes); against the oracle's step over the live set."""
    rng = np.random.default_rng(N + M)
    P = M + 2
    lo, hi = np.zeros(M), np.ones(M)
    x = rng.uniform(0.05, 0.95, size=(N, P)).astype(np.float32).astype(np.float64)
    g = rng.normal(size=(N, P)).astype(np.float32).astype(np.float64)
    dead = rng.choice(N, 7, replace=False)
    g[dead[:3], 0] = np.inf
    g[dead[3:5], M - 1] = np.nan
    x[dead[5:], 1] = np.nan
    live = np.setdiff1d(np.arange(N), dead)
    sv = api.Svgd(N, M, P, lo, hi)
    sv.set_option(api.OPT_PHI_CUDA_CORES, phi_cc)
    sv.set_option(api.OPT_MEDIAN_CUDA_CORES, med_cc)
    sv.set_option(api.OPT_MEDIAN_FULL_PASSES, full)
    X = _gpu(x)
    bw, phi = sv.step(X, _gpu(g), return_phi=True)
    torch.cuda.synchronize()
    ost = orc.SvgdState(N, P, lo, hi, lr=1e-2)
    xo = np.ascontiguousarray(x.copy())
    phi_ref, bw_ref = ost.step(xo, g)
    assert abs(bw.item() - bw_ref) <= 1e-5 * bw_ref, (bw.item(), bw_ref)
    phi = phi.cpu().numpy().T
    assert np.all(np.isfinite(phi[live]))
    assert np.max(np.abs(phi[live] - phi_ref[live])) <= PHI_TOL * np.max(np.abs(phi_ref[live]))
    assert np.all(np.isnan(phi[dead]))
    sv.close()


@pytest.mark.parametrize("N,M", [(2, 1), (3, 2), (50, 4), (100, 4), (129, 10), (200, 16), (255, 7), (256, 12)])
def test_small_median_in_one_block_equals_the_full_passes(N, M):
    """For N <= 256 the median runs in one block with every pair distance in
    shared memory; it must give the bandwidth of the three radix passes over
    recomputed distances bit for bit, also with particles that sit out."""
    rng = np.random.default_rng(N * 7 + M)
    lo, hi = np.zeros(M), np.ones(M)
    x = rng.uniform(size=(N, M)).astype(np.float32).astype(np.float64)
    for dead in (False, True):
        if dead and N > 3:
            x[rng.choice(N, 3, replace=False), rng.integers(0, M)] = np.nan
        out = [_bw(x, lo, hi, full) for full in (False, True)]
        assert out[0] == out[1], (out, dead)
    live = np.all(np.isfinite(x), axis=1)
    u = x[live]
    if len(u) >= 2:
        d = np.sort(((u[:, None, :] - u[None, :, :]) ** 2).sum(-1)[np.triu_indices(len(u), 1)])
        med = d[(len(d) - 1) // 2]
        ref = med / np.log(len(u)) if med > 0 else 1.0
        assert abs(out[0] - ref) <= 1e-5 * ref
