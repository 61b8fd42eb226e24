"""The allocation-free bandwidth entry point (pds_bandwidth_noalloc).

Some callers cannot allocate device memory -- code that runs inside another
framework's allocator or memory-pool callback, or a process whose device
memory is reserved up front -- so they cannot create the workspace that
pds_svgd_create allocates.  pds_bandwidth_noalloc gives them the median
bandwidth with its scratch in a static device array.  This test calls it
through the C ABI twice in a row (the shared scratch keeps the previous
call's contents, which the entry point must clear) and checks each result
against the bandwidth that pds_svgd_step reports for the same particles,
within the tolerance the SVGD tests use (relative 1e-5).

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu

BW_RTOL = 1e-5


def _particles(N, M, P, seed):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-2, 0, M).astype(np.float32)
    hi = (lo + rng.uniform(0.5, 3, M)).astype(np.float32)
    x = np.empty((P, N), np.float32)
    x[:M] = lo[:, None] + (hi - lo)[:, None] * rng.uniform(size=(M, N))
    x[M:] = rng.normal(size=(P - M, N))
    g = rng.normal(size=(P, N)).astype(np.float32)
    return lo, hi, torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()


def test_noalloc_bandwidth_matches_svgd_step_on_two_calls_in_a_row():
    L = api.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty(1, device="cuda", dtype=torch.float32)
    for N, M, P, seed in ((3000, 10, 30, 1), (1537, 4, 4, 2)):
        lo, hi, X, G = _particles(N, M, P, seed)
        rc = L.pds_bandwidth_noalloc(ctypes.c_void_p(X.data_ptr()), N, M, lo.ctypes.data_as(api._fp),
                                     hi.ctypes.data_as(api._fp), ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.pds_last_error()
        torch.cuda.synchronize()
        bw_noalloc = float(out.item())
        sv = api.Svgd(N, M, P, lo, hi)
        bw_ref, _ = sv.step(X.clone(), G)
        torch.cuda.synchronize()
        ref = float(bw_ref.item())
        assert abs(bw_noalloc - ref) <= BW_RTOL * ref, (N, M, bw_noalloc, ref)
        sv.close()


def _noalloc(X, N, M, lo, hi, out):
    L = api.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.pds_bandwidth_noalloc(ctypes.c_void_p(X.data_ptr()), N, M, lo.ctypes.data_as(api._fp),
                                   hi.ctypes.data_as(api._fp), ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_call_allocates_no_device_memory():
    """After a first call (which loads the module and reserves the array), a
    call on a new particle count leaves the device's free memory unchanged."""
    M = 6
    lo, hi, X1, _ = _particles(2000, M, M, 3)
    _, _, X2, _ = _particles(2900, M, M, 4)
    out = torch.empty(1, device="cuda", dtype=torch.float32)
    assert _noalloc(X1, 2000, M, lo, hi, out) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(X2, 2900, M, lo, hi, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.isfinite(out.item()) and out.item() > 0


def test_noalloc_particles_that_are_not_finite_sit_out():
    """Particles with a non-finite coordinate take no part, as in
    pds_svgd_step (checked against its bandwidth for the same particles with
    a zero gradient); all particles but one non-finite gives bandwidth 1."""
    N, M = 1200, 5
    lo, hi, X, _ = _particles(N, M, M, 5)
    X[1, 7] = float("nan")
    X[0, 100] = float("inf")
    X[4, N - 1] = float("-inf")
    out = torch.empty(1, device="cuda", dtype=torch.float32)
    assert _noalloc(X, N, M, lo, hi, out) == 0
    torch.cuda.synchronize()
    sv = api.Svgd(N, M, M, lo, hi)
    bw_ref, _ = sv.step(X.clone(), torch.zeros_like(X))
    torch.cuda.synchronize()
    ref = float(bw_ref.item())
    assert abs(float(out.item()) - ref) <= BW_RTOL * ref, (float(out.item()), ref)
    sv.close()
    Y = X.clone()
    Y[2, 1:] = float("nan")
    assert _noalloc(Y, N, M, lo, hi, out) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 1.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = api.lib()
    lo = np.zeros(16, np.float32)
    hi = np.ones(16, np.float32)
    X = torch.zeros((16, 4), device="cuda")
    out = torch.empty(1, device="cuda")
    # N * M = 65537 * 16 > 1048576: rejected before any launch
    rc = L.pds_bandwidth_noalloc(ctypes.c_void_p(X.data_ptr()), 65537, 16, lo.ctypes.data_as(api._fp),
                                 hi.ctypes.data_as(api._fp), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"1048576" in L.pds_last_error()
    # N = 65537 with M = 1 fits the array but not the 32-bit pair counts
    rc = L.pds_bandwidth_noalloc(ctypes.c_void_p(X.data_ptr()), 65537, 1, lo.ctypes.data_as(api._fp),
                                 hi.ctypes.data_as(api._fp), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"65536" in L.pds_last_error()
