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
