"""Request-stream drivers for the serving loop (pds_server_*) and for the
plain baseline that runs the same jobs one at a time.

A job is (workload, observations, initial particles, iterations).  Arrivals
follow a seeded Poisson process.  Time-to-posterior is measured from a job's
scheduled arrival to the moment its final particles are on the host.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api


def poisson_arrivals(n_jobs: int, rate: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))


def run_server(jobs, arrivals, mem_budget, max_active=256, checkpoint_stride=1, fast_math=True, stream=None,
               gate=None, iters_out=None):
    """Continuous batching: submit each job at its arrival time, tick the
    server until every job is done.  Returns (latencies [s], results, wall).
    ``gate`` = (metric, every, threshold, h) sets the server's convergence
    gate; ``iters_out`` (a list) receives each job's iterations run."""
    srv = api.Server(mem_budget, max_active=max_active, stream=stream, checkpoint_stride=checkpoint_stride,
                     fast_math=fast_math)
    if gate is not None:
        srv.set_gate(*gate)
    n = len(jobs)
    used = [0] * n
    ids = [None] * n
    done_at = [None] * n
    results = [None] * n
    t0 = time.perf_counter()
    nxt = 0
    pending = set()
    while nxt < n or pending:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            wl, obs, x, iters = jobs[nxt]
            ids[nxt] = srv.submit(wl, obs, x, iters)
            pending.add(nxt)
            nxt += 1
        if not pending:
            time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
            continue
        _, retired = srv.tick()
        if retired:
            t = time.perf_counter() - t0
            for k in list(pending):
                st, used[k] = srv.status(ids[k])
                if st == api.JOB_DONE:
                    results[k] = srv.result(ids[k])
                    done_at[k] = t
                    pending.discard(k)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([done_at[k] - arrivals[k] for k in range(n)])
    if iters_out is not None:
        iters_out[:] = used
    return lat, results, wall


def run_plain(jobs, arrivals, checkpoint_stride=1, fast_math=True, stream=None):
    """Baseline: one job at a time in arrival order, one kernel launch
    sequence per iteration (pds_iterate), no graph and no cross-job batching."""
    n = len(jobs)
    done_at = [None] * n
    results = [None] * n
    t0 = time.perf_counter()
    for k, (wl, obs, x, iters) in enumerate(jobs):
        now = time.perf_counter() - t0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        prob = api.Problem.from_workload(wl, obs, stream=stream, checkpoint_stride=checkpoint_stride,
                                         fast_math=fast_math)
        sv = api.Svgd(wl.N, wl.M, wl.P, wl.lo, wl.hi, lr=wl.lr, stream=stream)
        xh = np.ascontiguousarray(np.asarray(x).T, dtype=np.float32)
        lp = np.empty(wl.N, np.float32)
        api.iterate_host(prob, sv, xh, iters, lp)
        results[k] = (xh.T.copy(), lp)
        done_at[k] = time.perf_counter() - t0
        sv.close()
        prob.close()
    wall = time.perf_counter() - t0
    lat = np.array([done_at[k] - arrivals[k] for k in range(n)])
    return lat, results, wall


def percentiles(lat):
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat))}


def synchronize():
    torch.cuda.synchronize()
