"""Serving loop with continuous batching (pds_server_*).

Jobs arriving while others run are admitted as memory frees up and iterate
together in shared batched launches.  Each job's posterior particles must be
the same in the mix as when the job runs alone with the same settings (within
FP32 rounding: the batched rollout is a different kernel), admission must
respect the memory budget, and cancellation must release a job.
"""
import numpy as np
import pytest

from helpers import f32_workload, observations, particles
from paper_2109_08815_gb300 import api, serve
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu


def _jobs(n, seed, iters, **kw):
    wls = [f32_workload(w) for w in wlmod.batched_problems(n_jobs=n, seed=seed, **kw)]
    out = []
    for w in wls:
        o = observations(w)
        out.append((w, o, particles(w, o, seed=9), iters))
    return out


def _close(a, b, wl, rtol=1e-5):
    width = np.concatenate([wl.hi - wl.lo, np.ones(wl.P - wl.M)])
    return np.max(np.abs(a - b) / width) <= rtol


def test_results_in_the_mix_equal_alone():
    jobs = _jobs(6, seed=123, iters=4, T_range=(30, 150), W_range=(2, 8), N_range=(30, 500))
    arrivals = np.array([0.0, 0.0, 0.01, 0.02, 0.03, 0.05])
    lat, res, _ = serve.run_server(jobs, arrivals, mem_budget=8 << 30)
    _, alone, _ = serve.run_plain(jobs, np.zeros(len(jobs)))
    for k, (wl, _, _, _) in enumerate(jobs):
        assert _close(res[k][0], alone[k][0], wl), k
        np.testing.assert_allclose(res[k][1], alone[k][1], rtol=1e-6)
    assert np.all(lat >= 0)


def test_admission_respects_memory_budget():
    jobs = _jobs(5, seed=7, iters=3, T_range=(40, 80), W_range=(2, 4), N_range=(200, 300))
    srv = api.Server(mem_budget_bytes=1 << 40, max_active=2)
    ids = [srv.submit(w, o, x, it) for (w, o, x, it) in jobs]
    seen_active = 0
    for _ in range(100):
        a, _ = srv.tick()
        q, act, _ = srv.stats()
        seen_active = max(seen_active, act)
        assert act <= 2
        if all(srv.status(i)[0] == api.JOB_DONE for i in ids):
            break
    assert seen_active == 2
    for i in ids:
        assert srv.status(i) == (api.JOB_DONE, 3)
        x, lp = srv.result(i)
        assert np.all(np.isfinite(lp))
    srv.close()


def test_job_over_budget_is_rejected():
    (w, o, x, it), = _jobs(1, seed=3, iters=2, T_range=(100, 200), W_range=(4, 8), N_range=(500, 600))
    srv = api.Server(mem_budget_bytes=1 << 16)
    with pytest.raises(api.PdsError, match="budget"):
        srv.submit(w, o, x, it)
    srv.close()


def test_cancel_queued_and_active_jobs():
    jobs = _jobs(3, seed=11, iters=5, T_range=(30, 60), W_range=(2, 4), N_range=(50, 100))
    srv = api.Server(mem_budget_bytes=1 << 40, max_active=1)
    ids = [srv.submit(w, o, x, it) for (w, o, x, it) in jobs]
    srv.tick()                      # job 0 active, 1 and 2 queued
    assert srv.status(ids[0])[0] == api.JOB_ACTIVE
    srv.cancel(ids[1])              # queued
    srv.cancel(ids[0])              # active
    for _ in range(20):
        srv.tick()
    assert srv.status(ids[2]) == (api.JOB_DONE, 5)
    q, a, b = srv.stats()
    assert q == 0 and a == 0 and b == 0
    srv.close()


def test_admission_by_memory_budget():
    (w, o, x, it), = _jobs(1, seed=21, iters=3, T_range=(60, 80), W_range=(3, 4), N_range=(300, 310))
    probe = api.Server(mem_budget_bytes=1 << 40)
    jid = probe.submit(w, o, x, it)
    probe.tick()
    _, _, one = probe.stats()
    probe.close()
    assert one > 0
    srv = api.Server(mem_budget_bytes=int(1.5 * one))   # room for one such job at a time
    ids = [srv.submit(w, o, x, it) for _ in range(3)]
    for _ in range(30):
        srv.tick()
        q, act, used = srv.stats()
        assert act <= 1 and used <= 1.5 * one
        if all(srv.status(i)[0] == api.JOB_DONE for i in ids):
            break
    results = [srv.result(i)[0] for i in ids]
    for r in results[1:]:
        np.testing.assert_array_equal(r, results[0])   # same job, same result, whenever it ran
    srv.close()


def test_armbox_job_in_the_mix_equals_alone():
    jobs = _jobs(3, seed=55, iters=3, T_range=(30, 90), W_range=(2, 5), N_range=(30, 200))
    wl = wlmod.arm_box(N=256, seed=77, T=200, W=5)
    from oracle import pds_oracle as orc
    st = orc.ArmBox.from_workload(wl).simulate(wl.theta_true, wl.dt, wl.T, wl.s0)
    obs = (st[1:, wl.obs_index] + wl.sigma_obs * wl.noise[:wl.T]).astype(np.float32)
    shoot = st[[wl.window_start(w) for w in range(1, wl.W)]].ravel()
    x = np.concatenate([wl.theta_init, np.tile(shoot, (wl.N, 1))], 1)
    jobs.insert(1, (wl, obs, x, 3))
    arrivals = np.array([0.0, 0.0, 0.005, 0.01])
    _, res, _ = serve.run_server(jobs, arrivals, mem_budget=8 << 30)
    _, alone, _ = serve.run_plain(jobs, np.zeros(len(jobs)))
    for k, (w, _, _, _) in enumerate(jobs):
        width = np.concatenate([w.hi - w.lo, np.ones(w.P - w.M)])
        assert np.max(np.abs(res[k][0] - alone[k][0]) / width) <= 1e-5, k
