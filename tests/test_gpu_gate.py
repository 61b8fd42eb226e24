"""The server's convergence gate: the posterior metrics of Sec. IV (unbiased
RBF MMD^2 and the KNN-KL estimate with k = 3) between successive snapshots of
a job's theta particles in unit-box coordinates decide when the job has
reached its posterior.

Covers:
  * the gate's value equals the FP64 metric reference on the snapshots
    (taken from two gate-less servers stopped at the two snapshot
    iterations), for both metrics, with a particle that sits out (its log p
    is not finite; the update clips its theta back into the box) left out of
    both sets;
  * a threshold that holds retires the job at its first evaluation, one that
    never holds runs it to its cap with one evaluation per `every`
    iterations after the first snapshot;
  * the gate must be set before jobs are submitted.
"""
import numpy as np
import pytest

from helpers import f32_workload, observations, particles
from oracle import metrics_oracle as mo
from paper_2109_08815_gb300 import api
from paper_2109_08815_gb300 import workloads as wlmod

pytestmark = pytest.mark.gpu

EVERY = 3


def _job(nan_particle=False):
    wl = f32_workload(wlmod.batched_problems(n_jobs=1, seed=31, T_range=(60, 60), W_range=(3, 3),
                                             N_range=(300, 300))[0])
    obs = observations(wl)
    x = particles(wl, obs, seed=5).copy()
    if nan_particle:
        x[7, 0] = np.nan
    return wl, obs, x


def _run(wl, obs, x, iters, gate=None):
    srv = api.Server(1 << 34, max_active=4)
    if gate is not None:
        srv.set_gate(*gate)
    jid = srv.submit(wl, obs, x, iters)
    for _ in range(10 * iters):
        srv.tick()
        if srv.status(jid)[0] == api.JOB_DONE:
            break
    st, done = srv.status(jid)
    assert st == api.JOB_DONE
    checks, value = srv.gate(jid)
    xr, lp = srv.result(jid)
    srv.close()
    return (xr, lp), done, checks, value


def _unit_live(wl, res):
    x, lp = res
    u = (x[:, :wl.M].astype(np.float64) - wl.lo) / (wl.hi - wl.lo)
    return u[np.all(np.isfinite(u), axis=1) & np.isfinite(lp)]


@pytest.mark.parametrize("metric", [api.GATE_MMD2, api.GATE_KNN_KL])
def test_gate_value_equals_reference_metric(metric):
    wl, obs, x = _job(nan_particle=True)
    h = 1.0 / 6.0
    x1, _, _, _ = _run(wl, obs, x, EVERY)
    x2, _, _, _ = _run(wl, obs, x, 2 * EVERY)
    xg, done, checks, value = _run(wl, obs, x, 10 * EVERY, gate=(metric, EVERY, 1e30, h))
    assert done == 2 * EVERY and checks == 1
    assert np.array_equal(xg[0], x2[0], equal_nan=True)
    u_now, u_prev = _unit_live(wl, x2), _unit_live(wl, x1)
    assert len(u_now) == len(x) - 1
    if metric == api.GATE_MMD2:
        ref = mo.mmd2_unbiased(u_now, u_prev, h * wl.M)
        assert abs(value - ref) <= 1e-5 + 1e-4 * abs(ref), (value, ref)
    else:
        ref = mo.knn_kl(u_now, u_prev, k=3)
        assert abs(value - ref) <= 1e-4 * max(1.0, abs(ref)), (value, ref)


def test_gate_retires_early_or_runs_to_the_cap():
    wl, obs, x = _job()
    _, done, checks, value = _run(wl, obs, x, 8 * EVERY, gate=(api.GATE_MMD2, EVERY, 1e30, 1.0 / 6.0))
    assert done == 2 * EVERY and checks == 1 and np.isfinite(value)
    _, done, checks, value = _run(wl, obs, x, 8 * EVERY, gate=(api.GATE_MMD2, EVERY, -1e30, 1.0 / 6.0))
    assert done == 8 * EVERY and checks == 7 and np.isfinite(value)


def test_gate_is_set_before_jobs():
    wl, obs, x = _job()
    srv = api.Server(1 << 34)
    srv.submit(wl, obs, x, 2)
    with pytest.raises(api.PdsError):
        srv.set_gate(api.GATE_MMD2, 2, 1e-3)
    srv.close()
    srv = api.Server(1 << 34)
    with pytest.raises(api.PdsError):
        srv.set_gate(api.GATE_MMD2, 0, 1e-3)
    with pytest.raises(api.PdsError):
        srv.set_gate(7, 2, 1e-3)
    srv.close()
