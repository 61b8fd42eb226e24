"""The SVGD step replayed from a CUDA graph (PDS_OPT_GRAPH, on by default on
a stream of the caller's) computes exactly what its kernels launched one by
one compute: the same particles, bandwidth and phi bit for bit over several
steps, when the buffers change between calls (a new capture), when options
change, with the tensor-core and the CUDA-core passes, and inside a graph
the caller captures.  Also checked against the oracle's step."""
import numpy as np
import pytest
import torch

from helpers import PHI_TOL
from oracle import pds_oracle as orc
from paper_2109_08815_gb300 import api

pytestmark = pytest.mark.gpu


def _case(N, M, P, seed):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-1, 0, M)
    hi = lo + rng.uniform(0.5, 2, M)
    x = np.concatenate([lo + (hi - lo) * rng.uniform(size=(N, M)), rng.normal(size=(N, P - M))], 1)
    g = rng.normal(size=(N, P))
    return (lo.astype(np.float32).astype(np.float64), hi.astype(np.float32).astype(np.float64),
            x.astype(np.float32), g.astype(np.float32))


def _run(N, M, P, seed, graph, steps, stream, options=()):
    lo, hi, x, g = _case(N, M, P, seed)
    with torch.cuda.stream(stream):
        X = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
        G = torch.from_numpy(np.ascontiguousarray(g.T)).cuda()
        sv = api.Svgd(N, M, P, lo, hi, stream=stream)
        sv.set_option(api.OPT_GRAPH, int(graph))
        for opt, val in options:
            sv.set_option(opt, val)
        out = []
        for k in range(steps):
            bw, phi = sv.step(X, G, return_phi=(k % 2 == 0))
            out.append((bw, phi))
    stream.synchronize()
    res = [X.cpu().numpy()] + [(b.cpu().numpy(), None if p is None else p.cpu().numpy()) for b, p in out]
    sv.close()
    return res


def _same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    for (ba, pa), (bb, pb) in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(ba, bb)
        if pa is not None:
            np.testing.assert_array_equal(pa, pb)


@pytest.mark.parametrize("N,M,P,options", [(4096, 10, 30, ()), (700, 4, 9, ()),
                                           (3000, 6, 6, ((api.OPT_PHI_CUDA_CORES, 1), (api.OPT_MEDIAN_CUDA_CORES, 1))),
                                           (2500, 5, 12, ((api.OPT_MEDIAN_FULL_PASSES, 1),)),
                                           (150, 3, 5, ())])
def test_graph_replay_equals_direct_launches(N, M, P, options):
    s = torch.cuda.Stream()
    a = _run(N, M, P, N, True, 6, s, options)
    b = _run(N, M, P, N, False, 6, s, options)
    _same(a, b)


@pytest.mark.parametrize("N,M,P", [(4096, 10, 30), (300, 3, 7)])
def test_graph_on_the_default_stream_equals_direct_launches(N, M, P):
    """On torch's default stream (the legacy stream, which cannot be
    captured) the graph runs on the state's own stream, ordered by events:
    the same bits, and the caller's next default-stream work sees them."""
    s = torch.cuda.default_stream()
    a = _run(N, M, P, N + 1, True, 5, s)
    b = _run(N, M, P, N + 1, False, 5, s)
    _same(a, b)
    # default-stream work right after a replayed step reads its result
    lo, hi, x, g = _case(N, M, P, N + 2)
    X = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    G = torch.from_numpy(np.ascontiguousarray(g.T)).cuda()
    sv = api.Svgd(N, M, P, lo, hi)
    sums = []
    for _ in range(4):
        sv.step(X, G)
        sums.append(X.double().sum())  # queued on the default stream
    torch.cuda.synchronize()
    sv.close()
    ref = api.Svgd(N, M, P, lo, hi)
    ref.set_option(api.OPT_GRAPH, 0)
    Y = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    ref_sums = []
    for _ in range(4):
        ref.step(Y, G)
        ref_sums.append(Y.double().sum())
    torch.cuda.synchronize()
    ref.close()
    assert [float(v) for v in sums] == [float(v) for v in ref_sums]


def test_new_buffers_and_options_recapture():
    """Steps alternate between two particle sets (each captured on its second
    use) and switch an option midway; every step equals the direct path."""
    N, M, P = 2100, 8, 20
    s = torch.cuda.Stream()
    lo, hi, x, g = _case(N, M, P, 5)
    outs = []
    for graph in (1, 0):
        with torch.cuda.stream(s):
            XA = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
            XB = XA.clone()
            G = torch.from_numpy(np.ascontiguousarray(g.T)).cuda()
            sv = api.Svgd(N, M, P, lo, hi, stream=s)
            sv.set_option(api.OPT_GRAPH, graph)
            bws = []
            for k in range(8):
                if k == 5:
                    sv.set_option(api.OPT_FAST_MATH, 1)
                bw, _ = sv.step(XA if k % 2 == 0 else XB, G)
                bws.append(bw)
        s.synchronize()
        outs.append((XA.cpu().numpy(), XB.cpu().numpy(), [b.item() for b in bws]))
        sv.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_graph_step_matches_the_oracle_and_reports_its_launches():
    N, M, P = 4096, 10, 30
    s = torch.cuda.Stream()
    lo, hi, x, g = _case(N, M, P, 9)
    with torch.cuda.stream(s):
        X = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
        G = torch.from_numpy(np.ascontiguousarray(g.T)).cuda()
        sv = api.Svgd(N, M, P, lo, hi, stream=s)
        sv.step(X.clone(), G)  # first call with other buffers: direct
        n_direct = api.last_launch_count()
        Y = X.clone()
        sv.reset()
        sv.step(Y, G)          # direct (first use of Y)
        sv.reset()
        Y.copy_(X)
        sv.step(Y, G)          # captured and replayed
        n_graph = api.last_launch_count()
    s.synchronize()
    assert n_graph == n_direct > 10
    ost = orc.SvgdState(N, P, lo, hi, lr=1e-2)
    xo = np.ascontiguousarray(x.astype(np.float64))
    phi_ref, _ = ost.step(xo, g.astype(np.float64))
    d = np.abs(Y.cpu().numpy().T - xo) / np.concatenate([hi - lo, np.ones(P - M)])
    near0 = np.zeros_like(d, dtype=bool)
    near0[:, :M] = np.abs(phi_ref) <= PHI_TOL * np.max(np.abs(phi_ref))
    assert np.all(d[~near0] <= 1e-4)
    sv.close()


def test_step_inside_a_callers_graph():
    """When the caller captures the state's stream, the step's kernels go
    into the caller's graph (the library does not capture its own)."""
    N, M, P = 1500, 5, 7
    s = torch.cuda.Stream()
    lo, hi, x, g = _case(N, M, P, 13)
    with torch.cuda.stream(s):
        X = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
        G = torch.from_numpy(np.ascontiguousarray(g.T)).cuda()
        sv = api.Svgd(N, M, P, lo, hi, stream=s)
        sv.step(X.clone(), G)  # set-up outside the capture
        sv.reset()
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        sv.step(X, G)
    for _ in range(3):
        graph.replay()
    s.synchronize()
    ref = _run(N, M, P, 13, False, 3, s)
    np.testing.assert_array_equal(X.cpu().numpy(), ref[0])
    sv.close()
