"""qng_metric_noalloc, the metric entry point for callers that cannot allocate device memory
(their GPU memory belongs to a host application's pool, or cudaMalloc's synchronisation is not
allowed where they run). It must give the same metric as qng_metric, call after call.

This file is collected last so that a failure here does not hide any other test's result.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2011_02991_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def qng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_02991_gb300 import build as B
    B.build()
    from paper_2011_02991_gb300 import qng as Q
    L = Q.load()
    L.qng_metric_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(Q.qng_gate), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.qng_metric_noalloc.restype = ctypes.c_int
    return Q


def _noalloc(Q, p, theta, g, stream):
    ga, ng = Q._gates_array(p.circuit)
    return Q.load().qng_metric_noalloc(p.n, ga, ng, p.precision, ctypes.c_void_p(theta.data_ptr()),
                                       ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("maker,tol", [(W.config_rand12, 1e-10), (W.config_tfim4, 1e-10),
                                       (lambda: W.config_rand12(precision=W.C64), 2e-4),
                                       (lambda: W.random_problem(7, 60, 4, 808), 1e-10)])
def test_noalloc_matches_metric_twice(qng, maker, tol):
    p = maker()
    stream = torch.cuda.current_stream()
    ctx = qng.Context(p)
    theta = ctx.theta0()
    ref = ctx.metric(theta)
    ctx.sync()
    for call in range(2):  # the shared scratch keeps the last call's contents: both calls must agree
        g = torch.full((p.P * p.P,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(qng, p, theta, g, stream) == 0
        torch.cuda.synchronize()
        assert _rel(g.cpu(), ref.cpu()) <= tol, (p.name, call)


def test_noalloc_rejects_too_large(qng):
    # 14 qubits, P = 200 at complex128 needs about 52 MB of checkpoints, more than the scratch array
    c = W.layered_ansatz(14, 8)
    p = W.Problem("big", c, W.tfim_chain(14), np.zeros(c.num_params))
    theta = torch.zeros(p.P, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.P * p.P, dtype=torch.float64, device="cuda")
    assert _noalloc(qng, p, theta, g, torch.cuda.current_stream()) == qng.QNG_ERR_WORKSPACE


def test_noalloc_against_oracle(qng, oracle):
    """The allocation-free call against the CPU oracle directly (not only against qng_metric)."""
    stream = torch.cuda.current_stream()
    for p, tol in ((W.random_problem(6, 60, 4, 909), 1e-10), (W.config_rand12(), 1e-10)):
        ref = oracle.qng_step(p)["g"]
        theta = torch.tensor(p.theta, dtype=torch.float64, device="cuda")
        for call in range(2):
            g = torch.full((p.P * p.P,), float("nan"), dtype=torch.float64, device="cuda")
            assert _noalloc(qng, p, theta, g, stream) == 0
            torch.cuda.synchronize()
            assert _rel(g.cpu(), ref) <= tol, (p.name, call)


def test_noalloc_leaves_live_context_working(qng, oracle):
    """A small allocation-free call between two calls of a larger live context: the kernels' shared
    memory limits are process-wide, so the small call must not lower what the context needs."""
    big = W.config_rand12()
    ctx = qng.Context(big)
    ref = oracle.qng_step(big)
    small = W.config_tfim4()
    theta_s = torch.tensor(small.theta, dtype=torch.float64, device="cuda")
    g_s = torch.zeros(small.P * small.P, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = ctx.step(ctx.theta0(), big.dt, big.lam)
        ctx.sync()
        assert _rel(out["g"].cpu(), ref["g"]) <= 1e-10
        assert _rel(out["dtheta"].cpu(), ref["dtheta"]) <= 1e-10
        assert _noalloc(qng, small, theta_s, g_s, stream) == 0
        torch.cuda.synchronize()


def test_noalloc_refuses_capturing_stream(qng):
    """Under stream capture the call would record copies from stack memory that is gone when the
    graph runs: it must return QNG_ERR_UNSUPPORTED and issue nothing."""
    p = W.config_tfim4()
    theta = torch.tensor(p.theta, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.P * p.P, dtype=torch.float64, device="cuda")
    x = torch.zeros(16, device="cuda")
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        status = _noalloc(qng, p, theta, g, torch.cuda.current_stream())
    assert status == qng.QNG_ERR_UNSUPPORTED
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert _noalloc(qng, p, theta, g, torch.cuda.current_stream()) == 0  # outside capture it runs
    torch.cuda.synchronize()
