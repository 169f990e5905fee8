"""Parity at the full sizes of the 26- and 28-qubit workloads (streaming path, 1-4 GiB per state).

The oracle cannot build all P derivative states at these sizes (208 and 252 states of 1-4 GiB), so
it evaluates the definitions on a seeded subset S of parameters: G_ab, T_a and d<E>/d theta_a for
a, b in S, and <E>. Entries outside S are checked through properties that hold at any size: the
metric is symmetric, dtheta solves (g + lambda I) dtheta = -dt grad to float64 accuracy, and the
reverse-sweep gradient (through torch.autograd) equals the parameter-shift rule and central finite
differences of GPU energies on sampled parameters.

The complex128 run of the 28-qubit workload takes about two minutes of GPU time; it runs when the
environment variable QNG_FULL28_C128=1 is set.
"""
import os

import numpy as np
import pytest
import torch

from paper_2011_02991_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(got, ref):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


@pytest.fixture(scope="module")
def qng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_02991_gb300 import build as B
    B.build()
    from paper_2011_02991_gb300 import qng as Q
    return Q


def check_step(qng, oracle_ref, p, idx, tol):
    ctx = qng.Context(p)
    th = ctx.theta0()
    out = ctx.step(th, p.dt, p.lam)
    ctx.sync()
    g = out["g"].cpu().numpy().reshape(p.P, p.P)
    grad = out["grad"].cpu().numpy()
    dth = out["dtheta"].cpu().numpy()
    E = float(out["energy"].cpu().numpy()[0])
    Gs, Ts, grads, Eo = oracle_ref
    assert rel(g[np.ix_(idx, idx)], Gs.real) <= tol
    assert rel(grad[idx], grads) <= tol
    assert rel([E], [Eo]) <= tol
    # properties of the whole outputs
    assert np.abs(g - g.T).max() == 0.0
    A = g + p.lam * np.eye(p.P)
    r = A @ dth + p.dt * grad
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.dt * grad)
    return ctx, th, out


@pytest.fixture(scope="module")
def tfim26_ref(oracle):
    p = W.config_tfim26()
    idx = np.array([0, 60, 133, 207], dtype=np.int32)
    return p, idx, oracle.sampled(p, idx)


def test_tfim26_c128_sampled_and_autograd(qng, tfim26_ref):
    p, idx, ref = tfim26_ref
    ctx, th, out = check_step(qng, ref, p, idx, 1e-10)
    # torch.autograd through the reverse sweep vs parameter shift and central differences (eps 1e-5)
    theta = th.clone().requires_grad_(True)
    E = qng.energy(theta, ctx)
    E.sum().backward()
    g_ad = theta.grad.cpu().numpy()
    assert rel(g_ad, out["grad"].cpu().numpy()) <= 1e-12
    for k in (0, 103, 207):
        tp, tm = th.clone(), th.clone()
        tp[k] += np.pi / 2
        tm[k] -= np.pi / 2
        shift = 0.5 * (ctx.energy(tp) - ctx.energy(tm)).item()
        assert abs(g_ad[k] - shift) <= 1e-10 * max(1.0, abs(shift))
        eps = 1e-5
        tp, tm = th.clone(), th.clone()
        tp[k] += eps
        tm[k] -= eps
        fd = (ctx.energy(tp) - ctx.energy(tm)).item() / (2 * eps)
        assert abs(g_ad[k] - fd) <= 1e-7 * max(1.0, abs(fd))


@pytest.fixture(scope="module")
def rand28_ref(oracle):
    p = W.config_rand28(precision=W.C64)
    idx = np.array([17, 200], dtype=np.int32)
    return p, idx, oracle.sampled(p, idx)


def test_rand28_c64_sampled(qng, rand28_ref):
    p, idx, ref = rand28_ref
    check_step(qng, ref, p, idx, 2e-4)


@pytest.mark.skipif(os.environ.get("QNG_FULL28_C128") != "1", reason="two minutes of GPU time; QNG_FULL28_C128=1")
def test_rand28_c128_sampled(qng, rand28_ref):
    p, idx, ref = rand28_ref
    p128 = W.Problem(p.name.replace("c64", "c128"), p.circuit, p.hamiltonian, p.theta, precision=W.C128)
    check_step(qng, ref, p128, idx, 1e-10)
