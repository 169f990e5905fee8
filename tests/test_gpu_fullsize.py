"""Parity at the full sizes of the 26- and 28-qubit workloads (streaming path, 1-4 GiB per state).

The oracle cannot build all P derivative states at these sizes (208 and 252 states of 1-4 GiB), so
it evaluates the definitions on a seeded subset S of 8 parameters (the first, the last, and the
first and last of every layer boundary between): G_ab, T_a and d<E>/d theta_a for a, b in S, and
<E>. Entries outside S are checked through properties that hold at any size: the metric is
symmetric, dtheta solves (g + lambda I) dtheta = -dt grad to float64 accuracy, and the reverse-sweep
gradient (through torch.autograd) equals the parameter-shift rule and central finite differences of
GPU energies on sampled parameters. At 28 qubits the complex64 run is also compared with the
complex128 run element by element over the whole of g, grad and dtheta (the error of the complex64
path against the float64 path).
"""
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


def run_step(qng, p):
    ctx = qng.Context(p)
    th = ctx.theta0()
    out = ctx.step(th, p.dt, p.lam)
    ctx.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return ctx, th, res


def check_step(res, p, oracle_ref, idx, tol):
    g = res["g"].reshape(p.P, p.P)
    grad = res["grad"]
    dth = res["dtheta"]
    E = float(res["energy"][0])
    Gs, Ts, grads, Eo = oracle_ref
    assert rel(g[np.ix_(idx, idx)], Gs.real) <= tol
    assert rel(grad[idx], grads) <= tol
    assert rel([E], [Eo]) <= tol
    # properties of the whole outputs
    assert np.abs(g - g.T).max() == 0.0
    A = g + p.lam * np.eye(p.P)
    r = A @ dth + p.dt * grad
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.dt * grad)


def layer_sample(P, per_layer):
    """8 parameters: the first, the last, and the first and last of the layers between."""
    idx = {0, P - 1}
    for L in range(1, P // per_layer):
        idx |= {L * per_layer - 1, L * per_layer}
    idx = sorted(idx)
    while len(idx) > 8:  # keep the ends, thin the middle
        idx.pop(len(idx) // 2)
    mid = P // 2
    while len(idx) < 8:
        if mid not in idx:
            idx.append(mid)
        mid += 1
    return np.array(sorted(idx), dtype=np.int32)


@pytest.fixture(scope="module")
def tfim26_ref(oracle):
    p = W.config_tfim26()
    idx = layer_sample(p.P, 2 * p.circuit.n)
    return p, idx, oracle.sampled(p, idx)


def test_tfim26_c128_sampled_and_autograd(qng, tfim26_ref):
    p, idx, ref = tfim26_ref
    assert len(idx) == 8
    ctx, th, res = run_step(qng, p)
    check_step(res, p, ref, idx, 1e-10)
    # torch.autograd through the reverse sweep vs parameter shift and central differences (eps 1e-5)
    theta = th.clone().requires_grad_(True)
    E = qng.energy(theta, ctx)
    E.sum().backward()
    g_ad = theta.grad.cpu().numpy()
    assert rel(g_ad, res["grad"]) <= 1e-12
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
    ctx.close()


@pytest.fixture(scope="module")
def rand28_ref(oracle):
    p = W.config_rand28(precision=W.C64)
    idx = layer_sample(p.P, 3 * p.circuit.n)
    return p, idx, oracle.sampled(p, idx)


@pytest.fixture(scope="module")
def rand28_runs(qng):
    """The 28-qubit step in complex64 and complex128 (GPU), each run once for the tests below."""
    p64 = W.config_rand28(precision=W.C64)
    p128 = W.Problem(p64.name.replace("c64", "c128"), p64.circuit, p64.hamiltonian, p64.theta, precision=W.C128)
    out = {}
    for p in (p64, p128):
        ctx, _, res = run_step(qng, p)
        ctx.close()
        out[p.precision] = (p, res)
    return out


def test_rand28_c64_sampled(rand28_runs, rand28_ref):
    p, idx, ref = rand28_ref
    assert len(idx) == 8
    p64, res = rand28_runs[W.C64]
    check_step(res, p64, ref, idx, 2e-4)


def test_rand28_c128_sampled(rand28_runs, rand28_ref):
    p, idx, ref = rand28_ref
    p128, res = rand28_runs[W.C128]
    check_step(res, p128, ref, idx, 1e-10)


def test_rand28_c64_against_c128(rand28_runs):
    """The complex64 path against the float64 path over every entry of g, grad and dtheta: within the
    complex64 tolerance for g and grad; dtheta solves (g + lambda I) dtheta = -dt grad, whose small
    eigenvalues (lambda = 1e-3) amplify the complex64 error of g and grad, so its bound is the
    complex64 tolerance times the condition number of g + lambda I."""
    p, r64 = rand28_runs[W.C64]
    _, r128 = rand28_runs[W.C128]
    errs = {k: rel(r64[k], r128[k]) for k in ("g", "grad", "dtheta", "energy")}
    print("rand28 complex64 vs complex128 relative max-abs error:", errs)
    assert errs["g"] <= 2e-4 and errs["grad"] <= 2e-4 and errs["energy"] <= 2e-4
    g = r128["g"].reshape(p.P, p.P)
    cond = np.linalg.cond(g + p.lam * np.eye(p.P))
    assert errs["dtheta"] <= 2e-4 * cond
