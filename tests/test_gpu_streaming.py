"""GPU parity of the streaming path (state vectors in HBM, tiled passes) against the CPU oracle.

Small and medium instances are forced onto the streaming path and checked entry by entry; tiles of
2^11 (complex128) or 2^12 (complex64) amplitudes make instances of 13-16 qubits span many tiles and
many passes per column, with window qubits changing from pass to pass.
"""
import numpy as np
import pytest
import torch

from paper_2011_02991_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {W.C128: 1e-10, W.C64: 2e-4}


def rel(got, ref):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)) if ref.size else 0.0


@pytest.fixture(scope="module")
def qng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_02991_gb300 import build as B
    B.build()
    from paper_2011_02991_gb300 import qng as Q
    return Q


def run_streaming(qng, oracle, p, precision):
    ctx = qng.Context(p, precision=precision, path=2)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    g2, sig = ctx.metric(ctx.theta0(), want_sigma=True)
    gr, en = ctx.gradient(ctx.theta0())
    ctx.sync()
    ref = oracle.qng_step(p)
    t = TOL[precision]
    errs = {"g": rel(out["g"].cpu(), ref["g"]), "grad": rel(out["grad"].cpu(), ref["grad"]),
            "dtheta": rel(out["dtheta"].cpu(), ref["dtheta"]), "E": rel(out["energy"].cpu(), [ref["E"]]),
            "g_metric_call": rel(g2.cpu(), ref["g"]), "sigma": rel(sig.cpu(), -2.0 * ref["T"].imag),
            "grad_call": rel(gr.cpu(), ref["grad"]), "E_grad_call": rel(en.cpu(), [ref["E"]])}
    bad = {k: v for k, v in errs.items() if not v <= t}
    assert not bad, f"{p.name} precision={precision}: {bad}"


@pytest.mark.parametrize("precision", [W.C128, W.C64])
def test_streaming_small_configs(qng, oracle, precision):
    run_streaming(qng, oracle, W.config_tfim4() if precision == W.C128 else
                  W.Problem("tfim4_c64", W.config_tfim4().circuit, W.config_tfim4().hamiltonian,
                            W.config_tfim4().theta, precision=W.C64), precision)


@pytest.mark.parametrize("precision", [W.C128, W.C64])
@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2), (12, 5), (13, 3), (15, 4), (17, 6)])
def test_streaming_random_circuits(qng, oracle, n, seed, precision):
    """Every gate kind, on instances that span 1 to 64 tiles (complex64 from 12 qubits on runs the
    register-phase kernel: one tile at 12 qubits, 32 tiles over 152 CTAs at 17)."""
    p = W.random_problem(n, 50 + 4 * n, 10, 3000 + seed, precision)
    run_streaming(qng, oracle, p, precision)


@pytest.mark.parametrize("precision", [W.C128, W.C64])
def test_streaming_layered_14(qng, oracle, precision):
    """Ry/Rz/CZ and Ry/Rx/Rz/CNOT layers at 14 qubits (the ansatz families of the 26/28-qubit workloads)."""
    rng = np.random.Generator(np.random.PCG64(77))
    c = W.layered_ansatz(14, 2)
    p = W.Problem("layered14", c, W.tfim_chain(14, 1.0, rng.uniform(0.2, 1.0, 14)), W.uniform_theta(c.num_params, rng),
                  precision=precision)
    run_streaming(qng, oracle, p, precision)
    c = W.layered_ansatz(14, 2, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)
    p = W.Problem("layered14_cnot", c, W.random_pauli_hamiltonian(14, 20, rng), W.uniform_theta(c.num_params, rng),
                  precision=precision)
    run_streaming(qng, oracle, p, precision)


@pytest.mark.parametrize("n,seed", [(12, 21), (14, 22)])
def test_streaming_c64_diagonal_runs(qng, oracle, n, seed):
    """Runs of 1-24 RZ steps with CZ / Z gates between them, some broken by a CNOT or H, at complex64
    from 12 qubits: the register-phase kernel takes each run's inner products on its starting
    registers and applies the run's rotations and signs as one composed factor per amplitude. Real
    step and complex metric (Re and Im per step) against the oracle."""
    p = W.z_run_problem(n, 160, seed, W.C64)
    run_streaming(qng, oracle, p, W.C64)
    ctx = qng.Context(p, precision=W.C64, path=2)
    G = ctx.metric_complex(ctx.theta0()).reshape(p.P, p.P).cpu().numpy()
    ctx.sync()
    ref = oracle.qng_step(p)["G"]
    assert float(np.abs(G - ref).max() / np.abs(ref).max()) <= TOL[W.C64]
    assert np.all(G.imag == -G.imag.T)


def test_streaming_long_circuit_renormalisation(qng, oracle):
    """P = 600 with angles near pi/2: the register scales fall below 2^-200 and are renormalised."""
    run_streaming(qng, oracle, W.z_run_problem(7, 600, 6, W.C128, near_half_pi=True), W.C128)


def test_streaming_matches_onchip(qng):
    """The two paths agree on the 12-qubit, P = 192 workload."""
    p = W.config_rand12()
    a = qng.Context(p, path=1)
    b = qng.Context(p, path=2)
    oa = a.step(a.theta0(), p.dt, p.lam)
    ob = b.step(b.theta0(), p.dt, p.lam)
    a.sync()
    b.sync()
    for k in ("g", "grad", "dtheta", "energy"):
        assert rel(ob[k].cpu(), oa[k].cpu()) <= 1e-11, k


@pytest.mark.parametrize("seed", [11, 12])
def test_streaming_c64_matches_onchip_c64(qng, seed):
    """Complex64 at 12-14 qubits: the register-phase streaming kernel against the on-chip path, both
    at complex64, on g, grad and <E> (within the complex64 tolerance of each other)."""
    n = 12 + seed % 3
    p = W.random_problem(n, 140, 16, 4100 + seed, W.C64)
    a = qng.Context(p, path=1)
    b = qng.Context(p, path=2)
    ga, sa = a.metric(a.theta0(), want_sigma=True)
    gb, sb = b.metric(b.theta0(), want_sigma=True)
    ra, ea = a.gradient(a.theta0())
    rb, eb = b.gradient(b.theta0())
    a.sync()
    b.sync()
    assert rel(gb.cpu(), ga.cpu()) <= TOL[W.C64]
    assert rel(sb.cpu(), sa.cpu()) <= TOL[W.C64]
    assert rel(rb.cpu(), ra.cpu()) <= TOL[W.C64]
    assert rel(eb.cpu(), ea.cpu()) <= TOL[W.C64]


@pytest.mark.parametrize("precision", [W.C128, W.C64])
def test_column_partition_streaming(qng, oracle, precision):
    """The column partition on the streaming path: a rank's schedule runs the recurrence for its
    columns and only advances psi through the others' gates; merged, the parts give the same step
    as the unpartitioned schedule (psi takes the same operations in either schedule)."""
    from paper_2011_02991_gb300 import dist as D
    n = 14 if precision == W.C128 else 13
    rng = np.random.Generator(np.random.PCG64(515))
    c = W.layered_ansatz(n, 2, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)
    p = W.Problem("partition_stream", c, W.random_pauli_hamiltonian(n, 12, rng), W.uniform_theta(c.num_params, rng),
                  precision=precision)
    full = qng.Context(p, path=2)
    ref = full.step(full.theta0(), p.dt, p.lam)
    full.sync()
    ranks = 3
    owner = D.column_owners(p.P, ranks)
    Ls, ss, grads = [], [], []
    for r in range(ranks):
        ctx = qng.Context(p, path=2)
        ctx.set_column_subset(qng.column_partition(p.P, ranks, r))
        parts = ctx.metric_columns(ctx.theta0())
        ctx.sync()
        Ls.append(parts["L"])
        ss.append(parts["sigma"])
        grads.append(parts["grad"])
        ctx.close()
    L, sigma = D.merge_columns(Ls, ss, owner)
    out = full.step_from_parts(full.theta0(), L.reshape(-1), sigma, grads[0], p.dt, p.lam)
    full.sync()
    assert torch.equal(out["g"], ref["g"])
    assert torch.equal(out["dtheta"], ref["dtheta"])
    assert rel(out["g"].cpu(), oracle.qng_step(p)["g"]) <= TOL[precision]
