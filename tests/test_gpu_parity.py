"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerance: relative max-abs error err(x) = max_k |x_k - x_k^o| / max_k |x_k^o|, at most 1e-10 for
complex128 paths and 2e-4 for complex64 paths, applied separately to g, grad<E>, dtheta and <E>.
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


def check_problem(qng, oracle, p, precision, tuning=None, tol=None):
    ctx = qng.Context(p, precision=precision)
    if tuning is not None:
        ctx.set_tuning(*tuning)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    g_s, sig = ctx.metric(ctx.theta0(), want_sigma=True)
    ctx.sync()
    ref = oracle.qng_step(p)
    t = TOL[precision] if tol is None else tol
    errs = {
        "g": rel(out["g"].cpu(), ref["g"]),
        "grad": rel(out["grad"].cpu(), ref["grad"]),
        "dtheta": rel(out["dtheta"].cpu(), ref["dtheta"]),
        "E": rel(out["energy"].cpu(), [ref["E"]]),
        "g_metric_call": rel(g_s.cpu(), ref["g"]),
        "sigma": rel(sig.cpu(), -2.0 * ref["T"].imag),  # T_k = -(i/2) sigma_k
    }
    bad = {k: v for k, v in errs.items() if not v <= t}
    assert not bad, f"{p.name} precision={precision} tuning={tuning}: {bad} (tol {t})"
    return errs


def test_config_tfim4_c128(qng, oracle):
    check_problem(qng, oracle, W.config_tfim4(), W.C128)


@pytest.mark.parametrize("precision", [W.C128, W.C64])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_circuits_all_gate_kinds(qng, oracle, seed, precision):
    """Every gate kind (Rx/Ry/Rz, CZ, CNOT, X, Y, Z, H), fixed gates before, between and after."""
    p = W.random_problem(6, 60, 12, 500 + seed, precision)
    check_problem(qng, oracle, p, precision)


@pytest.mark.parametrize("cl", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", [W.C128, W.C64])
def test_cluster_distribution(qng, oracle, cl, precision):
    """The same circuit with the state split over 1, 2, 4, 8 CTAs (distributed top qubits)."""
    p = W.random_problem(7, 70, 10, 900, precision)
    check_problem(qng, oracle, p, precision, tuning=(0, cl, 64))


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_cta_sizes(qng, oracle, threads):
    p = W.random_problem(8, 50, 8, 77, W.C128)
    check_problem(qng, oracle, p, W.C128, tuning=(0, 1, threads))


@pytest.mark.parametrize("precision", [W.C64, W.C128])
@pytest.mark.parametrize("fwd_threads", [64, 96, 128, 256, 512])
def test_z_runs_forward_shapes(qng, oracle, precision, fwd_threads):
    """Runs of Z rotations with diagonal fixed blocks go through the checkpoint sweep in one pass
    each: 8, 4, 2 and 1 amplitudes per thread (512 per CTA), and 96 threads (no whole number of
    amplitudes per thread: one rotation at a time)."""
    p = W.z_run_problem(10, 160, 5, precision)
    ctx = qng.Context(p, precision=precision)
    ctx.set_forward_cluster(10, 1)
    ctx.set_shape(10, 1, 128, fwd_threads)
    assert ctx.get_tuning(10) == (1, 128, fwd_threads) and ctx.forward_cluster(10) == 1
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    ref = oracle.qng_step(p)
    for key in ("g", "grad"):
        assert rel(out[key].cpu(), ref[key]) <= TOL[precision], key
    if precision == W.C128:
        assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[precision]
    else:
        # Z rotations on Z eigenstates leave directions with g ~ 0 and an exactly zero gradient:
        # there complex64 rounding of the gradient (~1e-8) is divided by lambda. The step is
        # checked as the solution of its own float64 system instead.
        g = out["g"].cpu().numpy().reshape(p.P, p.P)
        res = (g + p.lam * np.eye(p.P)) @ out["dtheta"].cpu().numpy() + p.dt * out["grad"].cpu().numpy()
        assert np.linalg.norm(res) <= 1e-10 * p.dt * np.linalg.norm(out["grad"].cpu().numpy())


def test_z_runs_small_state(qng, oracle):
    """64 amplitudes and a 128-thread sweep: more threads than amplitudes."""
    p = W.z_run_problem(6, 120, 7, W.C128)
    ctx = qng.Context(p, precision=W.C128)
    ctx.set_shape(6, 0, 64, 128)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    ref = oracle.qng_step(p)
    assert rel(out["g"].cpu(), ref["g"]) <= TOL[W.C128]
    assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[W.C128]


def test_z_runs_long_circuit_renormalisation(qng, oracle):
    """P = 1000 on 7 qubits (2 amplitudes per thread in the sweep): the float64 scale of the scaled
    complex128 rotations falls below 2^-200 several times, also around Z runs. Angles near pi/2
    make every factor max(|cos|, |sin|) of a half angle close to 2^-1/2 and mix both forms."""
    p = W.z_run_problem(7, 1000, 6, W.C128, near_half_pi=True)
    ctx = qng.Context(p, precision=W.C128)
    ctx.set_shape(7, 0, 64, 64)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    ref = oracle.qng_step(p)
    for key in ("g", "grad", "dtheta"):
        assert rel(out[key].cpu(), ref[key]) <= TOL[W.C128], key
    assert rel(out["energy"].cpu(), [ref["E"]]) <= TOL[W.C128]


def test_config_rand12_c128_full(qng, oracle):
    """The 12-qubit, P = 192 workload, every entry against the oracle."""
    check_problem(qng, oracle, W.config_rand12(), W.C128)


def test_config_rand12_c64_full(qng, oracle):
    check_problem(qng, oracle, W.config_rand12(precision=W.C64), W.C64)


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_batch_subset_every_instance(qng, oracle, precision):
    probs = [p for p in W.config_batch(count=24, precision=precision)]
    ctx = qng.Context(probs, precision=precision)
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    gs, grads, dths = ctx.split_metric(out["g"]), ctx.split_params(out["grad"]), ctx.split_params(out["dtheta"])
    for b, p in enumerate(probs):
        ref = oracle.qng_step(p)
        t = TOL[precision]
        assert rel(gs[b].cpu(), ref["g"]) <= t, (b, p.name)
        assert rel(grads[b].cpu(), ref["grad"]) <= t, (b, p.name)
        assert rel(dths[b].cpu(), ref["dtheta"]) <= t, (b, p.name)
        assert rel(out["energy"][b:b + 1].cpu(), [ref["E"]]) <= t, (b, p.name)


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_batch256_sampled_instances(qng, oracle, precision):
    """The full 256-instance batch in one launch per group; 12 instances checked against the oracle."""
    probs = W.config_batch(precision=precision)
    ctx = qng.Context(probs, precision=precision)
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    gs, grads, dths = ctx.split_metric(out["g"]), ctx.split_params(out["grad"]), ctx.split_params(out["dtheta"])
    rng = np.random.default_rng(5)
    pick = sorted(set(rng.choice(len(probs), 10, replace=False).tolist())
                  | {int(np.argmax([p.n * 1000 + p.P for p in probs])), int(np.argmin([p.P for p in probs]))})
    t = TOL[precision]
    for b in pick:
        p = probs[b]
        ref = oracle.qng_step(p)
        assert rel(gs[b].cpu(), ref["g"]) <= t, (b, p.name)
        assert rel(grads[b].cpu(), ref["grad"]) <= t, (b, p.name)
        assert rel(dths[b].cpu(), ref["dtheta"]) <= t, (b, p.name)


def test_energy_autograd_backward(qng, oracle):
    p = W.random_problem(9, 80, 15, 1234, W.C128)
    ctx = qng.Context(p)
    theta = ctx.theta0().requires_grad_(True)
    E = qng.energy(theta, ctx)
    (3.0 * E.sum()).backward()
    grad_ref, E_ref = oracle.gradient(p.circuit, p.hamiltonian, p.theta)
    assert rel(E.detach().cpu(), [E_ref]) <= 1e-10
    assert rel(theta.grad.cpu() / 3.0, grad_ref) <= 1e-10


def test_gradient_vs_parameter_shift_on_gpu(qng):
    """d<E>/d theta from the reverse sweep equals the parameter-shift rule on GPU energies."""
    p = W.random_problem(7, 40, 10, 4321, W.C128)
    ctx = qng.Context(p)
    th = ctx.theta0()
    grad, _ = ctx.gradient(th)
    shifts = []
    for k in range(p.P):
        tp, tm = th.clone(), th.clone()
        tp[k] += np.pi / 2
        tm[k] -= np.pi / 2
        shifts.append(0.5 * (ctx.energy(tp) - ctx.energy(tm)).item())
    assert rel(grad.cpu(), shifts) <= 1e-10


def test_edge_cases(qng, oracle):
    # only fixed gates: P = 0, energy only
    c = W.Circuit(3, np.array([[W.H, 0, -1, -1], [W.CNOT, 0, 1, -1], [W.X, 2, -1, -1]], dtype=np.int32))
    ham = W.tfim_chain(3, 1.0, 0.5)
    p = W.Problem("fixed_only", c, ham, np.zeros(0))
    ctx = qng.Context(p)
    E = ctx.energy(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert rel(E.cpu(), [oracle.energy(c, ham, np.zeros(0))]) <= 1e-12
    # one qubit, one parameter
    c = W.Circuit(1, np.array([[W.RY, 0, -1, 0]], dtype=np.int32))
    p = W.Problem("one", c, W.hamiltonian_from_terms([(0.7, {0: "Z"}), (0.3, {0: "X"})]), np.array([0.9]))
    check_problem(qng, oracle, p, W.C128)
    # trailing fixed gates with H (W is part of psi and of <E>) and leading fixed gates
    base = W.config_tfim4()
    extra = np.array([[W.H, 0, -1, -1], [W.CNOT, 0, 3, -1], [W.Y, 2, -1, -1]], dtype=np.int32)
    lead = np.array([[W.H, 1, -1, -1], [W.CZ, 1, 2, -1]], dtype=np.int32)
    c2 = W.Circuit(4, np.concatenate([lead, base.circuit.gates, extra]))
    check_problem(qng, oracle, W.Problem("lead_trail", c2, base.hamiltonian, base.theta), W.C128)


def test_not_spd_reported(qng):
    """lambda = 0 with a singular metric (Rz first on |0> gives g_00 = 0) reports QNG_ERR_NOT_SPD."""
    c = W.Circuit(2, np.array([[W.RZ, 0, -1, 0], [W.RY, 1, -1, 1]], dtype=np.int32))
    p = W.Problem("singular", c, W.tfim_chain(2), np.array([0.3, 0.4]))
    ctx = qng.Context(p)
    ctx.step(ctx.theta0(), 0.1, 0.0)
    with pytest.raises(qng.QngError) as e:
        ctx.sync()
    assert e.value.status == qng.QNG_ERR_NOT_SPD
    ctx.sync()  # the status word is cleared after being reported
    ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()


def test_nonfinite_theta_reported(qng):
    p = W.config_tfim4()
    ctx = qng.Context(p)
    th = ctx.theta0()
    th[3] = float("nan")
    ctx.metric(th)
    with pytest.raises(qng.QngError) as e:
        ctx.sync()
    assert e.value.status == qng.QNG_ERR_ARG


def test_step_host_matches_device(qng, oracle):
    p = W.config_rand12()
    ctx = qng.Context(p)
    dev = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    host = ctx.step_host(p.theta, p.dt, p.lam)
    np.testing.assert_array_equal(host["dtheta"], dev["dtheta"].cpu().numpy())
    np.testing.assert_array_equal(host["g"], dev["g"].cpu().numpy())


def test_deterministic(qng):
    p = W.config_rand12()
    ctx = qng.Context(p)
    a = ctx.step(ctx.theta0(), p.dt, p.lam)
    a = {k: v.clone() for k, v in a.items()}
    b = ctx.step(ctx.theta0(), p.dt, p.lam)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_graph_capture_replay(qng):
    """One captured CUDA graph of the whole step replays to the same results as the direct calls."""
    for probs in (W.config_rand12(), W.config_batch(count=12)):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = qng.Context(probs, stream=stream)
            th = ctx.theta0()
            ref = ctx.step(th, 0.1, 1e-3)
            ctx.sync()
            ref = {k: v.clone() for k, v in ref.items()}
            out = ctx.graph_capture(th, 0.1, 1e-3)
            for _ in range(2):
                for v in out.values():
                    v.fill_(float("nan"))
                ctx.graph_launch()
                ctx.sync()
                for k in ref:
                    assert torch.equal(out[k], ref[k]), k


def test_autotune_keeps_results(qng, oracle):
    """The autotuner sweeps launch shapes per qubit count; results stay within tolerance."""
    probs = W.config_batch(count=16, precision=W.C64)
    ctx = qng.Context(probs, precision=W.C64)
    tried = ctx.autotune(ctx.theta0(), reps=1)
    assert tried >= len({p.n for p in probs})
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    gs, dths = ctx.split_metric(out["g"]), ctx.split_params(out["dtheta"])
    for b in (0, 5, 11, 15):
        ref = oracle.qng_step(probs[b])
        assert rel(gs[b].cpu(), ref["g"]) <= TOL[W.C64]
        assert rel(dths[b].cpu(), ref["dtheta"]) <= TOL[W.C64]
    for n in {p.n for p in probs}:
        cl, th, fth = ctx.get_tuning(n)
        assert 0 <= cl <= 3 and th in (64, 128, 256) and fth in (64, 128, 256, 512)


def test_z_runs_complex_metric_and_gradient_c64(qng, oracle):
    """complex64 column walks through long runs of Z rotations (9 qubits, 2 CTAs, 4 amplitudes per
    thread): Re and Im of G, and the gradient column, against the oracle."""
    p = W.z_run_problem(9, 240, 3, W.C64)
    check_complex(qng, oracle, p, W.C64, shape=(9, 1, 64, 0))
    ctx = qng.Context(p, precision=W.C64)
    ctx.set_shape(9, 1, 64, 0)
    gr, en = ctx.gradient(ctx.theta0())
    ctx.sync()
    ref = oracle.qng_step(p)
    assert rel(gr.cpu(), ref["grad"]) <= TOL[W.C64]


def check_complex(qng, oracle, probs, precision, shape=None):
    """qng_metric_complex against the oracle's G (Eq. 4), Re and Im, every instance."""
    probs = probs if isinstance(probs, list) else [probs]
    ctx = qng.Context(probs if len(probs) > 1 else probs[0], precision=precision)
    if shape is not None:
        ctx.set_shape(*shape)
    G, sg = ctx.metric_complex(ctx.theta0(), want_sigma=True)
    ctx.sync()
    Gs = ctx.split_metric(G) if len(probs) > 1 else [G.reshape(probs[0].P, probs[0].P)]
    for b, p in enumerate(probs):
        ref = oracle.qng_step(p)["G"]
        Gb = Gs[b].cpu().numpy().reshape(p.P, p.P)
        err = float(np.abs(Gb - ref).max() / np.abs(ref).max())
        assert err <= TOL[precision], f"{p.name}: {err}"
        assert np.all(Gb.imag == -Gb.imag.T) and np.all(np.diag(Gb.imag) == 0.0)
    return ctx


def test_metric_complex_closed_form(qng):
    """RY(a) RZ(b) on one qubit: G_01 = i sin(a)/4."""
    bld = W._CircuitBuilder(1)
    bld.rot(W.RY, 0)
    bld.rot(W.RZ, 0)
    p = W.Problem("ryrz", bld.build(), W.hamiltonian_from_terms([(1.0, {0: "Z"})]), np.array([0.7, -1.3]))
    ctx = qng.Context(p, precision=W.C128)
    G = ctx.metric_complex(ctx.theta0()).reshape(2, 2).cpu().numpy()
    ctx.sync()
    assert abs(G[0, 1] - 0.25j * np.sin(0.7)) < 1e-15


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_metric_complex_configs(qng, oracle, precision):
    check_complex(qng, oracle, W.config_tfim4(), precision)
    check_complex(qng, oracle, W.config_rand12(precision=precision), precision)


@pytest.mark.parametrize("cl", [0, 1, 2, 3])
def test_metric_complex_every_gate_kind_distributed(qng, oracle, cl):
    """Every gate kind, with 0..3 of the qubits distributed over the cluster."""
    p = W.random_problem(7, 90, 10, 910 + cl, W.C128)
    check_complex(qng, oracle, p, W.C128, shape=(7, cl, 64, 64))


def test_metric_complex_renormalisation(qng, oracle):
    check_complex(qng, oracle, W.z_run_problem(7, 600, 6, W.C128, near_half_pi=True), W.C128, shape=(7, 0, 64, 64))


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_metric_complex_batch(qng, oracle, precision):
    """A batch with several launch shapes, through the persistent column launch."""
    probs = [p for p in W.config_batch(count=12, precision=precision)]
    ctx = check_complex(qng, oracle, probs, precision)
    # the real part is qng_metric's metric up to the grouping of the warp sums (4 steps per
    # reduction instead of 8), i.e. float32 rounding for complex64
    g = ctx.metric(ctx.theta0())
    G = ctx.metric_complex(ctx.theta0())
    ctx.sync()
    assert rel(G.real.cpu(), g.cpu()) <= (1e-13 if precision == W.C128 else 1e-5)


@pytest.mark.parametrize("precision", [W.C64, W.C128])
@pytest.mark.parametrize("n,seed", [(6, 1), (13, 3)])
def test_metric_complex_streaming(qng, oracle, precision, n, seed):
    """The streaming path's complex schedule: every gate kind, 1 and 4 tiles (two slots per step)."""
    p = W.random_problem(n, 50 + 4 * n, 10, 3000 + seed, precision)
    ctx = qng.Context(p, precision=precision, path=2)
    G = ctx.metric_complex(ctx.theta0()).reshape(p.P, p.P).cpu().numpy()
    g = ctx.metric(ctx.theta0()).reshape(p.P, p.P).cpu().numpy()  # the real-only schedule after it
    ctx.sync()
    ref = oracle.qng_step(p)["G"]
    assert float(np.abs(G - ref).max() / np.abs(ref).max()) <= TOL[precision]
    assert np.all(G.imag == -G.imag.T)
    assert rel(g, ref.real) <= TOL[precision]


def test_optimize_matches_oracle_loop(qng, oracle):
    """qng_optimize's trajectory = the oracle's step iterated on the CPU (10 steps, tfim4)."""
    p = W.config_tfim4()
    ctx = qng.Context(p, precision=W.C128)
    th = ctx.theta0().clone()
    en = ctx.optimize(th, p.dt, p.lam, 10)
    ctx.sync()
    t_ref = p.theta.copy()
    e_ref = []
    for _ in range(10):
        r = oracle.qng_step(W.Problem(p.name, p.circuit, p.hamiltonian, t_ref, p.dt, p.lam))
        e_ref.append(r["E"])
        t_ref = t_ref + r["dtheta"]
    assert rel(th.cpu(), t_ref) <= 1e-10
    assert rel(en[:, 0].cpu(), e_ref) <= 1e-10


def test_optimize_batch_matches_steps(qng):
    """In a batch every instance follows its own qng_step iteration (host loop vs device loop)."""
    probs = [p for p in W.config_batch(count=6, precision=W.C128)]
    ctx = qng.Context(probs, precision=W.C128)
    th = ctx.theta0().clone()
    en = ctx.optimize(th, 0.1, 1e-3, 4)
    t2 = ctx.theta0().clone()
    e2 = []
    for _ in range(4):
        out = ctx.step(t2, 0.1, 1e-3)
        e2.append(out["energy"].clone())
        t2 = t2 + out["dtheta"]
    ctx.sync()
    assert torch.equal(th, t2)
    assert torch.equal(en, torch.stack(e2))


@pytest.mark.parametrize("n,layers,iters,rel_gap", [(6, 4, 300, 2e-3), (10, 5, 200, 5e-3), (12, 6, 300, 2e-3)])
def test_optimize_tfim_reaches_ground_energy(qng, oracle, n, layers, iters, rel_gap):
    """Natural-gradient descent on the open TFIM chain (J = 1, h = 0.7) from small angles reaches
    the exact ground energy (Lanczos on the oracle's H|v>) to within the ansatz's reach."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    ham = W.tfim_chain(n, 1.0, 0.7)
    N = 1 << n
    op = LinearOperator((N, N), matvec=lambda v: oracle.hamiltonian_apply(np.asarray(v, complex).ravel(), ham),
                        dtype=complex)
    E0 = float(eigsh(op, k=1, which="SA")[0][0])
    p = W.vqe_tfim(n, layers)
    c = p.circuit
    ctx = qng.Context(p, precision=W.C128)
    th = ctx.theta0().clone()
    en = ctx.optimize(th, 0.1, 1e-3, iters)[:, 0].cpu().numpy()
    ctx.sync()
    assert en[0] > 0.0 > E0
    assert en[-1] >= E0 - 1e-9  # variational bound
    assert (en[-1] - E0) / abs(E0) <= rel_gap
    # the final energy is the energy of the final parameters
    e_fin = ctx.energy(th)
    ctx.sync()
    assert abs(float(e_fin[0]) - oracle.energy(c, ham, th.cpu().numpy())) <= 1e-10 * abs(E0)


def _rand_params(n, P, seed, precision=W.C128):
    """A random circuit on n qubits with exactly P rotations (every gate kind)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bld = W._CircuitBuilder(n)
    while bld.P < P:
        if rng.random() < 0.35:
            kind = int(rng.choice([W.CZ, W.CNOT, W.X, W.Y, W.Z, W.H]))
            if kind in (W.CZ, W.CNOT):
                q0, q1 = rng.choice(n, size=2, replace=False)
                bld.fixed(kind, int(q0), int(q1))
            else:
                bld.fixed(kind, int(rng.integers(n)))
        else:
            bld.rot(int(rng.choice([W.RX, W.RY, W.RZ])), int(rng.integers(n)))
    c = bld.build()
    return W.Problem(f"rand_n{n}_p{P}", c, W.random_pauli_hamiltonian(n, 12, rng), W.uniform_theta(P, rng),
                     precision=precision)


@pytest.mark.parametrize("P", [340, 401, 600])
def test_block_solve_large_P(qng, oracle, P):
    """Beyond the cluster solve's shared memory (P > ~330) a single instance is solved one 16-column
    block per launch with the factor in global memory: ragged last blocks, every gate kind."""
    p = _rand_params(7, P, 4000 + P)
    ref = oracle.qng_step(p)
    ctx = qng.Context(p, precision=W.C128)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    for key in ("g", "grad", "dtheta"):
        assert rel(out[key].cpu(), ref[key]) <= TOL[W.C128], key
    assert rel(out["energy"].cpu(), [ref["E"]]) <= TOL[W.C128]
    A = out["g"].cpu().numpy().reshape(P, P) + p.lam * np.eye(P)
    r = A @ out["dtheta"].cpu().numpy() + p.dt * out["grad"].cpu().numpy()
    assert np.linalg.norm(r) <= 1e-10 * p.dt * np.linalg.norm(out["grad"].cpu().numpy())


def test_block_solve_not_spd(qng, oracle):
    """lambda = 0 and a last rotation RZ on an untouched qubit (|0>, <Z> = 1): g's last diagonal
    entry is exactly 0, the first pivot of the block factorisation (reversed order). The status
    word reports QNG_ERR_NOT_SPD, the later blocks and the back substitution stand down, and the
    next step runs."""
    base = _rand_params(2, 359, 77)
    extra = np.array([[W.RZ, 2, -1, 359]], dtype=np.int32)
    c = W.Circuit(3, np.concatenate([base.circuit.gates, extra]))
    p = W.Problem("singular_last", c, W.tfim_chain(3), np.concatenate([base.theta, [0.7]]))
    ctx = qng.Context(p)
    ctx.step(ctx.theta0(), 0.1, 0.0)
    with pytest.raises(qng.QngError) as e:
        ctx.sync()
    assert e.value.status == qng.QNG_ERR_NOT_SPD
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    ref = oracle.qng_step(W.Problem(p.name, c, p.hamiltonian, p.theta, 0.1, 1e-3))
    assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[W.C128]


@pytest.mark.parametrize("precision", [W.C64, W.C128])
@pytest.mark.parametrize("cl", [0, 1, 2, 3])
def test_generalised_rotations(qng, oracle, precision, cl):
    """Controlled rotations and (controlled) Pauli-string rotations (Sec. 2's generalised gates):
    K = C (x) S with the partner k ^ x in the CTA, in another CTA of the cluster (cl up to 3 puts
    three of the 7 qubits in the rank), or none (diagonal strings); every output against the oracle,
    the diagonal through <C_k>."""
    p = W.general_problem(7, 60, 700 + cl, precision)
    ctx = qng.Context(p, precision=precision)
    ctx.set_shape(7, cl, 64, 64)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    G = ctx.metric_complex(ctx.theta0())
    ctx.sync()
    ref = oracle.qng_step(p)
    for key in ("g", "grad"):
        assert rel(out[key].cpu(), ref[key]) <= TOL[precision], key
    assert rel(out["energy"].cpu(), [ref["E"]]) <= TOL[precision]
    if precision == W.C128:
        assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[precision]
    Gn = G.cpu().numpy().reshape(p.P, p.P)
    assert float(np.abs(Gn - ref["G"]).max() / np.abs(ref["G"]).max()) <= TOL[precision]


def test_generalised_rotations_larger(qng, oracle):
    """12 qubits, P = 150, 8-CTA clusters with 128 threads (the default shape)."""
    p = W.general_problem(12, 150, 777, W.C128)
    check_problem(qng, oracle, p, W.C128)


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_generalised_batch(qng, oracle, precision):
    """A batch mixing generalised and ordinary instances of 5..9 qubits (persistent column launch)."""
    probs = [W.general_problem(5 + b % 5, 20 + 4 * b, 800 + b, precision) if b % 2 == 0 else
             W.random_problem(5 + b % 5, 40 + 4 * b, 8, 820 + b, precision) for b in range(8)]
    ctx = qng.Context(probs, precision=precision)
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    gs, grads = ctx.split_metric(out["g"]), ctx.split_params(out["grad"])
    for b, p in enumerate(probs):
        ref = oracle.qng_step(p)
        assert rel(gs[b].cpu(), ref["g"]) <= TOL[precision], b
        assert rel(grads[b].cpu(), ref["grad"]) <= TOL[precision], b


def test_controlled_diagonal_on_gpu(qng):
    """H on the control, then CRY: g = (1/4) Prob(control = 1) - (1/4)<P1 (x) Y>^2 = 1/8 exactly."""
    b = W._CircuitBuilder(2)
    b.fixed(W.H, 0)
    b.crot(W.CRY, 0, 1)
    p = W.Problem("h_cry", b.build(), W.tfim_chain(2), np.array([0.9]))
    ctx = qng.Context(p, precision=W.C128)
    g = ctx.metric(ctx.theta0())
    ctx.sync()
    assert abs(float(g[0]) - 0.125) < 1e-15


def test_mixed_precision_solve_hands_over_not_spd(qng, oracle):
    """P = 100, lambda = 0 and a first rotation RZ on an untouched qubit: g_00 = 0 exactly, the first
    float32 pivot is not positive, the float64 cluster solve takes over and reports NOT_SPD; the
    next step (lambda = 1e-3) is solved in mixed precision and matches the oracle."""
    base = _rand_params(3, 99, 91)
    c = W.Circuit(4, np.concatenate([np.array([[W.RZ, 3, -1, 0]], dtype=np.int32),
                                     base.circuit.gates + np.array([0, 0, 0, 1], dtype=np.int32) * (base.circuit.gates[:, 3:4] >= 0)]))
    p = W.Problem("singular_first", c, W.tfim_chain(4), np.concatenate([[0.4], base.theta]))
    assert p.P == 100
    ctx = qng.Context(p)
    ctx.step(ctx.theta0(), 0.1, 0.0)
    with pytest.raises(qng.QngError) as e:
        ctx.sync()
    assert e.value.status == qng.QNG_ERR_NOT_SPD
    assert ctx.solve_report() == ("mixed", 1)
    out = ctx.step(ctx.theta0(), 0.1, 1e-3)
    ctx.sync()
    assert ctx.solve_report() == ("mixed", 0)
    ref = oracle.qng_step(W.Problem(p.name, c, p.hamiltonian, p.theta, 0.1, 1e-3))
    assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[W.C128]


@pytest.mark.parametrize("n,P,path", [(5, 40, "single"), (6, 120, "mixed"), (5, 222, "mixed"), (5, 223, "cluster"),
                                      (7, 340, "block")])
def test_solve_selection(qng, oracle, n, P, path):
    """Each solve the step can take matches the oracle's float64 step. The float32-factor solve
    takes every P from 48 up to the largest factor CTA 0's shared memory holds (222) and, at
    lambda = 1e-3 (condition numbers ~10^3), finishes without handing over to the float64 solve."""
    p = _rand_params(n, P, 5000 + P)
    ref = oracle.qng_step(p)
    ctx = qng.Context(p, precision=W.C128)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    assert ctx.solve_report() == (path, 0)
    for key in ("g", "grad", "dtheta"):
        assert rel(out[key].cpu(), ref[key]) <= TOL[W.C128], key


def test_bench_workload_solves_in_mixed_precision(qng, oracle):
    """12 qubits, P = 192 (the timed workload): the float32-factor solve finishes it alone."""
    p = W.config_rand12()
    ctx = qng.Context(p)
    out = ctx.step(ctx.theta0(), p.dt, p.lam)
    ctx.sync()
    assert ctx.solve_report() == ("mixed", 0)
    ref = oracle.qng_step(p)
    assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[W.C128]


@pytest.mark.parametrize("lam", [1e-6, 1e-9])
@pytest.mark.parametrize("which", ["rand12", "rand6_p200"])
def test_solve_ill_conditioned(qng, lam, which):
    """Small lambda makes g + lambda I nearly singular (float32 refinement stalls or its pivots
    fail, and the float64 solve takes over): the step still solves its float64 system, to the
    backward error of a float64 Cholesky solve and within cond(A) eps of LAPACK's solution."""
    p = W.config_rand12() if which == "rand12" else _rand_params(6, 200, 7200)
    ctx = qng.Context(p)
    out = ctx.step(ctx.theta0(), p.dt, lam)
    ctx.sync()
    g = out["g"].cpu().numpy().reshape(p.P, p.P)
    A = g + lam * np.eye(p.P)
    x = out["dtheta"].cpu().numpy()
    b = -p.dt * out["grad"].cpu().numpy()
    r = A @ x - b
    # backward error of a float64 Cholesky solve: |r| ~ eps |A| |x|
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(A, 2) * np.linalg.norm(x) + 1e-12 * np.linalg.norm(b)
    # forward error against LAPACK on the same float64 system: at most about cond(A) eps
    x_ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.abs(x - x_ref).max() <= 64 * cond * 2.0 ** -53 * np.abs(x_ref).max()


def test_live_contexts_of_different_sizes(qng, oracle):
    """Kernel attributes (the dynamic shared memory limit) are shared by every context of the
    process: creating a small context after a large one must leave the large one working."""
    big = W.config_rand12()
    ctx_big = qng.Context(big)
    small = W.config_tfim4()
    ctx_small = qng.Context(small)
    stream_big = W.random_problem(17, 30, 6, 4242)  # streaming path: its own pass kernels
    ctx_stream = qng.Context(stream_big)
    ref_big = oracle.qng_step(big)
    ref_small = oracle.qng_step(small)
    for _ in range(2):
        for ctx, p, ref in ((ctx_big, big, ref_big), (ctx_small, small, ref_small)):
            out = ctx.step(ctx.theta0(), p.dt, p.lam)
            ctx.sync()
            assert rel(out["g"].cpu(), ref["g"]) <= TOL[W.C128], p.name
            assert rel(out["dtheta"].cpu(), ref["dtheta"]) <= TOL[W.C128], p.name
        ctx_stream.metric(ctx_stream.theta0())
        ctx_stream.sync()


@pytest.mark.parametrize("ranks", [2, 3])
@pytest.mark.parametrize("which", ["rand12", "random6"])
def test_column_partition_onchip(qng, oracle, ranks, which):
    """The column partition (Sec. 3, columns independent given psi_{j-1}) emulated on one GPU: each
    rank's context computes its balanced column pairs (qng_set_column_subset, qng_metric_columns),
    the parts are merged by owner as the all-gather would, and qng_step_from_parts gives the step.
    Every column is computed by the same kernel whatever the subset, so g and dtheta equal the
    unpartitioned step bit for bit."""
    from paper_2011_02991_gb300 import dist as D
    p = W.config_rand12() if which == "rand12" else W.random_problem(6, 80, 8, 6161)
    full = qng.Context(p)
    ref = full.step(full.theta0(), p.dt, p.lam)
    full.sync()
    owner = D.column_owners(p.P, ranks)
    Ls, ss, grads = [], [], []
    for r in range(ranks):
        ctx = qng.Context(p)
        ctx.set_column_subset(qng.column_partition(p.P, ranks, r))
        with pytest.raises(qng.QngError):  # a subset context runs no whole metric
            ctx.step(ctx.theta0(), p.dt, p.lam)
        parts = ctx.metric_columns(ctx.theta0())
        ctx.sync()
        Ls.append(parts["L"])
        ss.append(parts["sigma"])
        grads.append(parts["grad"])
        ctx.close()
    L, sigma = D.merge_columns(Ls, ss, owner)
    for g in grads[1:]:
        assert torch.equal(g, grads[0])
    out = full.step_from_parts(full.theta0(), L.reshape(-1), sigma, grads[0], p.dt, p.lam)
    full.sync()
    assert torch.equal(out["g"], ref["g"])
    assert torch.equal(out["dtheta"], ref["dtheta"])
    assert rel(out["g"].cpu(), oracle.qng_step(p)["g"]) <= TOL[W.C128]


@pytest.mark.parametrize("precision", [W.C64, W.C128])
def test_graph_capture_batch256(qng, oracle, precision):
    """The 256-instance batch (6-14 qubits, 2-10 layers) captured whole in one CUDA graph: its launch
    groups run side by side on their own streams inside the capture; replays equal the direct step
    bit for bit, the side-by-side groups equal the groups run in turn, and sampled instances match
    the oracle."""
    probs = W.config_batch(precision=precision)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = qng.Context(probs, stream=stream)
        th = ctx.theta0()
        ref = ctx.step(th, 0.1, 1e-3)
        ctx.sync()
        ref = {k: v.clone() for k, v in ref.items()}
        ctx.set_pipeline(1)  # the groups in turn
        seq = ctx.step(th, 0.1, 1e-3)
        ctx.sync()
        for k in ref:
            assert torch.equal(seq[k], ref[k]), k
        ctx.set_pipeline(0)
        out = ctx.graph_capture(th, 0.1, 1e-3)
        for _ in range(2):
            for v in out.values():
                v.fill_(float("nan"))
            ctx.graph_launch()
            ctx.sync()
            for k in ref:
                assert torch.equal(out[k], ref[k]), k
    g = ref["g"].cpu().numpy()
    grad = ref["grad"].cpu().numpy()
    dth = ref["dtheta"].cpu().numpy()
    for b in (0, 101, 255):
        r = oracle.qng_step(probs[b])
        m0, m1 = ctx.metric_offsets[b], ctx.metric_offsets[b + 1]
        p0, p1 = ctx.param_offsets[b], ctx.param_offsets[b + 1]
        assert rel(g[m0:m1], r["g"]) <= TOL[precision]
        assert rel(grad[p0:p1], r["grad"]) <= TOL[precision]
        if precision == W.C128:
            assert rel(dth[p0:p1], r["dtheta"]) <= TOL[precision]
        else:  # complex64: dtheta solves its own float64 system (the tolerance reading for c64 dtheta)
            P = p1 - p0
            A = g[m0:m1].reshape(P, P) + 1e-3 * np.eye(P)
            res = A @ dth[p0:p1] + 0.1 * grad[p0:p1]
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(0.1 * grad[p0:p1])
