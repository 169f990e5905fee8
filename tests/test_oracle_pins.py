"""Pins for the CPU oracle: it is checked against things other than itself.

* gate, Pauli-string and circuit application against dense 2^n x 2^n operators built with
  numpy kron products from scipy's matrix exponential exp(-i theta sigma / 2) (n <= 3);
* derivative states against central finite differences of the state;
* the quantum geometric tensor (Eq. 4) against a dense brute force, and against finite-difference
  derivative states;
* closed forms: L_ii = 1/4 for a single-Pauli rotation (Eq. L_diag_when_single_pauli), a single
  Ry on |0> gives g = 1/4, g_ii = (1 - <sigma_i>^2)/4, first-layer entries on different qubits
  vanish (product state);
* invariants: G Hermitian positive semi-definite; fidelity 1 - |<psi(t)|psi(t+e)>|^2 = e^T g e + O(e^3);
* the energy gradient against the parameter-shift rule and central finite differences;
* the literal recurrences (Alg. 1, 3, 6, 8) against the definition, and their operation counts
  against Table 1 and the worked totals of Appendix A;
* the rotation-sign reading (paper's exp(+i theta sigma/2) vs the textbook sign).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2011_02991_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ------------------------------------------------------------------------------------------
# dense brute force (independent of the oracle's code)
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PH = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)
SIGMA = {W.RX: PX, W.RY: PY, W.RZ: PZ}
FIXED1 = {W.X: PX, W.Y: PY, W.Z: PZ, W.H: PH}


def embed(ops: dict, n: int) -> np.ndarray:
    """Kron product with ops[q] on qubit q (qubit q = bit q, so qubit 0 is the rightmost factor)."""
    out = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        out = np.kron(out, ops.get(q, I2))
    return out


def pauli_ops(x: int, z: int, n: int) -> dict:
    ops = {}
    for q in range(n):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        if xb or zb:
            ops[q] = PY if (xb and zb) else (PX if xb else PZ)
    return ops


def generator(kind, q0, q1, x, z, n):
    """K of a parametric gate exp(-i theta K / 2): sigma on q0; P1 (control q0) x sigma on q1;
    the Pauli string S; P1 (control q0) x S."""
    if kind in SIGMA:
        return embed({q0: SIGMA[kind]}, n)
    if kind in (W.CRX, W.CRY, W.CRZ):
        return embed({q0: P1, q1: SIGMA[kind - W.CRX + W.RX]}, n)
    if kind == W.RP:
        return embed(pauli_ops(x, z, n), n)
    if kind == W.CRP:
        ops = pauli_ops(x, z, n)
        ops[q0] = P1
        return embed(ops, n)
    raise ValueError(kind)


def dense_gate(row, n, theta, sign=-1.0, deriv=False, mask=(0, 0)):
    kind, q0, q1, p = (int(v) for v in row)
    if kind in W.ROTATIONS:
        K = generator(kind, q0, q1, int(mask[0]), int(mask[1]), n)
        R = sla.expm(sign * 1j * theta[p] / 2 * K)
        if deriv:
            R = (sign * 1j / 2) * K @ R
        return R
    if kind in FIXED1:
        return embed({q0: FIXED1[kind]}, n)
    if kind == W.CZ:
        return embed({q0: P0}, n) + embed({q0: P1, q1: PZ}, n)
    if kind == W.CNOT:
        return embed({q0: P0}, n) + embed({q0: P1, q1: PX}, n)
    raise ValueError(kind)


def dense_state(circuit, theta, deriv_param=-1, sign=-1.0):
    n = circuit.n
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    for row, m in zip(circuit.gates, circuit.gate_masks()):
        psi = dense_gate(row, n, theta, sign, deriv=(row[3] == deriv_param and row[3] >= 0), mask=m) @ psi
    return psi


def dense_qgt(circuit, theta, sign=-1.0):
    P = circuit.num_params
    psi = dense_state(circuit, theta, sign=sign)
    D = np.stack([dense_state(circuit, theta, p, sign) for p in range(P)], axis=1)
    T = psi.conj() @ D
    return D.conj().T @ D - np.outer(T.conj(), T), T


def dense_hamiltonian(ham, n):
    Hm = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, x, z in zip(ham.coeffs, ham.xmask, ham.zmask):
        ops = {}
        for q in range(n):
            xb, zb = (int(x) >> q) & 1, (int(z) >> q) & 1
            if xb and zb:
                ops[q] = PY
            elif xb:
                ops[q] = PX
            elif zb:
                ops[q] = PZ
        Hm += c * embed(ops, n)
    return Hm


def rand_state(n, rng):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------------------------------
# gate level
@pytest.mark.parametrize("kind", [W.RX, W.RY, W.RZ, W.X, W.Y, W.Z, W.H])
@pytest.mark.parametrize("q", [0, 1, 2])
def test_single_qubit_gates_vs_dense(oracle, kind, q):
    rng = np.random.default_rng(100 + 10 * kind + q)
    n, theta = 3, np.array([rng.uniform(0, 2 * np.pi)])
    psi = rand_state(n, rng)
    row = (kind, q, -1, 0 if kind in SIGMA else -1)
    U = dense_gate(row, n, theta)
    np.testing.assert_allclose(oracle.apply_gate(psi, kind, q, -1, theta[0], 0), U @ psi, atol=1e-14)
    np.testing.assert_allclose(oracle.apply_gate(psi, kind, q, -1, theta[0], 1), U.conj().T @ psi, atol=1e-14)
    if kind in SIGMA:
        dU = dense_gate(row, n, theta, deriv=True)
        np.testing.assert_allclose(oracle.apply_gate(psi, kind, q, -1, theta[0], 2), dU @ psi, atol=1e-14)
        np.testing.assert_allclose(oracle.apply_gate(psi, kind, q, -1, theta[0], 3), dU.conj().T @ psi, atol=1e-14)
        # the derivative of the gate is also its finite difference in theta
        h = 1e-6
        fd = (oracle.apply_gate(psi, kind, q, -1, theta[0] + h, 0) - oracle.apply_gate(psi, kind, q, -1, theta[0] - h, 0)) / (2 * h)
        np.testing.assert_allclose(oracle.apply_gate(psi, kind, q, -1, theta[0], 2), fd, atol=1e-9)


@pytest.mark.parametrize("kind", [W.CZ, W.CNOT])
@pytest.mark.parametrize("q0,q1", [(0, 1), (1, 0), (0, 2), (2, 1)])
def test_two_qubit_gates_vs_dense(oracle, kind, q0, q1):
    rng = np.random.default_rng(7 + q0 * 3 + q1 + kind)
    n = 3
    psi = rand_state(n, rng)
    U = dense_gate((kind, q0, q1, -1), n, np.zeros(1))
    np.testing.assert_allclose(oracle.apply_gate(psi, kind, q0, q1, 0.0, 0), U @ psi, atol=1e-15)
    np.testing.assert_allclose(oracle.apply_gate(psi, kind, q0, q1, 0.0, 1), U.conj().T @ psi, atol=1e-15)


def test_pauli_strings_and_hamiltonian_vs_dense(oracle):
    rng = np.random.default_rng(3)
    n = 3
    psi = rand_state(n, rng)
    ham = W.random_pauli_hamiltonian(n, 12, rng, max_weight=3)
    for c, x, z in zip(ham.coeffs, ham.xmask, ham.zmask):
        one = W.Hamiltonian(np.array([1.0]), np.array([x], dtype=np.uint64), np.array([z], dtype=np.uint64))
        np.testing.assert_allclose(oracle.apply_pauli(psi, int(x), int(z)), dense_hamiltonian(one, n) @ psi, atol=1e-15)
    np.testing.assert_allclose(oracle.hamiltonian_apply(psi, ham), dense_hamiltonian(ham, n) @ psi, atol=1e-13)


@pytest.mark.parametrize("kind", [W.CRX, W.CRY, W.CRZ])
@pytest.mark.parametrize("c,t", [(0, 1), (2, 0), (1, 2)])
def test_controlled_rotations_vs_dense(oracle, kind, c, t):
    """|0><0|_c (x) 1 + |1><1|_c (x) R_sigma(theta) = exp(-i theta (P1 (x) sigma) / 2) (Sec. 2's
    controlled rotations); derivative (-i/2) K U, also against a finite difference in theta."""
    rng = np.random.default_rng(500 + 10 * kind + 3 * c + t)
    n, theta = 3, np.array([rng.uniform(0, 2 * np.pi)])
    psi = rand_state(n, rng)
    row = (kind, c, t, 0)
    U, dU = dense_gate(row, n, theta), dense_gate(row, n, theta, deriv=True)
    # the exponential of P1 (x) sigma is the block form, written out
    blk = embed({c: P0}, n) + embed({c: P1, t: sla.expm(-1j * theta[0] / 2 * SIGMA[kind - W.CRX + W.RX])}, n)
    np.testing.assert_allclose(U, blk, atol=1e-14)
    for mode, M in ((0, U), (1, U.conj().T), (2, dU), (3, dU.conj().T)):
        np.testing.assert_allclose(oracle.apply_gate(psi, kind, c, t, theta[0], mode), M @ psi, atol=1e-14)
    h = 1e-6
    fd = (oracle.apply_gate(psi, kind, c, t, theta[0] + h, 0) - oracle.apply_gate(psi, kind, c, t, theta[0] - h, 0)) / (2 * h)
    np.testing.assert_allclose(oracle.apply_gate(psi, kind, c, t, theta[0], 2), fd, atol=1e-9)


@pytest.mark.parametrize("labels,control", [({0: "X", 1: "X"}, -1), ({0: "Y", 2: "Z"}, -1), ({0: "X", 1: "Y", 2: "Z"}, -1),
                                            ({1: "Y"}, 0), ({0: "Z", 2: "X"}, 1), ({1: "Y", 2: "Y"}, 0)])
def test_pauli_string_rotations_vs_dense(oracle, labels, control):
    """exp(-i theta S / 2) of a Pauli string (Sec. 2's multi-qubit rotations), optionally
    controlled: against scipy's matrix exponential of the dense generator."""
    rng = np.random.default_rng(len(labels) * 7 + control + 40)
    n, theta = 3, np.array([rng.uniform(0, 2 * np.pi)])
    psi = rand_state(n, rng)
    x, z = W._pauli_masks(labels)
    kind = W.RP if control < 0 else W.CRP
    row = (kind, control, -1, 0)
    U = dense_gate(row, n, theta, mask=(x, z))
    dU = dense_gate(row, n, theta, deriv=True, mask=(x, z))
    for mode, M in ((0, U), (1, U.conj().T), (2, dU), (3, dU.conj().T)):
        got = oracle.apply_gate(psi, kind, control, -1, theta[0], mode, xmask=x, zmask=z)
        np.testing.assert_allclose(got, M @ psi, atol=1e-14)
    # S^2 = 1: the uncontrolled rotation by 2 pi is -1
    if control < 0:
        np.testing.assert_allclose(oracle.apply_gate(psi, kind, -1, -1, 2 * np.pi, 0, xmask=x, zmask=z), -psi, atol=1e-14)


# ------------------------------------------------------------------------------------------
# circuit level
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_state_and_derivatives_vs_dense(oracle, seed):
    p = W.random_problem(3, 14, 6, seed)
    np.testing.assert_allclose(oracle.state(p.circuit, p.theta), dense_state(p.circuit, p.theta), atol=1e-13)
    for k in range(p.P):
        np.testing.assert_allclose(oracle.deriv_state(p.circuit, p.theta, k),
                                   dense_state(p.circuit, p.theta, k), atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_general_circuits_vs_dense(oracle, seed):
    """States, derivative states and the whole tensor G with every generalised kind (n = 3)."""
    p = W.general_problem(3, 12, 600 + seed)
    np.testing.assert_allclose(oracle.state(p.circuit, p.theta), dense_state(p.circuit, p.theta), atol=1e-13)
    for k in range(p.P):
        np.testing.assert_allclose(oracle.deriv_state(p.circuit, p.theta, k), dense_state(p.circuit, p.theta, k),
                                   atol=1e-13)
    G, T = oracle.qgt(p.circuit, p.theta)
    Gd, Td = dense_qgt(p.circuit, p.theta)
    np.testing.assert_allclose(G, Gd, atol=1e-13)
    np.testing.assert_allclose(T, Td, atol=1e-13)


def test_general_derivative_states_vs_finite_differences(oracle):
    p = W.general_problem(4, 20, 611)
    h = 1e-5
    for k in range(p.P):
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.state(p.circuit, tp) - oracle.state(p.circuit, tm)) / (2 * h)
        np.testing.assert_allclose(oracle.deriv_state(p.circuit, p.theta, k), fd, atol=2e-10)


def test_controlled_diagonal_closed_form(oracle):
    """Sec. 2: a controlled rotation's diagonal is L_ii = (1/4) Prob(control = 1), not 1/4.
    H on the control gives Prob = 1/2: CRY on |+>|0> has <P1 (x) Y> = 0, so G = 1/8; CRZ has
    <P1 (x) Z> = 1/2, T = -i/4 and G = 1/8 - 1/16 = 1/16. A control left in |0> gives G = 0."""
    for kind, expect in ((W.CRY, 1 / 8), (W.CRZ, 1 / 16)):
        b = W._CircuitBuilder(2)
        b.fixed(W.H, 0)
        b.crot(kind, 0, 1)
        G, _ = oracle.qgt(b.build(), np.array([0.9]))
        assert abs(G[0, 0] - expect) < 1e-15
    b = W._CircuitBuilder(2)
    b.crot(W.CRX, 0, 1)
    G, _ = oracle.qgt(b.build(), np.array([0.9]))
    assert abs(G[0, 0]) < 1e-16


def test_pauli_string_rotation_closed_forms(oracle):
    """RP(ZZ) on |00> (an eigenstate): G = 0; RP(XX) on |00>: <XX> = 0 and L = 1/4, so G = 1/4;
    two RP(XX), RP(YY) on |00>: XX and YY commute, G_01 = <XX YY>/4 - <XX><YY>/4 = -1/4."""
    for labels, expect in (({0: "Z", 1: "Z"}, 0.0), ({0: "X", 1: "X"}, 0.25)):
        b = W._CircuitBuilder(2)
        b.prot(labels)
        G, _ = oracle.qgt(b.build(), np.array([0.3]))
        assert abs(G[0, 0] - expect) < 1e-15
    b = W._CircuitBuilder(2)
    b.prot({0: "X", 1: "X"})
    b.prot({0: "Y", 1: "Y"})
    G, _ = oracle.qgt(b.build(), np.array([0.0, 0.0]))
    assert abs(G[0, 1] - (-0.25)) < 1e-15


def test_derivative_states_vs_finite_differences(oracle):
    p = W.random_problem(4, 18, 6, 11)
    h = 1e-5
    for k in range(p.P):
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.state(p.circuit, tp) - oracle.state(p.circuit, tm)) / (2 * h)
        np.testing.assert_allclose(oracle.deriv_state(p.circuit, p.theta, k), fd, atol=2e-10)


@pytest.mark.parametrize("n,seed", [(2, 21), (2, 22), (3, 23), (3, 24)])
def test_qgt_vs_dense_bruteforce(oracle, n, seed):
    p = W.random_problem(n, 12, 4, seed)
    G, T = oracle.qgt(p.circuit, p.theta)
    Gd, Td = dense_qgt(p.circuit, p.theta)
    np.testing.assert_allclose(T, Td, atol=1e-13)
    np.testing.assert_allclose(G, Gd, atol=1e-13)


def test_qgt_vs_finite_difference_states(oracle):
    """Eq. 4 evaluated with derivative states from finite differences (no derivative formula)."""
    p = W.config_tfim4()
    h = 1e-5
    psi = oracle.state(p.circuit, p.theta)
    D = []
    for k in range(p.P):
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[k] += h
        tm[k] -= h
        D.append((oracle.state(p.circuit, tp) - oracle.state(p.circuit, tm)) / (2 * h))
    D = np.stack(D, axis=1)
    T = psi.conj() @ D
    G_fd = D.conj().T @ D - np.outer(T.conj(), T)
    G, _ = oracle.qgt(p.circuit, p.theta)
    np.testing.assert_allclose(G, G_fd, atol=1e-9)


def test_qgt_subset_matches_full(oracle):
    p = W.config_tfim4()
    G, T = oracle.qgt(p.circuit, p.theta)
    idx = np.array([0, 5, 7, 15], dtype=np.int32)
    Gs, Ts = oracle.qgt(p.circuit, p.theta, idx)
    np.testing.assert_array_equal(Gs, G[np.ix_(idx, idx)])
    np.testing.assert_array_equal(Ts, T[idx])


# ------------------------------------------------------------------------------------------
# closed forms
@pytest.mark.parametrize("kind,expected", [(W.RY, 0.25), (W.RX, 0.25), (W.RZ, 0.0)])
def test_single_rotation_on_zero(oracle, kind, expected):
    """One rotation on |0>: g = (1 - <sigma>^2)/4, so 1/4 for Rx, Ry and 0 for Rz."""
    c = W.Circuit(1, np.array([[kind, 0, -1, 0]], dtype=np.int32))
    for th in (0.0, 0.3, 1.7, 4.0):
        g = oracle.metric(c, np.array([th]))
        assert abs(g[0, 0] - expected) < 1e-15


def test_diagonal_is_one_quarter(oracle):
    """L_ii = <d_i psi|d_i psi> = 1/4 for single-Pauli rotations (Eq. L_diag_when_single_pauli)."""
    for p in (W.config_tfim4(), W.random_problem(5, 30, 5, 9)):
        G, T = oracle.qgt(p.circuit, p.theta)
        L_diag = np.diag(G).real + np.abs(T) ** 2
        np.testing.assert_allclose(L_diag, 0.25, atol=1e-14)


def test_diagonal_closed_form(oracle):
    """g_ii = (1 - <psi_i|sigma_i|psi_i>^2)/4, the expectation taken on the state right after gate i."""
    p = W.random_problem(4, 24, 5, 31)
    g = oracle.metric(p.circuit, p.theta)
    n = p.n
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    k = 0
    for row in p.circuit.gates:
        psi = dense_gate(row, n, p.theta) @ psi
        if row[0] in SIGMA:
            s = embed({int(row[1]): SIGMA[int(row[0])]}, n)
            e = (psi.conj() @ s @ psi).real
            assert abs(g[k, k] - (1 - e * e) / 4) < 1e-14
            k += 1


def test_first_layer_product_state_entries_vanish(oracle):
    p = W.config_rand12()
    first = np.arange(2 * p.n)  # Ry on every qubit, then Rz on every qubit, before the first CZ
    g = oracle.metric(p.circuit, p.theta, first)
    q = np.concatenate([np.arange(p.n), np.arange(p.n)])
    off = q[:, None] != q[None, :]
    assert np.abs(g[off]).max() < 1e-14  # rounding of 4096-term sums; a dropped T term gives O(0.1)


def test_hermitian_psd(oracle):
    p = W.random_problem(4, 40, 5, 5)
    G, _ = oracle.qgt(p.circuit, p.theta)
    np.testing.assert_allclose(G, G.conj().T, atol=1e-15)
    assert np.linalg.eigvalsh(G).min() > -1e-13


@pytest.mark.parametrize("a,b", [(0.7, -1.3), (2.9, 0.4), (-2.2, 3.0)])
def test_imaginary_part_closed_form(oracle, a, b):
    """RY(a) then RZ(b) on |0>: with phi = RY(a)|0> real, <d_0 psi|d_1 psi> = (1/4)<phi|Y Z|phi> =
    (i/4)<phi|X|phi> = (i/4) sin a, and <psi|d_0 psi> = 0, so G_01 = i sin(a)/4 (Re 0); a conjugated
    or reversed inner product gives the opposite sign."""
    bld = W._CircuitBuilder(1)
    bld.rot(W.RY, 0)
    bld.rot(W.RZ, 0)
    G, _ = oracle.qgt(bld.build(), np.array([a, b]))
    assert abs(G[0, 1] - 0.25j * np.sin(a)) < 1e-15
    assert abs(G[1, 0] + 0.25j * np.sin(a)) < 1e-15


def test_imaginary_part_present(oracle):
    """On a generic circuit Im G is antisymmetric and far from zero (the Hermitian pin is not vacuous)."""
    p = W.random_problem(5, 60, 6, 31)
    G, _ = oracle.qgt(p.circuit, p.theta)
    assert np.abs(G.imag).max() > 0.05
    np.testing.assert_allclose(G.imag, -G.imag.T, atol=1e-15)


def test_fidelity_expansion(oracle):
    """1 - |<psi(theta)|psi(theta + eps)>|^2 = eps^T g eps + O(eps^3)."""
    p = W.config_tfim4()
    g = oracle.metric(p.circuit, p.theta)
    psi = oracle.state(p.circuit, p.theta)
    rng = np.random.default_rng(0)
    d = rng.standard_normal(p.P)
    d /= np.linalg.norm(d)
    res = []
    for scale in (2e-3, 1e-3, 5e-4):
        eps = scale * d
        lhs = 1 - abs(psi.conj() @ oracle.state(p.circuit, p.theta + eps)) ** 2
        rhs = eps @ g @ eps
        assert abs(lhs - rhs) < 1e-2 * abs(rhs)
        res.append(abs(lhs - rhs))
    assert res[1] < res[0] / 5 and res[2] < res[1] / 5  # residual falls at least like eps^3 (ratio 8)


def test_trailing_fixed_gates_cancel_in_G_not_in_E(oracle):
    p = W.config_tfim4()
    extra = np.array([[W.H, 0, -1, -1], [W.CNOT, 0, 3, -1], [W.X, 2, -1, -1]], dtype=np.int32)
    c2 = W.Circuit(p.n, np.concatenate([p.circuit.gates, extra]))
    G1, _ = oracle.qgt(p.circuit, p.theta)
    G2, _ = oracle.qgt(c2, p.theta)
    np.testing.assert_allclose(G1, G2, atol=1e-14)
    assert abs(oracle.energy(p.circuit, p.hamiltonian, p.theta) - oracle.energy(c2, p.hamiltonian, p.theta)) > 1e-3


# ------------------------------------------------------------------------------------------
# energy, gradient, step
def test_energy_vs_dense(oracle):
    p = W.random_problem(3, 16, 10, 41)
    psi = dense_state(p.circuit, p.theta)
    E = (psi.conj() @ dense_hamiltonian(p.hamiltonian, p.n) @ psi).real
    assert abs(oracle.energy(p.circuit, p.hamiltonian, p.theta) - E) < 1e-13


@pytest.mark.parametrize("maker", [W.config_tfim4, lambda: W.random_problem(4, 30, 8, 51)])
def test_gradient_parameter_shift_and_fd(oracle, maker):
    p = maker()
    grad, E = oracle.gradient(p.circuit, p.hamiltonian, p.theta)
    assert abs(E - oracle.energy(p.circuit, p.hamiltonian, p.theta)) < 1e-14
    for k in range(p.P):
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[k] += np.pi / 2
        tm[k] -= np.pi / 2
        shift = 0.5 * (oracle.energy(p.circuit, p.hamiltonian, tp) - oracle.energy(p.circuit, p.hamiltonian, tm))
        assert abs(grad[k] - shift) < 1e-13
        h = 1e-5
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.energy(p.circuit, p.hamiltonian, tp) - oracle.energy(p.circuit, p.hamiltonian, tm)) / (2 * h)
        assert abs(grad[k] - fd) < 1e-8


def test_step_residual_and_scalar_case(oracle):
    p = W.config_tfim4()
    r = oracle.qng_step(p)
    A = r["g"] + p.lam * np.eye(p.P)
    b = -p.dt * r["grad"]
    assert np.linalg.norm(A @ r["dtheta"] - b) <= 1e-12 * np.linalg.norm(b)
    # one parameter: dtheta = -dt * dE / (g + lam)
    c = W.Circuit(1, np.array([[W.RY, 0, -1, 0]], dtype=np.int32))
    ham = W.hamiltonian_from_terms([(0.7, {0: "Z"}), (0.3, {0: "X"})])
    th = np.array([0.9])
    g = oracle.metric(c, th)
    grad, _ = oracle.gradient(c, ham, th)
    # <Z> = cos t, <X> = sin t for Ry(t)|0>, so dE = -0.7 sin t + 0.3 cos t
    assert abs(grad[0] - (-0.7 * np.sin(0.9) + 0.3 * np.cos(0.9))) < 1e-15
    dth = oracle.solve_step(g, grad, 0.1, 1e-3)
    assert abs(dth[0] - (-0.1 * grad[0] / (0.25 + 1e-3))) < 1e-15


# ------------------------------------------------------------------------------------------
# the paper's recurrences and their operation counts
def _poly(coeffs, P):
    return sum(Fraction(c) * P ** (3 - k) for k, c in enumerate(coeffs))


@pytest.mark.parametrize("maker", [W.config_tfim4, lambda: W.random_problem(4, 26, 4, 61)])
def test_recurrences_agree_with_definition(oracle, maker):
    p = maker()
    G, T = oracle.qgt(p.circuit, p.theta)
    L_def = G + np.outer(T.conj(), T)
    L1, T1, _, psi1 = oracle.alg1(p.circuit, p.theta, skip_diag=False)
    np.testing.assert_allclose(T1, T, atol=1e-14)
    np.testing.assert_allclose(oracle.hermitian_from_upper(L1), L_def, atol=1e-14)
    L1s, _, _, _ = oracle.alg1(p.circuit, p.theta, skip_diag=True)
    np.testing.assert_allclose(oracle.hermitian_from_upper(L1s), L_def, atol=1e-14)
    for fn in (oracle.alg3, oracle.alg6, oracle.alg8):
        L, _ = fn(p.circuit, p.theta)
        np.testing.assert_allclose(oracle.hermitian_from_upper(L), L_def, atol=1e-14)


def test_recurrences_with_generalised_rotations(oracle):
    """Alg. 1 (diagonal by simulation), 3, 6 and 8 with controlled and Pauli-string rotations agree
    with the definition; with a control the a-priori diagonal 1/4 is wrong where Prob(control=1)
    differs from 1 (Sec. 2), and equals (1/4) Prob(control = 1) there."""
    p = W.general_problem(4, 24, 71)
    G, T = oracle.qgt(p.circuit, p.theta)
    L_def = G + np.outer(T.conj(), T)
    L1, T1, _, _ = oracle.alg1(p.circuit, p.theta, skip_diag=False)
    np.testing.assert_allclose(T1, T, atol=1e-14)
    np.testing.assert_allclose(oracle.hermitian_from_upper(L1), L_def, atol=1e-14)
    for fn in (oracle.alg3, oracle.alg6, oracle.alg8):
        L, _ = fn(p.circuit, p.theta)
        np.testing.assert_allclose(oracle.hermitian_from_upper(L), L_def, atol=1e-14)
    kinds = p.circuit.param_gates()[:, 0]
    ctl = np.isin(kinds, [W.CRX, W.CRY, W.CRZ, W.CRP])
    assert ctl.any() and np.abs(np.diag(L_def).real[ctl] - 0.25).max() > 1e-3
    np.testing.assert_allclose(np.diag(L_def).real[~ctl], 0.25, atol=1e-14)


def test_operation_counts_table1(oracle):
    gold = json.load(open(os.path.join(GOLDEN, "table1_op_counts.json")))
    poly = gold["polynomials"]
    for P in (1, 2, 5, 16, 100):
        c = W.Circuit(1, np.array([[W.RY, 0, -1, k] for k in range(P)], dtype=np.int32))
        th = np.linspace(0.1, 2.0, P)
        ip = _poly(gold["inner_products"]["coeffs"], P)
        if P <= 16:
            _, cnt = oracle.alg3(c, th)
            assert cnt[0] == _poly(poly["alg3"]["gates"], P) and cnt[1] == _poly(poly["alg3"]["clones"], P)
            assert cnt[2] == ip
        _, cnt = oracle.alg6(c, th, skip_last=True)
        assert cnt[0] == _poly(poly["alg6"]["gates"], P) and cnt[1] == _poly(poly["alg6"]["clones"], P)
        assert cnt[2] == ip
        _, cnt_lit = oracle.alg6(c, th, skip_last=False)
        assert cnt_lit[0] == cnt[0] + P  # the literal loop applies phi <- U_1^dag once more per column
        _, cnt = oracle.alg8(c, th)
        assert cnt[0] == _poly(poly["alg8"]["gates"], P) and cnt[1] == _poly(poly["alg8"]["clones"], P)
        assert cnt[2] == ip
        # Algorithm 1 itself (no Table 1 row): gates 3/2 P^2 + 1/2 P, clones 1/2 P^2 + 3/2 P + 1,
        # inner products (P^2 + P)/2 with the a-priori diagonal
        _, _, cnt, _ = oracle.alg1(c, th, skip_diag=True)
        assert cnt == (Fraction(3, 2) * P * P + Fraction(1, 2) * P, Fraction(1, 2) * P * P + Fraction(3, 2) * P + 1, ip)
    for name, total in gold["worked_totals_P100"].items():
        if name.startswith("_"):
            continue
        assert _poly(poly[name]["total"], 100) == total


def test_operation_count_alg3_at_100(oracle):
    """Alg. 3 run literally at P = 100 reproduces the worked total 681750."""
    gold = json.load(open(os.path.join(GOLDEN, "table1_op_counts.json")))
    P = 100
    c = W.Circuit(1, np.array([[W.RY, 0, -1, k] for k in range(P)], dtype=np.int32))
    _, cnt = oracle.alg3(c, np.linspace(0.1, 2.0, P))
    assert cnt[0] + cnt[1] == gold["worked_totals_P100"]["alg3"]
    _, cnt = oracle.alg6(c, np.linspace(0.1, 2.0, P))
    assert cnt[0] + cnt[1] == gold["worked_totals_P100"]["alg6"]
    _, cnt = oracle.alg8(c, np.linspace(0.1, 2.0, P))
    assert cnt[0] + cnt[1] == gold["worked_totals_P100"]["alg8"]


# ------------------------------------------------------------------------------------------
# readings
def test_rotation_sign_reading(oracle):
    """The paper writes R(theta) = exp(+i theta sigma/2); flipping the sign maps theta -> -theta:
    G_paper(theta) = G(-theta) and grad_paper(theta) = -grad(-theta)."""
    p = W.random_problem(3, 12, 5, 71)
    Gp, _ = dense_qgt(p.circuit, p.theta, sign=+1.0)
    G, _ = oracle.qgt(p.circuit, -p.theta)
    np.testing.assert_allclose(Gp, G, atol=1e-13)
    Hd = dense_hamiltonian(p.hamiltonian, p.n)
    psi = dense_state(p.circuit, p.theta, sign=+1.0)
    grad_p = np.array([2 * (psi.conj() @ Hd @ dense_state(p.circuit, p.theta, k, +1.0)).real for k in range(p.P)])
    grad, _ = oracle.gradient(p.circuit, p.hamiltonian, -p.theta)
    np.testing.assert_allclose(grad_p, -grad, atol=1e-13)


def test_workload_shapes():
    assert W.config_tfim4().P == 16
    assert W.config_rand12().P == 192 and W.config_rand12().hamiltonian.num_terms == 40
    assert W.config_tfim26().P == 208
    assert W.config_rand28().P == 252 and W.config_rand28().hamiltonian.num_terms == 64
    batch = W.config_batch()
    assert len(batch) == 256
    Ps = [b.P for b in batch]
    assert min(Ps) >= 24 and max(Ps) <= 280
    for b in batch:
        assert 6 <= b.n <= 14 and 16 <= b.hamiltonian.num_terms <= 48
        w = np.array([bin(int(x) | int(z)).count("1") for x, z in zip(b.hamiltonian.xmask, b.hamiltonian.zmask)])
        assert w.min() >= 1 and w.max() <= 4


def test_sampled_matches_full(oracle):
    p = W.random_problem(5, 40, 8, 91)
    idx = np.array([0, 3, p.P - 1], dtype=np.int32)
    Gs, Ts, gs, E = oracle.sampled(p, idx)
    G, T = oracle.qgt(p.circuit, p.theta)
    grad, E2 = oracle.gradient(p.circuit, p.hamiltonian, p.theta)
    np.testing.assert_allclose(Gs, G[np.ix_(idx, idx)], atol=1e-15)
    np.testing.assert_allclose(Ts, T[idx], atol=1e-15)
    np.testing.assert_allclose(gs, grad[idx], atol=1e-14)
    assert abs(E - E2) < 1e-14
