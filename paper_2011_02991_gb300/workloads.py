"""Seeded synthetic inputs: ansatz circuits, Pauli-string Hamiltonians and parameters.

This module only *describes* problems. It holds none of the method's arithmetic (no gate
matrices, no state vectors, no inner products), so both the CPU oracle and the CUDA path
can read the same inputs without sharing any code that computes a result.

Encoding (the C-ABI in ``include/qng.h`` declares the same numbers):

* A gate is four int32 values ``(kind, q0, q1, param)``. Parametric gates are the Pauli
  rotations R_sigma(theta) = exp(-i theta sigma / 2), sigma in {X, Y, Z}; ``param`` is the
  index of their angle in theta. The paper assumes one unique parameter per gate, applied in
  circuit order (Sec. 2, the definition of U(theta) as U_P ... U_1), so the k-th parametric
  gate of a circuit carries ``param == k``. Fixed gates carry ``param == -1``.
* Generalised rotations (Sec. 2's remark on multi-qubit and controlled Pauli-string rotations):
  CRX/CRY/CRZ are |0><0|_c (x) 1 + |1><1|_c (x) R_sigma(theta) with control q0 and target q1;
  RP is exp(-i theta S / 2) for a Pauli string S; CRP is RP controlled by q0. The string of an
  RP/CRP gate is the gate's row of ``Circuit.masks`` (xmask, zmask), as for Hamiltonian terms.
* Qubit q is bit q of a basis-state index (q0 is the least significant bit).
* A Pauli string is ``(coeff, xmask, zmask)``: bit q of ``xmask``/``zmask`` set means the
  factor on qubit q has an X/Z part; both set means Y; neither means identity.

The five named workloads follow the benchmark descriptions: hardware-efficient layers of
per-qubit rotations followed by an entangling ladder, a transverse-field Ising chain or random
Pauli strings of weight 1..4 with N(0, 1) coefficients, and theta uniform in [0, 2 pi). All
draws use numpy's PCG64 generator from a stated seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# gate kinds ----------------------------------------------------------------------------
RX, RY, RZ = 0, 1, 2
CZ, CNOT = 3, 4
X, Y, Z, H = 5, 6, 7, 8
CRX, CRY, CRZ, RP, CRP = 9, 10, 11, 12, 13
ROTATIONS = (RX, RY, RZ, CRX, CRY, CRZ, RP, CRP)
SIMPLE_ROTATIONS = (RX, RY, RZ)
GENERAL_ROTATIONS = (CRX, CRY, CRZ, RP, CRP)
FIXED_ONE_QUBIT = (X, Y, Z, H)
FIXED_TWO_QUBIT = (CZ, CNOT)
KIND_NAMES = {RX: "RX", RY: "RY", RZ: "RZ", CZ: "CZ", CNOT: "CNOT", X: "X", Y: "Y", Z: "Z", H: "H",
              CRX: "CRX", CRY: "CRY", CRZ: "CRZ", RP: "RP", CRP: "CRP"}

# precisions ----------------------------------------------------------------------------
C64, C128 = 0, 1

BASE_SEED = 20110299


@dataclass
class Circuit:
    """A gate list on ``n`` qubits; ``gates`` is an (G, 4) int32 array of (kind, q0, q1, param);
    ``masks`` (G, 2) uint64 holds the (xmask, zmask) Pauli string of RP/CRP gates (zeros
    elsewhere; None when the circuit has none)."""

    n: int
    gates: np.ndarray
    masks: np.ndarray | None = None

    def gate_masks(self) -> np.ndarray:
        if self.masks is None:
            return np.zeros((len(self.gates), 2), dtype=np.uint64)
        return np.ascontiguousarray(self.masks, dtype=np.uint64).reshape(-1, 2)

    @property
    def has_general(self) -> bool:
        return bool(np.isin(self.gates[:, 0], GENERAL_ROTATIONS).any())

    @property
    def num_params(self) -> int:
        return int(np.count_nonzero(np.isin(self.gates[:, 0], ROTATIONS)))

    def param_gates(self) -> np.ndarray:
        return self.gates[np.isin(self.gates[:, 0], ROTATIONS)]


@dataclass
class Hamiltonian:
    """H = sum_k coeffs[k] * sigma_k with sigma_k given by its X and Z bit masks."""

    coeffs: np.ndarray  # float64 (T,)
    xmask: np.ndarray  # uint64 (T,)
    zmask: np.ndarray  # uint64 (T,)

    @property
    def num_terms(self) -> int:
        return int(self.coeffs.shape[0])


@dataclass
class Problem:
    """One QNG instance: circuit, Hamiltonian and parameters, plus the step settings."""

    name: str
    circuit: Circuit
    hamiltonian: Hamiltonian
    theta: np.ndarray  # float64 (P,)
    dt: float = 0.1
    lam: float = 1e-3
    precision: int = C128
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.circuit.n

    @property
    def P(self) -> int:
        return self.circuit.num_params


# circuit builders ------------------------------------------------------------------------
class _CircuitBuilder:
    def __init__(self, n: int):
        self.n = n
        self.rows: list[tuple[int, int, int, int]] = []
        self.mrows: list[tuple[int, int]] = []
        self.P = 0

    def rot(self, kind: int, q: int) -> None:
        self.rows.append((kind, q, -1, self.P))
        self.mrows.append((0, 0))
        self.P += 1

    def crot(self, kind: int, control: int, target: int) -> None:
        """CRX/CRY/CRZ: rotation of target, controlled by control."""
        self.rows.append((kind, control, target, self.P))
        self.mrows.append((0, 0))
        self.P += 1

    def prot(self, labels: dict[int, str], control: int = -1) -> None:
        """RP (or CRP with a control) of the Pauli string {qubit: 'X'|'Y'|'Z'}."""
        x, z = _pauli_masks(labels)
        self.rows.append((RP if control < 0 else CRP, control, -1, self.P))
        self.mrows.append((x, z))
        self.P += 1

    def fixed(self, kind: int, q0: int, q1: int = -1) -> None:
        self.rows.append((kind, q0, q1, -1))
        self.mrows.append((0, 0))

    def build(self) -> Circuit:
        g = np.array(self.rows, dtype=np.int32).reshape(-1, 4)
        m = np.array(self.mrows, dtype=np.uint64).reshape(-1, 2)
        return Circuit(self.n, g, m if m.any() else None)


def layered_ansatz(n: int, layers: int, rotation_kinds=(RY, RZ), entangler: int = CZ) -> Circuit:
    """``layers`` repetitions of [each kind in ``rotation_kinds`` on q0..q_{n-1}] + a ladder.

    The ladder is CZ(q_k, q_{k+1}) or CNOT(control q_k, target q_{k+1}) for k = 0..n-2 in
    increasing k. Parameters are numbered layer-major, then by rotation kind, then by qubit.
    """
    b = _CircuitBuilder(n)
    for _ in range(layers):
        for kind in rotation_kinds:
            for q in range(n):
                b.rot(kind, q)
        for q in range(n - 1):
            b.fixed(entangler, q, q + 1)
    return b.build()


def random_circuit(n: int, num_gates: int, rng: np.random.Generator, p_fixed: float = 0.35) -> Circuit:
    """A random mix of every supported gate kind; used by tests to cover all gate code paths."""
    b = _CircuitBuilder(n)
    for _ in range(num_gates):
        if rng.random() < p_fixed:
            choices = list(FIXED_ONE_QUBIT) + (list(FIXED_TWO_QUBIT) if n >= 2 else [])
            kind = int(rng.choice(choices))
            if kind in FIXED_TWO_QUBIT:
                q0, q1 = rng.choice(n, size=2, replace=False)
                b.fixed(kind, int(q0), int(q1))
            else:
                b.fixed(kind, int(rng.integers(n)))
        else:
            b.rot(int(rng.choice(SIMPLE_ROTATIONS)), int(rng.integers(n)))
    return b.build()


# Hamiltonian builders --------------------------------------------------------------------
def _pauli_masks(labels: dict[int, str]) -> tuple[int, int]:
    x = z = 0
    for q, p in labels.items():
        if p in ("X", "Y"):
            x |= 1 << q
        if p in ("Z", "Y"):
            z |= 1 << q
    return x, z


def hamiltonian_from_terms(terms: list[tuple[float, dict[int, str]]]) -> Hamiltonian:
    c = np.array([t[0] for t in terms], dtype=np.float64)
    masks = [_pauli_masks(t[1]) for t in terms]
    x = np.array([m[0] for m in masks], dtype=np.uint64)
    z = np.array([m[1] for m in masks], dtype=np.uint64)
    return Hamiltonian(c, x, z)


def tfim_chain(n: int, J: float = 1.0, h=0.5) -> Hamiltonian:
    """Open chain sum_i J Z_i Z_{i+1} + sum_i h_i X_i (h scalar or per-site array)."""
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    terms = [(J, {i: "Z", i + 1: "Z"}) for i in range(n - 1)]
    terms += [(float(hs[i]), {i: "X"}) for i in range(n)]
    return hamiltonian_from_terms(terms)


def random_pauli_hamiltonian(n: int, num_terms: int, rng: np.random.Generator, max_weight: int = 4) -> Hamiltonian:
    """Random strings: weight w ~ U{1..min(max_weight, n)}, w distinct qubits, X/Y/Z uniform, c ~ N(0,1)."""
    terms = []
    for _ in range(num_terms):
        w = int(rng.integers(1, min(max_weight, n) + 1))
        qs = rng.choice(n, size=w, replace=False)
        ps = rng.choice(np.array(["X", "Y", "Z"]), size=w)
        c = float(rng.standard_normal())
        terms.append((c, {int(q): str(p) for q, p in zip(qs, ps)}))
    return hamiltonian_from_terms(terms)


def uniform_theta(P: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(0.0, 2.0 * np.pi, size=P)


# the named workloads ---------------------------------------------------------------------
def config_tfim4(seed: int = BASE_SEED + 1) -> Problem:
    """4 qubits, 2 x [Ry all, Rz all, CZ ladder] (P=16), H = sum Z_i Z_{i+1} + 0.5 sum X_i, c128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = layered_ansatz(4, 2)
    return Problem("tfim4_p16_c128", c, tfim_chain(4, 1.0, 0.5), uniform_theta(c.num_params, rng),
                   precision=C128, meta={"seed": seed})


def config_rand12(seed: int = BASE_SEED + 2, precision: int = C128) -> Problem:
    """12 qubits, 8 x [Ry all, Rz all, CZ ladder] (P=192), 40 random Pauli strings, c128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = layered_ansatz(12, 8)
    theta = uniform_theta(c.num_params, rng)
    h = random_pauli_hamiltonian(12, 40, rng)
    return Problem("rand12_p192_c128" if precision == C128 else "rand12_p192_c64", c, h, theta,
                   precision=precision, meta={"seed": seed})


def config_batch(count: int = 256, seed: int = BASE_SEED + 3, precision: int = C64,
                 n_range=(6, 14), layer_range=(2, 10), term_range=(16, 48)) -> list[Problem]:
    """Independent instances of uneven size: n ~ U{6..14}, layers ~ U{2..10}, 16..48 terms each.

    Instance b draws from its own generator seeded ``seed * 1000 + b``.
    """
    out = []
    for b in range(count):
        rng = np.random.Generator(np.random.PCG64(seed * 1000 + b))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        layers = int(rng.integers(layer_range[0], layer_range[1] + 1))
        terms = int(rng.integers(term_range[0], term_range[1] + 1))
        c = layered_ansatz(n, layers)
        theta = uniform_theta(c.num_params, rng)
        h = random_pauli_hamiltonian(n, terms, rng)
        out.append(Problem(f"batch{b}_n{n}_l{layers}", c, h, theta, precision=precision,
                           meta={"seed": seed * 1000 + b, "layers": layers}))
    return out


def config_tfim26(seed: int = BASE_SEED + 4, n: int = 26, layers: int = 4) -> Problem:
    """26 qubits, 4 x [Ry all, Rz all, CZ ladder] (P=208), TFIM J=1, h_i ~ U[0.2, 1.0], c128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = layered_ansatz(n, layers)
    theta = uniform_theta(c.num_params, rng)
    h = rng.uniform(0.2, 1.0, size=n)
    return Problem(f"tfim{n}_p{c.num_params}_c128", c, tfim_chain(n, 1.0, h), theta,
                   precision=C128, meta={"seed": seed})


def config_rand28(seed: int = BASE_SEED + 5, precision: int = C64, n: int = 28, layers: int = 3) -> Problem:
    """28 qubits, 3 x [Ry all, Rx all, Rz all, CNOT ladder] (P=252), 64 random strings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = layered_ansatz(n, layers, rotation_kinds=(RY, RX, RZ), entangler=CNOT)
    theta = uniform_theta(c.num_params, rng)
    h = random_pauli_hamiltonian(n, 64, rng)
    tag = "c64" if precision == C64 else "c128"
    return Problem(f"rand{n}_p{c.num_params}_{tag}", c, h, theta, precision=precision, meta={"seed": seed})


def vqe_tfim(n: int = 12, layers: int = 6, seed: int = 5, precision: int = C128) -> Problem:
    """Natural-gradient VQE on the open TFIM chain (J = 1, h = 0.7): layered Ry/Rz/CZ ansatz from
    small angles, theta ~ U[-0.2, 0.2] (the descent tests and the loop benchmark)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = layered_ansatz(n, layers)
    return Problem(f"vqe_tfim{n}_l{layers}", c, tfim_chain(n, 1.0, 0.7), rng.uniform(-0.2, 0.2, c.num_params),
                   precision=precision, meta={"seed": seed})


def z_run_problem(n: int, num_params: int, seed: int, precision: int = C128, max_run: int = 24,
                  near_half_pi: bool = False) -> Problem:
    """Runs of RZ rotations (1..max_run long) separated by RX/RY rotations (test workload).

    Inside a run the fixed gates before each RZ are none, CZ, Z or CZ + Z (all diagonal); with
    probability 1/8 a CNOT or H is placed instead, which breaks the run. near_half_pi draws the
    angles from pi/2 +- 0.3 instead of [-pi, pi): each half-angle factor max(|cos|, |sin|) is then
    close to 2^-1/2, so long circuits drive a running product of them through many binades.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _CircuitBuilder(n)
    while b.P < num_params:
        b.rot(int(rng.choice([RX, RY])), int(rng.integers(n)))
        for _ in range(int(rng.integers(1, max_run + 1))):
            if b.P >= num_params:
                break
            r = rng.random()
            if r < 0.125:
                if n >= 2 and rng.random() < 0.5:
                    q0, q1 = rng.choice(n, size=2, replace=False)
                    b.fixed(CNOT, int(q0), int(q1))
                else:
                    b.fixed(H, int(rng.integers(n)))
            elif r < 0.4 and n >= 2:
                q0, q1 = rng.choice(n, size=2, replace=False)
                b.fixed(CZ, int(q0), int(q1))
                if rng.random() < 0.5:
                    b.fixed(Z, int(rng.integers(n)))
            elif r < 0.55:
                b.fixed(Z, int(rng.integers(n)))
            b.rot(RZ, int(rng.integers(n)))
    c = b.build()
    theta = uniform_theta(c.num_params, rng)
    if near_half_pi:
        theta = np.pi / 2 + rng.uniform(-0.3, 0.3, c.num_params)
    h = random_pauli_hamiltonian(n, 2 * n, rng)
    return Problem(f"zrun_n{n}_p{num_params}", c, h, theta, precision=precision, meta={"seed": seed})


def general_problem(n: int, num_params: int, seed: int, precision: int = C128, max_weight: int = 3) -> Problem:
    """Every parametric kind, generalised ones included (test and benchmark workload): RX/RY/RZ,
    CRX/CRY/CRZ with random control and target, RP and CRP of random Pauli strings of weight
    1..max_weight (the control outside the string), and CZ/CNOT/H fixed gates in between."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _CircuitBuilder(n)
    while b.P < num_params:
        r = rng.random()
        if r < 0.15 and n >= 2:
            q0, q1 = rng.choice(n, size=2, replace=False)
            b.fixed(int(rng.choice([CZ, CNOT])), int(q0), int(q1))
        elif r < 0.2:
            b.fixed(H, int(rng.integers(n)))
        elif r < 0.4:
            b.rot(int(rng.choice([RX, RY, RZ])), int(rng.integers(n)))
        elif r < 0.6 and n >= 2:
            c, t = rng.choice(n, size=2, replace=False)
            b.crot(int(rng.choice([CRX, CRY, CRZ])), int(c), int(t))
        else:
            ctrl = -1
            pool = list(range(n))
            if rng.random() < 0.4 and n >= 2:
                ctrl = int(rng.integers(n))
                pool.remove(ctrl)
            w = int(rng.integers(1, min(max_weight, len(pool)) + 1))
            qs = rng.choice(pool, size=w, replace=False)
            b.prot({int(q): "XYZ"[int(rng.integers(3))] for q in qs}, ctrl)
    c = b.build()
    theta = uniform_theta(c.num_params, rng)
    h = random_pauli_hamiltonian(n, 2 * n, rng)
    return Problem(f"general_n{n}_p{num_params}", c, h, theta, precision=precision, meta={"seed": seed})


def random_problem(n: int, num_gates: int, num_terms: int, seed: int, precision: int = C128) -> Problem:
    """A small random problem with every gate kind (test workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = random_circuit(n, num_gates, rng)
    theta = uniform_theta(c.num_params, rng)
    h = random_pauli_hamiltonian(n, num_terms, rng)
    return Problem(f"random_n{n}_g{num_gates}", c, h, theta, precision=precision, meta={"seed": seed})
