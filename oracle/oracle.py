"""Python side of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this module. It wraps ``qng_oracle.c`` (complex128 definitions, see that file's header) with
ctypes and adds the one step the C file leaves out: the Tikhonov-regularised solve of the
natural-gradient equation g(theta) dtheta = -dt grad<E> (Eq. 3) with g + lam*I in place of g,
done by LAPACK through numpy in float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qng_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile qng_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_apply_gate.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int]
            L.oracle_apply_pauli.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_hamiltonian_apply.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _u64p, _u64p]
            L.oracle_state.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, _dp]
            L.oracle_deriv_state.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.oracle_qgt.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, _i32p, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_energy.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp, _u64p, _u64p, _dp]
            L.oracle_gradient.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp, _u64p, _u64p,
                                          _i32p, ctypes.c_int, _dp, _dp]
            L.oracle_alg1.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _i64p, _dp]
            L.oracle_alg1_columns.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, _u8p, _dp, _dp]
            L.oracle_alg3.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, _dp, _i64p]
            L.oracle_alg6.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp, _i64p]
            L.oracle_alg8.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, _dp, _i64p]
            L.oracle_sampled.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _dp, ctypes.c_int, _dp, _u64p, _u64p, _i32p,
                                         ctypes.c_int, _dp, _dp, _dp, _dp]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


# one gate record of the C oracle: kind, q0, q1, param (int32), then the Pauli string of RP/CRP
_GATE_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("param", "<i4"),
                        ("xmask", "<u8"), ("zmask", "<u8")])


def _gates(circuit):
    g = np.ascontiguousarray(circuit.gates, dtype=np.int32).reshape(-1, 4)
    out = np.zeros(len(g), dtype=_GATE_DTYPE)
    for f, name in enumerate(("kind", "q0", "q1", "param")):
        out[name] = g[:, f]
    masks = circuit.gate_masks() if hasattr(circuit, "gate_masks") else np.zeros((len(g), 2), np.uint64)
    out["xmask"] = masks[:, 0]
    out["zmask"] = masks[:, 1]
    return out


def _check(rc):
    if rc != 0:
        raise MemoryError("oracle: allocation failed")


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(t: int) -> None:
    lib().oracle_set_num_threads(int(t))


# single operations ----------------------------------------------------------------------
def apply_gate(psi: np.ndarray, kind: int, q0: int, q1: int = -1, theta: float = 0.0, mode: int = 0,
               xmask: int = 0, zmask: int = 0) -> np.ndarray:
    """Return gate(psi); mode 0 gate, 1 adjoint, 2 derivative, 3 adjoint of the derivative.
    xmask/zmask give the Pauli string of RP/CRP gates."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    n = int(np.log2(out.size))
    lib().oracle_apply_gate(n, _p(out.view(np.float64), _dp), kind, q0, q1, int(xmask), int(zmask), float(theta), mode)
    return out


def apply_pauli(psi: np.ndarray, xmask: int, zmask: int) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    n = int(np.log2(psi.size))
    lib().oracle_apply_pauli(n, _p(psi.view(np.float64), _dp), _p(out.view(np.float64), _dp), xmask, zmask)
    return out


def hamiltonian_apply(psi: np.ndarray, ham) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    n = int(np.log2(psi.size))
    c = np.ascontiguousarray(ham.coeffs, dtype=np.float64)
    x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
    z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
    _check(lib().oracle_hamiltonian_apply(n, _p(psi.view(np.float64), _dp), _p(out.view(np.float64), _dp),
                                          len(c), _p(c, _dp), _p(x, _u64p), _p(z, _u64p)))
    return out


# circuit-level definitions ----------------------------------------------------------------
def state(circuit, theta) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    out = np.empty(1 << circuit.n, dtype=np.complex128)
    lib().oracle_state(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), _p(out.view(np.float64), _dp))
    return out


def deriv_state(circuit, theta, p: int) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    out = np.empty(1 << circuit.n, dtype=np.complex128)
    lib().oracle_deriv_state(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), int(p), _p(out.view(np.float64), _dp))
    return out


def qgt(circuit, theta, idx=None, want_state: bool = False):
    """(G, T[, psi]) over the parameter subset ``idx`` (all parameters when None). Eq. 4."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    P = circuit.num_params
    idx = np.arange(P, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    m = len(idx)
    G = np.empty((m, m), dtype=np.complex128)
    T = np.empty(m, dtype=np.complex128)
    psi = np.empty(1 << circuit.n, dtype=np.complex128) if want_state else None
    _check(lib().oracle_qgt(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), _p(idx, _i32p), m,
                            _p(G.view(np.float64), _dp), _p(T.view(np.float64), _dp),
                            _p(psi.view(np.float64), _dp) if want_state else None))
    return (G, T, psi) if want_state else (G, T)


def metric(circuit, theta, idx=None) -> np.ndarray:
    """Fubini-Study metric g = Re G (Eq. 3's g)."""
    return qgt(circuit, theta, idx)[0].real.copy()


def energy(circuit, ham, theta) -> float:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    c = np.ascontiguousarray(ham.coeffs, dtype=np.float64)
    x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
    z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
    E = np.zeros(1)
    _check(lib().oracle_energy(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), len(c), _p(c, _dp), _p(x, _u64p),
                               _p(z, _u64p), _p(E, _dp)))
    return float(E[0])


def gradient(circuit, ham, theta, idx=None):
    """(grad, E): grad[a] = d<E>/d theta_{idx[a]} = 2 Re <psi|H|d psi> (Eq. 2)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    P = circuit.num_params
    idx = np.arange(P, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    c = np.ascontiguousarray(ham.coeffs, dtype=np.float64)
    x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
    z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
    out = np.empty(len(idx))
    E = np.zeros(1)
    _check(lib().oracle_gradient(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), len(c), _p(c, _dp), _p(x, _u64p),
                                 _p(z, _u64p), _p(idx, _i32p), len(idx), _p(out, _dp), _p(E, _dp)))
    return out, float(E[0])


def sampled(problem, idx):
    """(G_sub, T_sub, grad_sub, E) over the parameter subset idx (Eq. 4 and Eq. 2), one sweep."""
    c, ham = problem.circuit, problem.hamiltonian
    theta = np.ascontiguousarray(problem.theta, dtype=np.float64)
    g = _gates(c)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    m = len(idx)
    co = np.ascontiguousarray(ham.coeffs, dtype=np.float64)
    x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
    z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
    G = np.empty((m, m), dtype=np.complex128)
    T = np.empty(m, dtype=np.complex128)
    grad = np.empty(m)
    E = np.zeros(1)
    _check(lib().oracle_sampled(c.n, _p(g, _i32p), len(g), _p(theta, _dp), len(co), _p(co, _dp), _p(x, _u64p),
                                _p(z, _u64p), _p(idx, _i32p), m, _p(G.view(np.float64), _dp),
                                _p(T.view(np.float64), _dp), _p(grad, _dp), _p(E, _dp)))
    return G, T, grad, float(E[0])


def solve_step(g: np.ndarray, grad: np.ndarray, dt: float, lam: float) -> np.ndarray:
    """dtheta solving (g + lam I) dtheta = -dt grad (Eq. 3 with Tikhonov lam), LAPACK float64."""
    A = np.asarray(g, dtype=np.float64) + lam * np.eye(g.shape[0])
    return np.linalg.solve(A, -dt * np.asarray(grad, dtype=np.float64))


def qng_step(problem):
    """Everything one QNG step produces: dict(g, grad, dtheta, E, T)."""
    G, T = qgt(problem.circuit, problem.theta)
    g = G.real.copy()
    grad, E = gradient(problem.circuit, problem.hamiltonian, problem.theta)
    dtheta = solve_step(g, grad, problem.dt, problem.lam)
    return {"g": g, "grad": grad, "dtheta": dtheta, "E": E, "T": T, "G": G}


# literal recurrences -----------------------------------------------------------------------
def alg1(circuit, theta, skip_diag: bool = True):
    """Algorithm 1 transcribed literally: (L upper triangle, T, counts=(gates, clones, IPs), psi)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    P = circuit.num_params
    L = np.zeros((P, P), dtype=np.complex128)
    T = np.zeros(P, dtype=np.complex128)
    cnt = np.zeros(3, dtype=np.int64)
    psi = np.zeros(1 << circuit.n, dtype=np.complex128)
    _check(lib().oracle_alg1(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), int(skip_diag),
                             _p(L.view(np.float64), _dp), _p(T.view(np.float64), _dp), _p(cnt, _i64p),
                             _p(psi.view(np.float64), _dp)))
    return L, T, tuple(int(v) for v in cnt), psi


def alg1_columns(circuit, theta, cols):
    """Algorithm 1 with only the inner loops of columns `cols` (0-based) run: (L, T), the other
    columns zero. psi still advances through every gate (Sec. 3's inner loop reads only psi_{j-1})."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    P = circuit.num_params
    want = np.zeros(max(P, 1), dtype=np.uint8)
    want[np.asarray(cols, dtype=np.int64)] = 1
    L = np.zeros((P, P), dtype=np.complex128)
    T = np.zeros(P, dtype=np.complex128)
    _check(lib().oracle_alg1_columns(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), _p(want, _u8p),
                                     _p(L.view(np.float64), _dp), _p(T.view(np.float64), _dp)))
    return L, T


def _alg_L(fn, circuit, theta, *extra):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = _gates(circuit)
    P = circuit.num_params
    L = np.zeros((P, P), dtype=np.complex128)
    cnt = np.zeros(3, dtype=np.int64)
    _check(fn(circuit.n, _p(g, _i32p), len(g), _p(theta, _dp), *extra, _p(L.view(np.float64), _dp), _p(cnt, _i64p)))
    return L, tuple(int(v) for v in cnt)


def alg3(circuit, theta):
    return _alg_L(lib().oracle_alg3, circuit, theta)


def alg6(circuit, theta, skip_last: bool = True):
    return _alg_L(lib().oracle_alg6, circuit, theta, int(skip_last))


def alg8(circuit, theta):
    return _alg_L(lib().oracle_alg8, circuit, theta)


def hermitian_from_upper(L: np.ndarray) -> np.ndarray:
    """Fill i > j from L_ij = L_ji^* (Sec. 2, below Eq. L_def)."""
    U = np.triu(L)
    return U + np.conj(np.triu(L, 1)).T
