"""CPU-only checks of the C ABI: the library loads, exports every declared symbol, and its host
logic (validation, sizes, offsets, workspace layout) behaves. No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2011_02991_gb300 import build as B
from paper_2011_02991_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2011_02991_gb300 import qng
    return qng.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(qng_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "qng_create" in names and "qng_step" in names
    for name in names:
        assert hasattr(lib, name), name


def _create(lib, n, gates, terms=(), precision=W.C128):
    from paper_2011_02991_gb300 import qng
    ga = (qng.qng_gate * max(len(gates), 1))(*[qng.qng_gate(*g) for g in gates])
    ta = (qng.qng_pauli * max(len(terms), 1))(*[qng.qng_pauli(*t) for t in terms])
    h = ctypes.c_void_p()
    st = lib.qng_create(n, ga, len(gates), ta, len(terms), precision, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("gates,n,expect", [
    ([(W.RY, 0, -1, 0)], 1, 0),
    ([(W.RY, 1, -1, 0)], 1, 1),            # qubit out of range
    ([(W.RY, 0, -1, 1)], 1, 1),            # parameters must be numbered in circuit order
    ([(W.CZ, 0, 0, -1)], 2, 1),            # two-qubit gate on one qubit
    ([(W.CZ, 0, 1, 0)], 2, 1),             # fixed gate with a parameter
    ([(42, 0, -1, -1)], 2, 1),             # unknown kind
    ([(W.RX, 0, -1, 0), (W.H, 1, -1, -1), (W.RZ, 1, -1, 1)], 2, 0),
    ([], 3, 0),                            # no gates at all
    ([(W.RY, 0, -1, 0)], 17, 0),           # streaming path (state vectors in HBM)
    ([(W.RY, 0, -1, 0)], 31, 1),           # more qubits than any path takes
])
def test_validation(lib, gates, n, expect):
    st, h = _create(lib, n, gates)
    assert st == expect
    if st == 0:
        lib.qng_destroy(h)


def _create_ex(lib, n, gates, masks, terms=(), precision=W.C128):
    from paper_2011_02991_gb300 import qng
    ga = (qng.qng_gate * max(len(gates), 1))(*[qng.qng_gate(*g) for g in gates])
    ta = (qng.qng_pauli * max(len(terms), 1))(*[qng.qng_pauli(*t) for t in terms])
    m = None if masks is None else (ctypes.c_uint64 * (2 * len(gates)))(*[v for pair in masks for v in pair])
    h = ctypes.c_void_p()
    st = lib.qng_create_ex(n, ga, len(gates), m, ta, len(terms), precision, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("gates,masks,n,expect", [
    ([(W.CRX, 0, 1, 0)], None, 2, 0),                      # controlled rotation: no string needed
    ([(W.CRY, 1, 1, 0)], None, 2, 1),                      # control = target
    ([(W.CRZ, 0, 2, 0)], None, 2, 1),                      # target out of range
    ([(W.RP, -1, -1, 0)], [(0b11, 0b01)], 2, 0),           # exp(-i theta Y0 X1 / 2)
    ([(W.RP, -1, -1, 0)], None, 2, 1),                     # a string gate needs the masks
    ([(W.RP, 0, -1, 0)], [(0b11, 0)], 2, 1),               # RP takes no qubit
    ([(W.RP, -1, -1, 0)], [(0b100, 0)], 2, 1),             # string outside the qubits
    ([(W.CRP, 0, -1, 0)], [(0b10, 0b10)], 2, 0),           # Y1 controlled by q0
    ([(W.CRP, 0, -1, 0)], [(0b11, 0)], 2, 1),              # the string acts on the control
    ([(W.CRX, 0, 1, 0)], None, 17, 7),                     # generalised rotations: on-chip path only
])
def test_generalised_validation(lib, gates, masks, n, expect):
    st, h = _create_ex(lib, n, gates, masks)
    assert st == expect
    if st == 0:
        lib.qng_destroy(h)


def test_pauli_validation(lib):
    st, h = _create(lib, 2, [(W.RY, 0, -1, 0)], [(1.0, 0b100, 0)])
    assert st == 1
    st, h = _create(lib, 2, [(W.RY, 0, -1, 0)], [(float("nan"), 1, 0)])
    assert st == 1


def test_sizes_offsets_workspace(lib):
    from paper_2011_02991_gb300 import qng
    probs = W.config_batch(count=5)
    rows = [np.ascontiguousarray(p.circuit.gates, dtype=np.int32) for p in probs]
    allg = np.concatenate(rows)
    ga = (qng.qng_gate * len(allg))()
    ctypes.memmove(ga, allg.ctypes.data, allg.nbytes)
    terms = [(float(c), int(x), int(z)) for p in probs for c, x, z in
             zip(p.hamiltonian.coeffs, p.hamiltonian.xmask, p.hamiltonian.zmask)]
    ta = (qng.qng_pauli * len(terms))(*[qng.qng_pauli(*t) for t in terms])
    nq = np.array([p.n for p in probs], dtype=np.int32)
    ng = np.array([len(r) for r in rows], dtype=np.int32)
    nt = np.array([p.hamiltonian.num_terms for p in probs], dtype=np.int32)
    h = ctypes.c_void_p()
    i32 = ctypes.POINTER(ctypes.c_int32)
    assert lib.qng_create_batch(5, nq.ctypes.data_as(i32), ga, ng.ctypes.data_as(i32), ta, nt.ctypes.data_as(i32),
                                W.C64, ctypes.byref(h)) == 0
    cnt, tp, tm = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    assert lib.qng_get_sizes(h, ctypes.byref(cnt), ctypes.byref(tp), ctypes.byref(tm)) == 0
    Ps = [p.P for p in probs]
    assert cnt.value == 5 and tp.value == sum(Ps) and tm.value == sum(P * P for P in Ps)
    po = np.zeros(6, dtype=np.int64)
    mo = np.zeros(6, dtype=np.int64)
    i64 = ctypes.POINTER(ctypes.c_int64)
    assert lib.qng_get_offsets(h, po.ctypes.data_as(i64), mo.ctypes.data_as(i64)) == 0
    assert list(po) == list(np.concatenate([[0], np.cumsum(Ps)]))
    assert list(mo) == list(np.concatenate([[0], np.cumsum([P * P for P in Ps])]))
    nb = ctypes.c_size_t()
    assert lib.qng_workspace_size(h, ctypes.byref(nb)) == 0
    # checkpoints dominate: (P+1) 2^n complex64 amplitudes per instance
    assert nb.value >= sum((p.P + 1) * (1 << p.n) * 8 for p in probs)
    assert nb.value % 256 == 0
    # compute calls without a workspace are refused on the host
    theta = ctypes.c_void_p(0)
    assert lib.qng_metric(h, theta, ctypes.c_void_p(8), None) == 6
    assert lib.qng_set_workspace(h, ctypes.c_void_p(0x1000 + 8), nb.value, None) == 6  # misaligned
    assert lib.qng_set_workspace(h, ctypes.c_void_p(0x1000), nb.value - 256, None) == 6  # too small
    lib.qng_destroy(h)


def test_streaming_workspace(lib):
    """A 20-qubit instance runs on the streaming path: three registers of 2^20 amplitudes, no checkpoints."""
    c = W.layered_ansatz(20, 2)
    st, h = _create(lib, 20, [tuple(int(v) for v in r) for r in c.gates], [(1.0, 1, 0)], W.C128)
    assert st == 0
    nb = ctypes.c_size_t()
    assert lib.qng_workspace_size(h, ctypes.byref(nb)) == 0
    regs = 3 * (1 << 20) * 16
    assert regs <= nb.value < regs + 64 * 1024 * 1024
    assert lib.qng_set_path(h, 1) == 7  # on-chip path cannot hold 20 qubits
    lib.qng_destroy(h)
    # a batch cannot hold a streaming instance
    from paper_2011_02991_gb300 import qng
    ga = (qng.qng_gate * 1)(qng.qng_gate(W.RY, 0, -1, 0))
    ta = (qng.qng_pauli * 1)(qng.qng_pauli(1.0, 1, 0))
    i32 = ctypes.POINTER(ctypes.c_int32)
    nq = np.array([20, 20], dtype=np.int32)
    ng = np.array([1, 0], dtype=np.int32)
    nt = np.array([1, 0], dtype=np.int32)
    h = ctypes.c_void_p()
    assert lib.qng_create_batch(2, nq.ctypes.data_as(i32), ga, ng.ctypes.data_as(i32), ta, nt.ctypes.data_as(i32),
                                W.C128, ctypes.byref(h)) == 7


def test_status_strings(lib):
    for s in range(8):
        assert lib.qng_status_string(s)


def test_pipeline_forward_cluster_and_solve_report_on_the_host(lib):
    """Host-side settings: the chunk count of the pipelined sweep and the sweep's cluster size are
    validated and planned without a device; the solve report is empty before any step."""
    c = W.layered_ansatz(12, 8)
    st, h = _create(lib, 12, [tuple(int(v) for v in r) for r in c.gates], [(1.0, 1, 0)], W.C128)
    assert st == 0
    chunks = ctypes.c_int32()
    for bad in (-1, 9):
        assert lib.qng_set_pipeline(h, bad) == 1
    for ok in (0, 1, 2, 8):
        assert lib.qng_set_pipeline(h, ok) == 0
    assert lib.qng_get_pipeline(h, ctypes.byref(chunks)) == 0
    assert chunks.value == 0  # no workspace yet: nothing pipelines
    fcl = ctypes.c_int32()
    assert lib.qng_get_forward_cluster(h, 12, ctypes.byref(fcl)) == 0
    assert fcl.value == 4  # one instance: twice the column kernel's 8 CTAs
    for bad in (-2, 5):
        assert lib.qng_set_forward_cluster(h, 12, bad) == 1
    assert lib.qng_set_forward_cluster(h, 0, 2) == 1  # qubit count out of range
    assert lib.qng_set_forward_cluster(h, 12, 2) == 0
    assert lib.qng_get_forward_cluster(h, 12, ctypes.byref(fcl)) == 0 and fcl.value == 2
    assert lib.qng_set_forward_cluster(h, 12, -1) == 0
    assert lib.qng_get_forward_cluster(h, 12, ctypes.byref(fcl)) == 0 and fcl.value == 4
    path, handed = ctypes.c_int32(), ctypes.c_int32()
    assert lib.qng_solve_report(h, ctypes.byref(path), ctypes.byref(handed)) == 0
    assert path.value == 0 and handed.value == 0
    lib.qng_destroy(h)
    # a batch keeps one cluster size for both kernels
    from paper_2011_02991_gb300 import qng
    probs = W.config_batch(count=3)
    rows = [np.ascontiguousarray(p.circuit.gates, dtype=np.int32) for p in probs]
    allg = np.concatenate(rows)
    ga = (qng.qng_gate * len(allg))()
    ctypes.memmove(ga, allg.ctypes.data, allg.nbytes)
    ta = (qng.qng_pauli * 3)(*[qng.qng_pauli(1.0, 1, 0)] * 3)
    i32 = ctypes.POINTER(ctypes.c_int32)
    nq = np.array([p.n for p in probs], dtype=np.int32)
    ng = np.array([len(r) for r in rows], dtype=np.int32)
    nt = np.ones(3, dtype=np.int32)
    hb = ctypes.c_void_p()
    assert lib.qng_create_batch(3, nq.ctypes.data_as(i32), ga, ng.ctypes.data_as(i32), ta, nt.ctypes.data_as(i32),
                                W.C64, ctypes.byref(hb)) == 0
    cl, th, fth = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    for n in {p.n for p in probs}:
        assert lib.qng_get_tuning(hb, n, ctypes.byref(cl), ctypes.byref(th), ctypes.byref(fth)) == 0
        assert lib.qng_get_forward_cluster(hb, n, ctypes.byref(fcl)) == 0
        assert fcl.value == cl.value
    lib.qng_destroy(hb)


def _noalloc_status(lib, n, circuit, precision):
    """Call qng_metric_noalloc with placeholder device pointers on inputs it must reject on the
    host, before it touches the device (the pointers are never dereferenced)."""
    from paper_2011_02991_gb300 import qng
    f = lib.qng_metric_noalloc
    f.argtypes = [ctypes.c_int, ctypes.POINTER(qng.qng_gate), ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    ga, ng = qng._gates_array(circuit)
    fake = ctypes.c_void_p(1 << 40)
    return f(n, ga, ng, precision, fake, fake, None)


@pytest.mark.parametrize("n,layers,precision,expect", [
    (16, 1, W.C128, 7),   # 16 qubits at complex128: the cluster's state buffers exceed shared memory
    (16, 1, W.C64, 6),    # 16 qubits complex64, P = 32: the checkpoints exceed the 16 MiB array
    (15, 1, W.C128, 6),   # 15 qubits complex128, P = 30
    (12, 16, W.C128, 6),  # 12 qubits complex128, P = 384 > 320 parameters
    (17, 1, W.C64, 1),    # beyond the on-chip path
])
def test_noalloc_limits_rejected_on_host(lib, n, layers, precision, expect):
    c = W.layered_ansatz(n, layers)
    assert _noalloc_status(lib, n, c, precision) == expect
