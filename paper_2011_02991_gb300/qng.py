"""Python binding of libqng (argument marshalling only; every step runs in the CUDA kernels).

The ``qng_*`` functions mirror the C ABI of ``include/qng.h`` one to one. ``Context`` wraps them
for PyTorch users: PyTorch provides the device workspace and the stream, the library does the
work. There is no CPU fallback: without a built ``libqng.so`` or without a CUDA device every
call raises.
"""
from __future__ import annotations

import atexit
import ctypes
import weakref
import os
from typing import Sequence

import numpy as np
import torch

from . import workloads as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libqng.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "host allocation failed", 3: "CUDA error", 4: "device wait timed out",
          5: "g + lambda I is not positive definite", 6: "workspace missing, too small or misaligned",
          7: "unsupported request"}
QNG_OK, QNG_ERR_ARG, QNG_ERR_OOM, QNG_ERR_CUDA, QNG_ERR_TIMEOUT, QNG_ERR_NOT_SPD, QNG_ERR_WORKSPACE, QNG_ERR_UNSUPPORTED = range(8)


class QngError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, 'unknown status')} ({status})")
        self.status = status


class qng_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32), ("param", ctypes.c_int32)]


class qng_pauli(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64)]


_lib = None
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
SYMBOLS = {
    "qng_create": [ctypes.c_int, ctypes.POINTER(qng_gate), ctypes.c_int, ctypes.POINTER(qng_pauli), ctypes.c_int,
                   ctypes.c_int, ctypes.POINTER(_vp)],
    "qng_create_batch": [ctypes.c_int, _i32p, ctypes.POINTER(qng_gate), _i32p, ctypes.POINTER(qng_pauli), _i32p,
                         ctypes.c_int, ctypes.POINTER(_vp)],
    "qng_create_ex": [ctypes.c_int, ctypes.POINTER(qng_gate), ctypes.c_int, _vp, ctypes.POINTER(qng_pauli),
                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "qng_create_batch_ex": [ctypes.c_int, _i32p, ctypes.POINTER(qng_gate), _i32p, _vp, ctypes.POINTER(qng_pauli), _i32p,
                            ctypes.c_int, ctypes.POINTER(_vp)],
    "qng_get_sizes": [_vp, _i32p, _i64p, _i64p],
    "qng_get_offsets": [_vp, _i64p, _i64p],
    "qng_workspace_size": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "qng_set_workspace": [_vp, _vp, ctypes.c_size_t, _vp],
    "qng_set_stream": [_vp, _vp],
    "qng_metric": [_vp, _vp, _vp, _vp],
    "qng_metric_complex": [_vp, _vp, _vp, _vp, _vp],
    "qng_optimize": [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp],
    "qng_gradient": [_vp, _vp, _vp, _vp],
    "qng_energy": [_vp, _vp, _vp],
    "qng_energy_backward": [_vp, _vp, _vp, _vp],
    "qng_step": [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp],
    "qng_step_host": [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp],
    "qng_sync": [_vp],
    "qng_set_tuning": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "qng_last_launch_count": [_vp, _i64p],
    "qng_solve_report": [_vp, _i32p, _i32p],
    "qng_set_pipeline": [_vp, ctypes.c_int],
    "qng_set_forward_cluster": [_vp, ctypes.c_int, ctypes.c_int],
    "qng_get_forward_cluster": [_vp, ctypes.c_int, _i32p],
    "qng_get_pipeline": [_vp, _i32p],
    "qng_profile": [_vp, ctypes.c_int],
    "qng_set_path": [_vp, ctypes.c_int],
    "qng_stream_traffic": [_vp, _i64p, _i64p, _i64p],
    "qng_stream_segments": [_vp, _i64p, _i64p],
    "qng_column_partition": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, ctypes.POINTER(ctypes.c_int)],
    "qng_set_column_subset": [_vp, _i32p, ctypes.c_int],
    "qng_metric_columns": [_vp, _vp, _vp, _vp, _vp, _vp],
    "qng_step_from_parts": [_vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp],
    "qng_graph_capture": [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp],
    "qng_graph_launch": [_vp],
    "qng_autotune": [_vp, _vp, ctypes.c_int, _i64p],
    "qng_get_tuning": [_vp, ctypes.c_int, _i32p, _i32p, _i32p],
    "qng_set_shape": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "qng_profile_read": [_vp, ctypes.POINTER(ctypes.c_double), _i64p],
    "qng_destroy": [_vp],
    "qng_status_string": [ctypes.c_int],
}


# Contexts still open at interpreter exit are closed by an atexit hook: the library releases its
# CUDA streams and events then, before the CUDA runtime itself shuts down.
_live: "weakref.WeakSet" = weakref.WeakSet()


@atexit.register
def _close_live_contexts():
    for ctx in list(_live):
        try:
            ctx.close()
        except Exception:
            pass


def column_partition(P: int, ranks: int, rank: int) -> list[int]:
    """The metric columns rank `rank` of `ranks` computes (qng_column_partition: balanced pairs)."""
    cols = (ctypes.c_int32 * max(P, 1))()
    n = ctypes.c_int()
    _chk(load().qng_column_partition(int(P), int(ranks), int(rank), cols, ctypes.byref(n)), "qng_column_partition")
    return [int(cols[k]) for k in range(n.value)]


def load(path: str = LIB_PATH):
    """Load libqng.so (built by ``paper_2011_02991_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libqng.so not built ({path}); run paper_2011_02991_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, args in SYMBOLS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "qng_status_string" else (None if name == "qng_destroy" else ctypes.c_int)
        _lib = L
    return _lib


def _chk(status: int, where: str):
    if status != QNG_OK:
        raise QngError(status, where)


def _gates_array(circuit: W.Circuit):
    g = np.ascontiguousarray(circuit.gates, dtype=np.int32)
    arr = (qng_gate * max(len(g), 1))()
    ctypes.memmove(arr, g.ctypes.data, g.nbytes)
    return arr, len(g)


def _terms_array(ham: W.Hamiltonian):
    T = ham.num_terms
    arr = (qng_pauli * max(T, 1))()
    for t in range(T):
        arr[t].coeff = float(ham.coeffs[t])
        arr[t].xmask = int(ham.xmask[t])
        arr[t].zmask = int(ham.zmask[t])
    return arr, T


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Context:
    """A libqng context over one or more instances, with a torch-allocated workspace.

    ``problems`` is a Problem or a list of Problems (a batch). theta and the per-parameter outputs
    are concatenated over instances; metrics are concatenated P_b x P_b blocks.
    """

    def __init__(self, problems, precision: int | None = None, device=None, stream: torch.cuda.Stream | None = None,
                 path: int = 0):
        L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libqng needs a CUDA device")
        self.problems = [problems] if isinstance(problems, W.Problem) else list(problems)
        self.precision = self.problems[0].precision if precision is None else precision
        self.device = torch.device(device if device is not None else "cuda")
        self._h = _vp()
        if len(self.problems) == 1:
            p = self.problems[0]
            ga, ng = _gates_array(p.circuit)
            ta, nt = _terms_array(p.hamiltonian)
            masks = np.ascontiguousarray(p.circuit.gate_masks(), dtype=np.uint64)
            self._masks = masks  # kept alive for the call
            _chk(L.qng_create_ex(p.n, ga, ng, ctypes.c_void_p(masks.ctypes.data), ta, nt, self.precision,
                                 ctypes.byref(self._h)), "qng_create_ex")
        else:
            rows = [np.ascontiguousarray(p.circuit.gates, dtype=np.int32) for p in self.problems]
            allg = np.concatenate(rows) if rows else np.zeros((0, 4), np.int32)
            ga = (qng_gate * max(len(allg), 1))()
            ctypes.memmove(ga, allg.ctypes.data, allg.nbytes)
            nq = np.array([p.n for p in self.problems], dtype=np.int32)
            ngs = np.array([len(r) for r in rows], dtype=np.int32)
            nts = np.array([p.hamiltonian.num_terms for p in self.problems], dtype=np.int32)
            ta = (qng_pauli * max(int(nts.sum()), 1))()
            k = 0
            for p in self.problems:
                h = p.hamiltonian
                for t in range(h.num_terms):
                    ta[k].coeff = float(h.coeffs[t]); ta[k].xmask = int(h.xmask[t]); ta[k].zmask = int(h.zmask[t])
                    k += 1
            masks = np.ascontiguousarray(np.concatenate([p.circuit.gate_masks() for p in self.problems])
                                         if self.problems else np.zeros((0, 2)), dtype=np.uint64)
            self._masks = masks
            _chk(L.qng_create_batch_ex(len(self.problems), nq.ctypes.data_as(_i32p), ga, ngs.ctypes.data_as(_i32p),
                                       ctypes.c_void_p(masks.ctypes.data), ta, nts.ctypes.data_as(_i32p), self.precision,
                                       ctypes.byref(self._h)), "qng_create_batch_ex")
        _live.add(self)
        cnt = ctypes.c_int32()
        tp, tm = ctypes.c_int64(), ctypes.c_int64()
        _chk(L.qng_get_sizes(self._h, ctypes.byref(cnt), ctypes.byref(tp), ctypes.byref(tm)), "qng_get_sizes")
        self.count, self.total_params, self.total_metric = cnt.value, tp.value, tm.value
        po = np.zeros(self.count + 1, dtype=np.int64)
        mo = np.zeros(self.count + 1, dtype=np.int64)
        _chk(L.qng_get_offsets(self._h, po.ctypes.data_as(_i64p), mo.ctypes.data_as(_i64p)), "qng_get_offsets")
        self.param_offsets, self.metric_offsets = po, mo
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if path:
            _chk(L.qng_set_path(self._h, int(path)), "qng_set_path")
        self._alloc_workspace()

    def _alloc_workspace(self):
        L = load()
        nb = ctypes.c_size_t()
        _chk(L.qng_workspace_size(self._h, ctypes.byref(nb)), "qng_workspace_size")
        self.workspace = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        _chk(L.qng_set_workspace(self._h, _ptr(self.workspace), self.workspace.numel(),
                                 ctypes.c_void_p(self.stream.cuda_stream)), "qng_set_workspace")

    # -- helpers -----------------------------------------------------------------------------
    def _f64(self, n):
        return torch.empty(int(n), dtype=torch.float64, device=self.device)

    def _theta(self, theta):
        if not isinstance(theta, torch.Tensor):
            theta = torch.as_tensor(np.asarray(theta, dtype=np.float64))
        theta = theta.to(device=self.device, dtype=torch.float64).contiguous()
        if theta.numel() != self.total_params:
            raise ValueError(f"theta has {theta.numel()} entries, expected {self.total_params}")
        return theta

    def split_params(self, v: torch.Tensor):
        return [v[self.param_offsets[b]:self.param_offsets[b + 1]] for b in range(self.count)]

    def split_metric(self, g: torch.Tensor):
        out = []
        for b in range(self.count):
            P = int(self.param_offsets[b + 1] - self.param_offsets[b])
            out.append(g[self.metric_offsets[b]:self.metric_offsets[b + 1]].view(P, P))
        return out

    def theta0(self):
        return torch.as_tensor(np.concatenate([p.theta for p in self.problems]), dtype=torch.float64, device=self.device)

    # -- entry points --------------------------------------------------------------------------
    def metric(self, theta, want_sigma: bool = False):
        theta = self._theta(theta)
        g = self._f64(self.total_metric)
        sg = self._f64(self.total_params) if want_sigma else None
        _chk(load().qng_metric(self._h, _ptr(theta), _ptr(g), _ptr(sg)), "qng_metric")
        return (g, sg) if want_sigma else g

    def metric_complex(self, theta, want_sigma: bool = False):
        """The quantum geometric tensor G = g + i Im G as a complex128 tensor (flat, like metric)."""
        theta = self._theta(theta)
        g, gi = self._f64(self.total_metric), self._f64(self.total_metric)
        sg = self._f64(self.total_params) if want_sigma else None
        _chk(load().qng_metric_complex(self._h, _ptr(theta), _ptr(g), _ptr(gi), _ptr(sg)), "qng_metric_complex")
        G = torch.complex(g, gi)
        return (G, sg) if want_sigma else G

    def gradient(self, theta):
        theta = self._theta(theta)
        gr, en = self._f64(self.total_params), self._f64(self.count)
        _chk(load().qng_gradient(self._h, _ptr(theta), _ptr(gr), _ptr(en)), "qng_gradient")
        return gr, en

    def energy(self, theta):
        theta = self._theta(theta)
        en = self._f64(self.count)
        _chk(load().qng_energy(self._h, _ptr(theta), _ptr(en)), "qng_energy")
        return en

    def energy_backward(self, theta, grad_out):
        theta = self._theta(theta)
        go = grad_out.to(device=self.device, dtype=torch.float64).contiguous()
        gt = self._f64(self.total_params)
        _chk(load().qng_energy_backward(self._h, _ptr(theta), _ptr(go), _ptr(gt)), "qng_energy_backward")
        return gt

    def step(self, theta, dt: float = 0.1, lam: float = 1e-3, outputs: dict | None = None):
        """One QNG step; returns dict(dtheta, g, grad, energy) of device tensors."""
        theta = self._theta(theta)
        o = outputs if outputs is not None else {
            "dtheta": self._f64(self.total_params), "g": self._f64(self.total_metric),
            "grad": self._f64(self.total_params), "energy": self._f64(self.count)}
        _chk(load().qng_step(self._h, _ptr(theta), float(dt), float(lam), _ptr(o["dtheta"]), _ptr(o.get("g")),
                             _ptr(o.get("grad")), _ptr(o.get("energy"))), "qng_step")
        return o

    def optimize(self, theta: torch.Tensor, dt: float = 0.1, lam: float = 1e-3, iters: int = 100):
        """QNG descent on the device: theta (a float64 tensor on this context's device, contiguous)
        is updated in place iters times; returns <E> per iteration, shape (iters, count)."""
        if not (isinstance(theta, torch.Tensor) and theta.dtype == torch.float64 and theta.is_contiguous()
                and theta.device == self.workspace.device and theta.numel() == self.total_params):
            raise ValueError("theta must be a contiguous float64 tensor on the context's device with total_params entries")
        en = torch.empty((int(iters), self.count), dtype=torch.float64, device=self.device)
        _chk(load().qng_optimize(self._h, _ptr(theta), float(dt), float(lam), int(iters), _ptr(en)), "qng_optimize")
        return en

    def step_host(self, theta_host: np.ndarray, dt: float = 0.1, lam: float = 1e-3, out: dict | None = None,
                  want_all: bool = True):
        """qng_step_host: host (numpy, ideally pinned) buffers in and out; waits for completion."""
        th = np.ascontiguousarray(theta_host, dtype=np.float64)
        o = out if out is not None else {"dtheta": np.empty(self.total_params), "g": np.empty(self.total_metric),
                                         "grad": np.empty(self.total_params), "energy": np.empty(self.count)}
        p = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
        _chk(load().qng_step_host(self._h, p(th), float(dt), float(lam), p(o["dtheta"]),
                                  p(o.get("g")) if want_all else None, p(o.get("grad")) if want_all else None,
                                  p(o.get("energy")) if want_all else None), "qng_step_host")
        return o

    def graph_capture(self, theta, dt: float = 0.1, lam: float = 1e-3, outputs: dict | None = None) -> dict:
        """Capture one step into a CUDA graph; the returned output tensors are refreshed by graph_launch."""
        theta = self._theta(theta)
        self._graph_theta = theta
        o = outputs if outputs is not None else {
            "dtheta": self._f64(self.total_params), "g": self._f64(self.total_metric),
            "grad": self._f64(self.total_params), "energy": self._f64(self.count)}
        self._graph_out = o
        _chk(load().qng_graph_capture(self._h, _ptr(theta), float(dt), float(lam), _ptr(o["dtheta"]), _ptr(o.get("g")),
                                      _ptr(o.get("grad")), _ptr(o.get("energy"))), "qng_graph_capture")
        return o

    def graph_launch(self):
        _chk(load().qng_graph_launch(self._h), "qng_graph_launch")

    def autotune(self, theta, reps: int = 3) -> int:
        theta = self._theta(theta)
        n = ctypes.c_int64()
        _chk(load().qng_autotune(self._h, _ptr(theta), int(reps), ctypes.byref(n)), "qng_autotune")
        return int(n.value)

    def get_tuning(self, n_qubits: int):
        """(cluster_log2, column CTA size, checkpoint-sweep CTA size) for n_qubits."""
        cl, th, fth = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _chk(load().qng_get_tuning(self._h, int(n_qubits), ctypes.byref(cl), ctypes.byref(th), ctypes.byref(fth)),
             "qng_get_tuning")
        return cl.value, th.value, fth.value

    def set_shape(self, n_qubits: int, cluster_log2: int, threads: int, forward_threads: int = 0):
        _chk(load().qng_set_shape(self._h, int(n_qubits), int(cluster_log2), int(threads), int(forward_threads)),
             "qng_set_shape")

    def stream_traffic(self):
        """(metric_bytes, other_bytes, metric_passes) of one step on the streaming path."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _chk(load().qng_stream_traffic(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "qng_stream_traffic")
        return a.value, b.value, c.value

    def sync(self):
        _chk(load().qng_sync(self._h), "qng_sync")

    PATH_AUTO, PATH_ONCHIP, PATH_STREAMING = 0, 1, 2

    def set_path(self, path: int):
        """Choose the execution path (re-plans; the workspace is re-allocated when it grows)."""
        L = load()
        st = L.qng_set_path(self._h, int(path))
        if st == QNG_ERR_WORKSPACE:
            self._alloc_workspace_for_new_plan(path)
            return
        _chk(st, "qng_set_path")

    def _alloc_workspace_for_new_plan(self, path: int):
        # release the workspace binding, re-plan without one, then allocate the new size
        L = load()
        self.close()
        self.__init__(self.problems, self.precision, self.device, self.stream, path=path)

    def set_tuning(self, min_qubits: int, cluster_log2: int, threads: int):
        _chk(load().qng_set_tuning(self._h, min_qubits, cluster_log2, threads), "qng_set_tuning")

    # -- column partition (one instance over several ranks) -----------------------------------
    def set_column_subset(self, cols=None):
        """Restrict the metric recurrence to columns `cols` (0-based); None restores every column."""
        L = load()
        if cols is None:
            _chk(L.qng_set_column_subset(self._h, None, -1), "qng_set_column_subset")
            return
        c = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
        self._subset = c
        _chk(L.qng_set_column_subset(self._h, c.ctypes.data_as(_i32p), int(c.size)), "qng_set_column_subset")

    def metric_columns(self, theta):
        """The subset's columns: dict(L (P x P, (1/4) Re L_ij for i < j of the subset's columns),
        sigma (P), grad (P), energy (1)) as device tensors."""
        theta = self._theta(theta)
        P = self.total_params
        out = {"L": self._f64(P * P), "sigma": self._f64(P), "grad": self._f64(P), "energy": self._f64(1)}
        _chk(load().qng_metric_columns(self._h, _ptr(theta), _ptr(out["L"]), _ptr(out["sigma"]), _ptr(out["grad"]),
                                       _ptr(out["energy"])), "qng_metric_columns")
        return out

    def step_from_parts(self, theta, L, sigma, grad, dt: float = 0.1, lam: float = 1e-3):
        """Assembly and solve from gathered parts (device tensors): dict(dtheta, g)."""
        theta = self._theta(theta)
        P = self.total_params
        out = {"dtheta": self._f64(P), "g": self._f64(P * P)}
        L, sigma, grad = (t.to(self.device, torch.float64).contiguous() for t in (L, sigma, grad))
        _chk(load().qng_step_from_parts(self._h, _ptr(theta), _ptr(L), _ptr(sigma), _ptr(grad), float(dt), float(lam),
                                        _ptr(out["dtheta"]), _ptr(out["g"])), "qng_step_from_parts")
        return out

    # kernel classes of qng_profile_read (include/qng.h); 4-7 are streaming-path segments
    KERNEL_CLASSES = ("coef", "forward", "columns", "finish", "energy", "hpsi", "adjoint", "reduce")

    def profile(self, enable: bool):
        _chk(load().qng_profile(self._h, int(bool(enable))), "qng_profile")

    def profile_read(self) -> dict:
        """Per kernel class: (milliseconds, launches) since the last read; waits for the stream."""
        k = len(self.KERNEL_CLASSES)
        ms = (ctypes.c_double * k)()
        n = (ctypes.c_int64 * k)()
        _chk(load().qng_profile_read(self._h, ms, n), "qng_profile_read")
        return {name: (ms[i], n[i]) for i, name in enumerate(self.KERNEL_CLASSES)}

    def stream_segments(self) -> dict:
        """Per kernel class: (HBM bytes the schedule moves in one step, launches); streaming path."""
        k = len(self.KERNEL_CLASSES)
        b = (ctypes.c_int64 * k)()
        n = (ctypes.c_int64 * k)()
        _chk(load().qng_stream_segments(self._h, b, n), "qng_stream_segments")
        return {name: (b[i], n[i]) for i, name in enumerate(self.KERNEL_CLASSES)}

    def last_launch_count(self) -> int:
        v = ctypes.c_int64()
        _chk(load().qng_last_launch_count(self._h, ctypes.byref(v)), "qng_last_launch_count")
        return int(v.value)

    def set_forward_cluster(self, n_qubits: int, cluster_log2: int):
        """Cluster size (log2, up to 4) of the checkpoint sweep for n_qubits; -1 = the column kernel's."""
        _chk(load().qng_set_forward_cluster(self._h, int(n_qubits), int(cluster_log2)), "qng_set_forward_cluster")

    def forward_cluster(self, n_qubits: int) -> int:
        v = ctypes.c_int32()
        _chk(load().qng_get_forward_cluster(self._h, int(n_qubits), ctypes.byref(v)), "qng_get_forward_cluster")
        return int(v.value)

    def set_pipeline(self, chunks: int):
        """Chunks of the pipelined checkpoint sweep: 0 automatic, 1 off, 2..8 that many."""
        _chk(load().qng_set_pipeline(self._h, int(chunks)), "qng_set_pipeline")

    def pipeline(self) -> int:
        """Chunk count the next call uses (0: no pipelining)."""
        v = ctypes.c_int32()
        _chk(load().qng_get_pipeline(self._h, ctypes.byref(v)), "qng_get_pipeline")
        return int(v.value)

    SOLVE_PATHS = {0: "none", 1: "single", 2: "cluster", 3: "mixed", 4: "block"}

    def solve_report(self) -> tuple[str, int]:
        """(solve the last step ran, instances the mixed-precision solve handed to float64)."""
        path, handed = ctypes.c_int32(), ctypes.c_int32()
        _chk(load().qng_solve_report(self._h, ctypes.byref(path), ctypes.byref(handed)), "qng_solve_report")
        return self.SOLVE_PATHS[int(path.value)], int(handed.value)

    def close(self):
        if self._h:
            load().qng_destroy(self._h)
            self._h = _vp()
            _live.discard(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Energy(torch.autograd.Function):
    """<E>(theta) with the reverse-sweep (adjoint) backward of libqng."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, qctx: Context):
        ctx.qctx = qctx
        ctx.save_for_backward(theta)
        return qctx.energy(theta)

    @staticmethod
    def backward(ctx, grad_out):
        (theta,) = ctx.saved_tensors
        return ctx.qctx.energy_backward(theta, grad_out), None


def energy(theta: torch.Tensor, qctx: Context) -> torch.Tensor:
    return Energy.apply(theta, qctx)
