"""Host checks of the streaming planner (no GPU): schedules of layered, random and Z-run circuits,
whole or restricted to a rank's columns, built by a host-only probe (tests/planner_probe.cu) that
links the library's planner source.

What is checked, for complex64 (register-phase passes from 12 qubits) and complex128 (tile-program
passes):
- every entry of Algorithm 1's output is reduced exactly once: (1/4) Re L_ij for i < j and
  <sigma_j> for every computed column j, Im L_ij as well in the complex-metric segment, every
  gradient entry (Eq. 2) and the energy;
- a column subset computes exactly its own columns;
- the bench's float64 flop count of the streaming metric segment equals the schedule's steps;
- the probe's structural invariants: two columns walk together only as (l, l + 1) with l odd, a pass
  holds at most three registers and never psi with b2, every non-diagonal target of a register
  phase is a register bit, a composed run holds only diagonal operations, and a straight-line block
  is the phase's last operations in register-bit order.
"""
import shutil
import subprocess

import numpy as np
import pytest

from paper_2011_02991_gb300 import workloads as W

ROOT = __import__("pathlib").Path(__file__).resolve().parents[1]
SEG_FORWARD, SEG_ENERGY, SEG_ADJOINT, SEG_METRIC, SEG_METRIC_IM = range(5)
REG_SIGMA, REG_L, REG_GRAD, REG_ENERGY, REG_LIM = range(5)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not shutil.which(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path_factory.mktemp("probe") / "planner_probe"
    src = ROOT / "paper_2011_02991_gb300" / "csrc"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", str(ROOT / "include"), "-I", str(src), "-o", str(exe),
                        str(ROOT / "tests" / "planner_probe.cu"), str(src / "qng_large_plan.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run_probe(exe, circuit, precision, want=None, with_steps=False):
    """The schedule's reduction destinations {(segment, region): [index]}, and with with_steps its
    recurrence steps [(segment, kind, rotates)] as well."""
    g = np.asarray(circuit.gates, dtype=np.int64)
    lines = [f"{circuit.n} {circuit.num_params} {len(g)} {precision} {-1 if want is None else len(want)}"]
    lines += [" ".join(str(int(v)) for v in row) for row in g]
    if want is not None:
        lines.append(" ".join(str(int(j)) for j in want))
    r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True)
    out = r.stdout.split("\n")
    assert r.returncode == 0 and "ok" in out, f"probe: {[x for x in out if x.startswith('bad')]} {r.stderr}"
    reds = {}
    steps = []
    for x in out:
        if x.startswith("red "):
            _, seg, region, idx = x.split()
            reds.setdefault((int(seg), int(region)), []).append(int(idx))
        elif x.startswith("step "):
            steps.append(tuple(int(v) for v in x.split()[1:]))
    return (reds, steps) if with_steps else reds


def check_coverage(reds, P, cols):
    upper = sorted(i * P + j for j in cols for i in range(j))
    for seg, regions in ((SEG_METRIC, (REG_L,)), (SEG_METRIC_IM, (REG_L, REG_LIM))):
        for reg in regions:
            assert sorted(reds.get((seg, reg), [])) == upper, (seg, reg)
        assert sorted(reds.get((seg, REG_SIGMA), [])) == sorted(cols), seg
    assert sorted(reds.get((SEG_ADJOINT, REG_GRAD), [])) == list(range(P))
    assert reds.get((SEG_ENERGY, REG_ENERGY)) == [0]


CIRCUITS = [
    ("ry_rz_cz_13", lambda: W.layered_ansatz(13, 3)),
    ("ry_rx_rz_cnot_12", lambda: W.layered_ansatz(12, 2, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)),
    ("ry_rx_rz_cnot_14", lambda: W.layered_ansatz(14, 2, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)),
    ("z_runs_12", lambda: W.z_run_problem(12, 150, 21, W.C64).circuit),
    ("z_runs_9", lambda: W.z_run_problem(9, 80, 5, W.C64).circuit),
    ("layered_6", lambda: W.layered_ansatz(6, 4, rotation_kinds=(W.RX, W.RZ), entangler=W.CNOT)),
]


@pytest.mark.parametrize("precision", [W.C64, W.C128])
@pytest.mark.parametrize("name,make", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_schedule_reduces_every_entry_once(probe, name, make, precision):
    c = make()
    reds = run_probe(probe, c, precision)
    check_coverage(reds, c.num_params, list(range(c.num_params)))


@pytest.mark.parametrize("ranks", [2, 3])
@pytest.mark.parametrize("name,make", CIRCUITS[:3], ids=[c[0] for c in CIRCUITS[:3]])
def test_column_subset_schedules(probe, name, make, ranks):
    """Each rank's schedule computes exactly its columns of qng_column_partition; together they
    cover the instance once."""
    from paper_2011_02991_gb300 import qng
    c = make()
    P = c.num_params
    seen = []
    for r in range(ranks):
        cols = list(qng.column_partition(P, ranks, r))
        for precision in (W.C64, W.C128):
            check_coverage(run_probe(probe, c, precision, cols), P, cols)
        seen += cols
    assert sorted(seen) == list(range(P))


def test_subset_breaking_pairs(probe):
    """A subset that holds one column of an adjacent pair (l, l + 1) still computes exactly its
    columns (that column walks alone)."""
    c = W.layered_ansatz(12, 2, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)
    P = c.num_params
    cols = [0, 1, 4, 7, 8, P - 2]
    for precision in (W.C64, W.C128):
        check_coverage(run_probe(probe, c, precision, cols), P, cols)


@pytest.mark.parametrize("P_layers", [1, 2, 3])
def test_bench_flop_count_matches_schedule(probe, P_layers):
    """The roofline's float64 work of the streaming metric segment (bench.stream_flops_per_amp) is
    what the paired schedule runs: per amplitude, 4 flop per inner product and 4 per register
    rotated (scaled form), a single step rotating a and b, a paired one a, b and b2."""
    import bench
    c = W.layered_ansatz(12, P_layers, rotation_kinds=(W.RY, W.RX, W.RZ), entangler=W.CNOT)
    _, steps = run_probe(probe, c, W.C128, with_steps=True)
    flops = 0.0
    for seg, kind, rot in steps:
        if seg != SEG_METRIC:
            continue
        ips, regs = (1, 2) if kind == 8 else (2, 3)
        flops += 4.0 * ips + (4.0 * regs if rot else 0.0)
    assert flops == bench.stream_flops_per_amp(c.num_params)
