"""GPU: the pipelined checkpoint sweep (chunks of parameters on a high-priority stream, the columns
each chunk makes ready on streams of their own) against the unchunked sweep and the oracle.

Column j of Algorithm 1's recurrence reads only the checkpoints psi_0..psi_j, and a chunk that
restarts from checkpoint K carries that checkpoint exactly as the uninterrupted sweep carried it
(renormalisation by 2^200 is exact), so every output is bit-identical to the unchunked sweep.
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


def _step(ctx, chunks, th, dt=0.1, lam=1e-3):
    ctx.set_pipeline(chunks)
    out = ctx.step(th, dt, lam)
    ctx.sync()
    return {k: v.clone() for k, v in out.items()}


def _same(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [W.C128, W.C64])
def test_chunk_counts_bit_identical(qng, oracle, precision):
    """12 qubits, P = 192: 2..8 chunks (boundaries every P/S parameters, P/S not whole for 5 and 7)
    give the unchunked step's outputs bit for bit, and the step matches the oracle."""
    p = W.config_rand12(precision=precision)
    ctx = qng.Context(p, precision=precision)
    th = ctx.theta0()
    ctx.set_pipeline(0)
    assert ctx.pipeline() == 0  # automatic: plain rotations run unchunked
    ref = _step(ctx, 1, th)
    assert ctx.pipeline() == 0
    for chunks in (2, 3, 4, 5, 7, 8):
        _same(_step(ctx, chunks, th), ref)
    o = oracle.qng_step(p)
    for key in ("g", "grad", "dtheta"):
        if precision == W.C64 and key == "dtheta":
            continue  # float32 rounding in near-singular directions; the c64 solve is checked by its residual
        assert rel(ref[key].cpu(), o[key]) <= TOL[precision], key


@pytest.mark.parametrize("chunks", [3, 6, 8])
def test_chunks_cut_z_runs_and_renormalisations(qng, chunks):
    """P = 1000 on 7 qubits with long runs of RZ (fused into one pass each) and angles near pi/2
    (the float64 scale crosses 2^-200 many times): chunk ends clip runs and restart next to
    renormalisations, and the outputs stay bit-identical."""
    p = W.z_run_problem(7, 1000, 6, W.C128, near_half_pi=True)
    ctx = qng.Context(p, precision=W.C128)
    ctx.set_shape(7, 0, 64, 64)
    th = ctx.theta0()
    ref = _step(ctx, 1, th)
    _same(_step(ctx, chunks, th), ref)


def test_generalised_rotations_pipelined(qng, oracle):
    """Controlled and Pauli-string rotations (their own kernel instantiations) through 4 chunks."""
    p = W.general_problem(8, 150, 11, W.C128)
    ctx = qng.Context(p, precision=W.C128)
    th = ctx.theta0()
    ref = _step(ctx, 1, th)
    out = _step(ctx, 4, th)
    _same(out, ref)
    o = oracle.qng_step(p)
    for key in ("g", "grad", "dtheta"):
        assert rel(out[key].cpu(), o[key]) <= TOL[W.C128], key


def test_metric_only_and_complex_metric_pipelined(qng):
    """qng_metric (no gradient column) and qng_metric_complex take the pipelined sweep too."""
    p = W.config_rand12()
    ctx = qng.Context(p)
    th = ctx.theta0()
    res = {}
    for chunks in (1, 4):
        ctx.set_pipeline(chunks)
        g, sg = ctx.metric(th, want_sigma=True)
        G = ctx.metric_complex(th)
        gr, en = ctx.gradient(th)
        ctx.sync()
        res[chunks] = (g.clone(), sg.clone(), G.clone(), gr.clone(), en.clone())
    for a, b in zip(res[1], res[4]):
        assert torch.equal(a, b)


def test_graph_capture_and_descent_pipelined(qng):
    """A captured graph of a pipelined step (fork and join across four streams) replays to the
    direct step's outputs, and qng_optimize follows the same trajectory as without chunks."""
    p = W.vqe_tfim(10, 8, seed=3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = qng.Context(p, stream=stream)
        th = ctx.theta0()
        ref = _step(ctx, 4, th)
        out = ctx.graph_capture(th, 0.1, 1e-3)
        for _ in range(2):
            for v in out.values():
                v.fill_(float("nan"))
            ctx.graph_launch()
            ctx.sync()
            _same(out, ref)
        runs = {}
        for chunks in (1, 4):
            ctx.set_pipeline(chunks)
            t = ctx.theta0().clone()
            en = ctx.optimize(t, 0.1, 1e-3, 5)
            ctx.sync()
            runs[chunks] = (t, en)
        assert torch.equal(runs[1][0], runs[4][0]) and torch.equal(runs[1][1], runs[4][1])


def test_pipeline_applies_to_single_on_chip_instances(qng):
    """Automatic chunking: one on-chip instance with generalised rotations and P >= 64; plain
    rotations, batches and small P run unchunked, and the setting is validated."""
    small = qng.Context(W.z_run_problem(6, 40, 2, W.C128))
    assert small.pipeline() == 0
    batch = qng.Context(W.config_batch(count=4))
    batch.set_pipeline(4)
    assert batch.pipeline() == 0
    ctx = qng.Context(W.config_rand12())
    assert ctx.pipeline() == 0
    gen = qng.Context(W.general_problem(8, 150, 11, W.C128))
    assert gen.pipeline() == 3
    ctx.set_pipeline(8)
    assert ctx.pipeline() == 8
    with pytest.raises(qng.QngError):
        ctx.set_pipeline(9)


@pytest.mark.parametrize("fwd_threads", [64, 128, 256])
def test_sweep_on_sixteen_ctas(qng, oracle, fwd_threads):
    """The checkpoint sweep on a 16-CTA cluster (the column kernel stays on 8): each amplitude goes
    through the same float64 operations whichever CTA holds it, so g, grad and dtheta are
    bit-identical; <E> is a cluster-wide sum taken in another order."""
    p = W.config_rand12()
    ctx = qng.Context(p)
    th = ctx.theta0()
    ctx.set_forward_cluster(12, 3)
    ref = _step(ctx, 1, th)
    ctx.set_forward_cluster(12, 4)
    ctx.set_shape(12, 3, 128, fwd_threads)
    assert ctx.forward_cluster(12) == 4 and ctx.get_tuning(12)[0] == 3
    for chunks in (1, 3):
        out = _step(ctx, chunks, th)
        for k in ("g", "grad", "dtheta"):
            assert torch.equal(out[k], ref[k]), k
        assert rel(out["energy"].cpu(), ref["energy"].cpu()) <= 1e-14
    o = oracle.qng_step(p)
    assert rel(out["energy"].cpu(), [o["E"]]) <= TOL[W.C128]
    ctx.set_forward_cluster(12, 3)
    assert ctx.forward_cluster(12) == 3
    ctx.set_forward_cluster(12, -1)  # default for one instance: twice the column kernel's CTAs
    assert ctx.forward_cluster(12) == 4
    batch = qng.Context(W.config_batch(count=4))
    assert all(batch.forward_cluster(n) == batch.get_tuning(n)[0] for n in range(6, 15))
