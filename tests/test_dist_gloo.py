"""The multi-process path on CPU: two gloo ranks shard a batch, compute their instances with the
oracle (the GPU kernels are not needed to test the partition and the gather), gather the
per-instance dtheta on every rank, and compare with a single-process computation."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2011_02991_gb300 import dist as D
from paper_2011_02991_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, count, out_dir):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs = W.config_batch(count=count, n_range=(2, 4), layer_range=(1, 3), term_range=(2, 4))
        shards = D.shard_batch(probs, world)
        local = {b: O.qng_step(probs[b])["dtheta"] for b in shards[rank]}
        D.barrier()
        allv = D.gather_per_instance(local, count)
        t = D.max_over_ranks(float(rank + 1))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate(allv))
        np.save(os.path.join(out_dir, f"rank{rank}_max.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_shard_batch_is_a_balanced_partition():
    probs = W.config_batch(count=64)
    for ws in (1, 2, 3, 8):
        shards = D.shard_batch(probs, ws)
        flat = sorted(b for s in shards for b in s)
        assert flat == list(range(64))
        loads = [sum(D.instance_cost(probs[b]) for b in s) for s in shards]
        biggest = max(D.instance_cost(p) for p in probs)
        assert max(loads) - min(loads) <= biggest  # LPT bound


def test_two_gloo_ranks_gather(tmp_path):
    count, world = 10, 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, count, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    from oracle import oracle as O
    probs = W.config_batch(count=count, n_range=(2, 4), layer_range=(1, 3), term_range=(2, 4))
    ref = np.concatenate([O.qng_step(p)["dtheta"] for p in probs])
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        np.testing.assert_array_equal(got, ref)
        assert np.load(tmp_path / f"rank{r}_max.npy")[0] == float(world)


def _column_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2011_02991_gb300 import qng
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.random_problem(5, 70, 6, 9191)
        P = p.P
        cols = qng.column_partition(P, world, rank)
        L, T = O.alg1_columns(p.circuit, p.theta, cols)  # this rank's columns of Algorithm 1
        Lt = torch.view_as_real(torch.from_numpy(L)).contiguous()
        Tt = torch.view_as_real(torch.from_numpy(T)).contiguous()
        L_all = [torch.empty_like(Lt) for _ in range(world)]
        T_all = [torch.empty_like(Tt) for _ in range(world)]
        dist.all_gather(L_all, Lt)
        dist.all_gather(T_all, Tt)
        owner = D.column_owners(P, world)
        Lm, Tm = D.merge_columns([torch.view_as_complex(x) for x in L_all], [torch.view_as_complex(x) for x in T_all],
                                 owner)
        np.save(os.path.join(out_dir, f"L{rank}.npy"), Lm.numpy())
        np.save(os.path.join(out_dir, f"T{rank}.npy"), Tm.numpy())
    finally:
        dist.destroy_process_group()


def test_column_partition_two_gloo_ranks(tmp_path):
    """Sec. 3's column independence: two ranks each run Algorithm 1's inner loop for their balanced
    column pairs only (psi still advances through every gate), all-gather the columns of L and T,
    and the merged L, T and the assembled G equal the single-process Algorithm 1 bit for bit."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_column_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    from oracle import oracle as O
    p = W.random_problem(5, 70, 6, 9191)
    L, T, _, _ = O.alg1(p.circuit, p.theta)
    iu = np.triu_indices(p.P, 1)
    G = O.hermitian_from_upper(L) - np.outer(T.conj(), T)
    for r in range(world):
        Lm = np.load(tmp_path / f"L{r}.npy")
        Tm = np.load(tmp_path / f"T{r}.npy")
        np.testing.assert_array_equal(Lm[iu], L[iu])  # the entries the recurrence computes, i < j
        np.testing.assert_array_equal(Tm, T)
        Lfull = Lm.copy()
        np.fill_diagonal(Lfull, 0.25)  # L_jj = 1/4 a priori (Eq. L_diag_when_single_pauli)
        Gm = O.hermitian_from_upper(Lfull) - np.outer(Tm.conj(), Tm)
        np.testing.assert_array_equal(Gm, G)


def test_column_partition_is_balanced():
    from paper_2011_02991_gb300 import qng
    for P in (0, 1, 2, 7, 16, 192, 208, 252):
        for R in (1, 2, 3, 4, 8):
            parts = [qng.column_partition(P, R, r) for r in range(R)]
            assert sorted(j for c in parts for j in c) == list(range(P))
            work = [sum(j for j in c) for c in parts]  # column j has j recurrence steps
            # at most one group (two balanced pairs, 2P steps at most) apart
            assert max(work) - min(work) <= max(2 * P, 0)
            # the adjacent pairs (l, l + 1), l odd, stay on one rank
            for c in parts:
                s = set(c)
                assert all((l + 1 in s) == (l in s) for l in range(1, P - 1, 2))
