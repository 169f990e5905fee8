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
