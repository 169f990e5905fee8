"""Multi-process helpers: one process per GPU, launched by torch.distributed.run.

Two ways the path shards:
  - batches: instances are independent problems. `shard_batch` gives each rank a balanced share of
    them, and `gather_per_instance` brings the per-instance results to every rank after the step,
    once per step, outside the compute path (no collective on the data path);
  - one instance (the column partition, Sec. 3: Algorithm 1's inner loop for column j reads only
    psi_{j-1}, so the columns of L are independent): every rank computes its balanced column pairs
    (`column_partition`, qng_column_partition), then one all-gather of the columns of L and of
    sigma (`gather_columns`) lets each rank assemble G and solve (`sharded_step`).
Timing follows the benchmark contract: a barrier on both sides of the timed region and the slowest
rank's time (`max_over_ranks`).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def instance_cost(problem) -> float:
    """Work of one instance: (P^2 / 2) recurrence steps over 2^n amplitudes each."""
    return float(problem.P * problem.P) * float(1 << problem.n)


def shard_batch(problems, world_size: int) -> list[list[int]]:
    """Longest-processing-time-first partition of instance indices over ranks (deterministic)."""
    order = sorted(range(len(problems)), key=lambda b: (-instance_cost(problems[b]), b))
    load = [0.0] * world_size
    shards: list[list[int]] = [[] for _ in range(world_size)]
    for b in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        shards[r].append(b)
        load[r] += instance_cost(problems[b])
    return [sorted(s) for s in shards]


def gather_per_instance(local: dict[int, np.ndarray], count: int) -> list[np.ndarray]:
    """Every rank's {instance index: float64 vector} to a list ordered by instance, on every rank."""
    rank, ws = world()
    if ws == 1:
        return [local[b] for b in range(count)]
    items = sorted(local.items())
    idx = torch.tensor([b for b, _ in items] + [-1], dtype=torch.int64)
    lens = torch.tensor([len(v) for _, v in items] + [0], dtype=torch.int64)
    flat = torch.from_numpy(np.concatenate([v for _, v in items]) if items else np.zeros(0)).to(torch.float64)
    # sizes first, then padded payloads
    n_items = torch.tensor([len(items)], dtype=torch.int64)
    n_flat = torch.tensor([flat.numel()], dtype=torch.int64)
    all_items = [torch.zeros(1, dtype=torch.int64) for _ in range(ws)]
    all_flat = [torch.zeros(1, dtype=torch.int64) for _ in range(ws)]
    dist.all_gather(all_items, n_items)
    dist.all_gather(all_flat, n_flat)
    mi = int(max(t.item() for t in all_items)) + 1
    mf = max(int(max(t.item() for t in all_flat)), 1)
    pad_idx = torch.full((mi,), -1, dtype=torch.int64)
    pad_idx[: idx.numel()] = idx
    pad_len = torch.zeros(mi, dtype=torch.int64)
    pad_len[: lens.numel()] = lens
    pad_flat = torch.zeros(mf, dtype=torch.float64)
    pad_flat[: flat.numel()] = flat
    g_idx = [torch.zeros(mi, dtype=torch.int64) for _ in range(ws)]
    g_len = [torch.zeros(mi, dtype=torch.int64) for _ in range(ws)]
    g_flat = [torch.zeros(mf, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(g_idx, pad_idx)
    dist.all_gather(g_len, pad_len)
    dist.all_gather(g_flat, pad_flat)
    out: list[np.ndarray | None] = [None] * count
    for r in range(ws):
        off = 0
        for b, n in zip(g_idx[r].tolist(), g_len[r].tolist()):
            if b < 0:
                break
            out[b] = g_flat[r][off:off + n].numpy().copy()
            off += n
    missing = [b for b in range(count) if out[b] is None]
    if missing:
        raise RuntimeError(f"gather_per_instance: no rank returned instances {missing[:8]}")
    return out  # type: ignore[return-value]


def max_over_ranks(value: float, device=None) -> float:
    rank, ws = world()
    if ws == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    if world()[1] > 1:
        dist.barrier()


def column_owners(P: int, world_size: int) -> np.ndarray:
    """owner[j]: the rank that computes metric column j (qng_column_partition)."""
    from . import qng
    owner = np.full(P, -1, dtype=np.int64)
    for r in range(world_size):
        owner[qng.column_partition(P, world_size, r)] = r
    return owner


def merge_columns(L_all, sigma_all, owner: np.ndarray):
    """Every rank's L (P x P) and sigma (P) -> one L and sigma: column j (its entries i < j, the
    only ones the recurrence writes) and sigma[j] from the rank that owns j."""
    P = owner.size
    L = torch.zeros(P, P, dtype=L_all[0].dtype, device=L_all[0].device)
    sigma = torch.zeros(P, dtype=sigma_all[0].dtype, device=sigma_all[0].device)
    iu = torch.triu_indices(P, P, offset=1, device=L.device)
    own = torch.as_tensor(owner, device=L.device)
    for r, (Lr, sr) in enumerate(zip(L_all, sigma_all)):
        Lr = Lr.reshape(P, P)
        sel = own[iu[1]] == r
        L[iu[0][sel], iu[1][sel]] = Lr[iu[0][sel], iu[1][sel]]
        sigma[own == r] = sr.reshape(P)[own == r]
    return L, sigma


def gather_columns(L_local, sigma_local, owner: np.ndarray):
    """All-gather every rank's partial L and sigma (one collective each) and merge them."""
    rank, ws = world()
    if ws == 1:
        return merge_columns([L_local], [sigma_local], owner)
    L_all = [torch.empty_like(L_local) for _ in range(ws)]
    s_all = [torch.empty_like(sigma_local) for _ in range(ws)]
    dist.all_gather(L_all, L_local.contiguous())
    dist.all_gather(s_all, sigma_local.contiguous())
    return merge_columns(L_all, s_all, owner)


def sharded_step(ctx, theta, dt: float, lam: float):
    """One QNG step of a single-instance context with the metric columns split over the ranks: the
    rank's columns (qng_metric_columns), one all-gather, assembly and solve on every rank
    (qng_step_from_parts). Returns dict(dtheta, g, grad, energy). The context must have been
    restricted to this rank's columns with ctx.set_column_subset(column_partition(...))."""
    rank, ws = world()
    P = ctx.total_params
    parts = ctx.metric_columns(theta)
    owner = column_owners(P, ws)
    L, sigma = gather_columns(parts["L"], parts["sigma"], owner)
    out = ctx.step_from_parts(theta, L.reshape(-1), sigma, parts["grad"], dt, lam)
    out["grad"], out["energy"] = parts["grad"], parts["energy"]
    return out
