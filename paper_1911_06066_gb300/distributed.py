"""Multi-device MLMC and checkpoint / resume on top of the C ABI.

The samples of an MLMC estimator are independent (Sec. 3: every level's
correction is a plain Monte Carlo mean of i.i.d. pairs), and every sample's
random input is a function of (seed, level, sample id) alone.  So a run over
several devices shards the sample ids of each level across ranks, every rank
runs its shard with ``mlmc_run_more`` on its own device with no exchange on
the data path, and the only collective is one all-gather of the per-level
accumulator states at the end, merged on the host in rank order with
``mlmc_merge_states`` (the pairwise update of Chan, Golub and LeVeque).
Every rank ends with the same merged state.

Checkpointing is the same state written to a file together with the next
sample id of every level; resuming loads it into a context and continues
from those ids, so an interrupted run gives the sample set of an
uninterrupted one.
"""
import json

import numpy as np

from .binding import State


def shard(N_l, rank, world):
    """Per-level (first_id, count) of this rank's contiguous share of ids
    0 .. N_l[l]-1; shares differ in size by at most one."""
    first, count = [], []
    for n in N_l:
        n = int(n)
        q, r = divmod(n, world)
        lo = rank * q + min(rank, r)
        first.append(lo)
        count.append(q + (1 if rank < r else 0))
    return np.array(first, np.int64), np.array(count, np.int64)


def allgather_states(state, group=None):
    """All-gather of one State per rank; returns the list in rank order.

    One collective of a flat float64 vector (counts carried exactly: they are
    far below 2^53).  On an NCCL group the vector travels through the current
    CUDA device; on gloo it stays on the host.
    """
    import torch
    import torch.distributed as dist

    L, n0 = state.mean.shape
    flat = torch.from_numpy(state.as_array())
    if dist.get_backend(group) == "nccl":
        flat = flat.cuda()
    parts = [torch.empty_like(flat) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, flat, group=group)
    return [State.from_array(p.cpu().numpy(), L, n0) for p in parts]


def merge_in_order(states):
    """Rank-ordered merge (the same order on every rank, so every rank gets
    bitwise the same result)."""
    L, n0 = states[0].mean.shape
    acc = State.empty(L, n0)
    for s in states:
        acc.merge(s)
    return acc


def run_sharded(ctx, N_l, seed=0, batch=None, group=None, stream=None):
    """Fixed-count MLMC over all ranks of ``group``: each rank runs its id
    shard on its own device, then the states are gathered and merged, loaded
    back into ``ctx`` and estimated.  Returns ctx.estimate() plus this rank's
    per-level solve seconds."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, count = shard(N_l, rank, world)
    ctx.reset(stream)
    secs = ctx.run_more(first, count, seed=seed, batch=batch, stream=stream)
    merged = merge_in_order(allgather_states(ctx.get_state(stream), group))
    ctx.set_state(merged, stream)
    out = ctx.estimate(stream)
    out["solve_seconds"] = secs
    return out


def save_checkpoint(path, state, next_id, seed, meta=None):
    """Writes the accumulator state, the next sample id per level and the
    seed to ``path`` (a .npz file).  ``meta`` (JSON-serialisable) identifies
    the configuration and is checked on load by the caller."""
    np.savez(path, N=state.N, mean=state.mean, m2=state.m2, mean2=state.mean2,
             next_id=np.asarray(next_id, np.int64), seed=np.uint64(seed),
             meta=json.dumps(meta or {}))


def load_checkpoint(path):
    """Returns (state, next_id, seed, meta) written by save_checkpoint."""
    z = np.load(path)
    st = State(z["N"], z["mean"], z["m2"], z["mean2"])
    return st, z["next_id"].astype(np.int64), int(z["seed"]), json.loads(str(z["meta"]))
