"""Worker functions for the multi-process (gloo, CPU) tests.  Kept in their
own module so that spawned children import them without the test module."""
import os

import numpy as np


def oracle_shard_state(w, rank, world, seed):
    """This rank's accumulator state from oracle pairs of its id shard."""
    import oracle as O
    from helpers import oracle_levels
    from paper_1911_06066_gb300.binding import State
    from paper_1911_06066_gb300.distributed import shard

    lv = oracle_levels(w)
    n0 = lv[0].nodes
    first, count = shard(w["N"], rank, world)
    st = State.empty(w["levels"], n0)
    for l in range(w["levels"]):
        Y, Y2 = O.level_pairs(lv, l, w["sigma2"], w["ell"], w["M"], seed,
                              range(first[l], first[l] + count[l]))
        wy, wy2 = O.Welford(n0), O.Welford(n0)
        for r in range(Y.shape[0]):
            wy.add(Y[r])
            wy2.add(Y2[r])
        st.N[l] = count[l]
        st.mean[l], st.m2[l], st.mean2[l] = wy.mean, wy.m2, wy2.mean
    return st


def gloo_merge_worker(rank, world, port, w, seed, out_dir):
    import torch.distributed as dist
    from paper_1911_06066_gb300.distributed import allgather_states, merge_in_order

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = oracle_shard_state(w, rank, world, seed)
        merged = merge_in_order(allgather_states(st))
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), N=merged.N, mean=merged.mean,
                 m2=merged.m2, mean2=merged.mean2)
    finally:
        dist.destroy_process_group()


def gloo_fail_worker(rank, world, port, out_dir):
    """Rank 1 raises before the collective; rank 0's gather must end with an
    error (short process-group timeout), not hang."""
    import datetime

    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise RuntimeError("rank 1 fails before the exchange")
    try:
        parts = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.ones(4, dtype=torch.float64))
        open(os.path.join(out_dir, "rank0.txt"), "w").write("completed")
    except Exception as e:  # the expected outcome
        open(os.path.join(out_dir, "rank0.txt"), "w").write("error: %s" % type(e).__name__)
