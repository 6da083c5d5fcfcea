"""Multi-rank host logic on CPU (gloo, world_size 2): frames shard across ranks with no
data-path exchange, error counts and elapsed times reduce across ranks, and the sharded
result equals a single-process decode."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2108_12550_gb300 import inputs as I
from paper_2108_12550_gb300 import replicas


def test_shards_cover_every_frame_once():
    for n in [0, 1, 7, 100, 262144]:
        for world in [1, 2, 3, 8]:
            seen = []
            for rank in range(world):
                s, c = replicas.shard(n, world, rank)
                seen.extend(range(s, s + c))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle as O

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, r, P, L = 5, 2, 4, 2
    fr = I.make_frames(m, r, 301, 1.5, seed=12)
    start, count = replicas.shard(301, world, rank)
    out = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=2), fr["llr"][start:start + count], n_threads=1)
    errs = int(np.sum(np.any(out["info"] != fr["u"][start:start + count], axis=1)))
    tot_errs, tot_frames = replicas.allreduce_sum([errs, count])
    tmax = replicas.allreduce_max(float(rank + 1))
    if rank == 0:
        np.save(out_path, np.array([tot_errs, tot_frames, tmax]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import oracle as O

    out_path = str(tmp_path / "res.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out_path), nprocs=2, join=True)
    tot_errs, tot_frames, tmax = np.load(out_path)
    m, r, P, L = 5, 2, 4, 2
    fr = I.make_frames(m, r, 301, 1.5, seed=12)
    ref = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=2), fr["llr"])
    assert tot_frames == 301 and tmax == 2.0
    assert tot_errs == int(np.sum(np.any(ref["info"] != fr["u"], axis=1)))
