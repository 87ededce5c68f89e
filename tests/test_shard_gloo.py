"""The multi-rank partition of an enclosure (x_1-slabs, no data exchange) on gloo ranks.

Rank r of N = 2^s starts Algorithm 3 at level s from the boxes whose x_1 index is r and runs it
to the full depth (CPU oracle); gathering the survivors in rank order must give the
single-process result exactly, in lexicographic order.  The gather is test-only: the benchmark
never exchanges boxes.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2406_09857_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _system():
    return synth.random_small(3, 5, 2, 4242), synth.cube(3), 5


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    polys, dom, depth = _system()
    s, start = shard.rank_start(3, depth, rank, world)
    mine = oracle.enclose(polys, dom, depth, start_level=s, start=start)["tuples"]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        np.save(out, np.concatenate(gathered, axis=0))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slab_shards_reproduce_the_full_enclosure(tmp_path, world):
    out = str(tmp_path / "gathered.npy")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    polys, dom, depth = _system()
    full = oracle.enclose(polys, dom, depth)["tuples"]
    assert full.shape[0] > 0
    assert np.array_equal(got, full)


def test_rank_start_geometry():
    s, t = shard.rank_start(3, 10, 3, 4)
    assert s == 2 and t.shape == (16, 3)
    assert np.all(t[:, 0] == 3) and np.array_equal(t[np.lexsort(t.T[::-1])], t)
    assert shard.rank_start(1, 5, 1, 2)[1].tolist() == [[1]]
    with pytest.raises(ValueError):
        shard.rank_start(3, 10, 0, 3)
    with pytest.raises(ValueError):
        shard.rank_start(3, 1, 0, 4)
