"""Sharding over ranks (CPU, gloo, world size 2): brick ranges partition the volume, and the shared
tables built from the ranks' summed prepass counts equal the tables of the whole volume."""
import os

import numpy as np
import torch.multiprocessing as mp

import oracle as O
from paper_2308_16619_b300 import shard


def test_brick_ranges_partition():
    for n in (1, 7, 64, 4096, 32769):
        for w in (1, 2, 3, 8):
            got = [shard.brick_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[i][1] == got[i + 1][0] for i in range(w - 1))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1


def _worker(rank, world, port, counts, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = shard.shared_tables(counts[rank])
    q.put((rank, list(t.freq), list(t.counts)))
    dist.destroy_process_group()


def test_shared_tables_gloo_world2():
    import synth
    vol = synth.voronoi((64, 64, 128), 120, seed=9, warp_amp=4, bg_permille=300)
    # each "rank" owns one half of the volume along x (two 64^3 halves = two brick ranges of b=16 bricks)
    halves = [np.ascontiguousarray(vol[:, :, :64]), np.ascontiguousarray(vol[:, :, 64:])]
    counts = []
    for h in halves:
        ci, cl = O.count_nibbles(h, 4, stride=1)
        counts.append(np.concatenate([ci, cl]))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, counts, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1]  # same tables on both ranks
    total = counts[0] + counts[1]
    assert res[0][2] == list(total)
    # the shared table equals the oracle's normalisation of the summed counts
    want = np.concatenate([O.normalize(total[:16]), O.normalize(total[16:])])
    assert res[0][1] == want.tolist()
