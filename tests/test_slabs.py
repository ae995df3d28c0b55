"""Host bookkeeping of the row-slab decomposition (paper_2406_09654_gb300/slabs.py), on the CPU:
the row partition, the ghost-row sources (checked by assembling slabs from a world array), the
combine of the radiation scans, and the same combine and ghost-row exchange across two gloo
processes (one slab per rank)."""
import os

import numpy as np
import pytest

from paper_2406_09654_gb300 import slabs


def test_partition_covers_rows_in_order():
    for H, n in [(3, 1), (7, 2), (100, 3), (97, 4), (12, 4)]:
        parts = slabs.partition_rows(H, n)
        assert parts[0][0] == 0 and parts[-1][1] == H
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [y1 - y0 for y0, y1 in parts]
        assert min(sizes) >= slabs.GHOST and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.partition_rows(11, 4)


@pytest.mark.parametrize("H,n", [(9, 1), (20, 2), (31, 3), (40, 4)])
def test_ghost_copies_reproduce_the_torus_rows(H, n):
    rng = np.random.default_rng(H + n)
    world = rng.random((H, 5))
    parts = slabs.partition_rows(H, n)
    G = slabs.GHOST
    # slab arrays: own rows filled, ghost rows garbage; then the copies of ghost_copies
    arrs = []
    for (y0, y1) in parts:
        a = np.full((slabs.slab_height(y0, y1), 5), np.nan)
        a[G:G + (y1 - y0)] = world[y0:y1]
        arrs.append(a)
    src = [a.copy() for a in arrs]
    for r in range(n):
        for dst_row, s, src_row, k in slabs.ghost_copies(parts, r):
            arrs[r][dst_row:dst_row + k] = src[s][src_row:src_row + k]
    for (y0, y1), a in zip(parts, arrs):
        rows = np.arange(y0 - G, y1 + G) % H
        assert np.array_equal(a, world[rows])


def test_combine_radiation_or_concat_sum():
    cap = 8
    a = (np.array([1, 0, 0, 1, 0, 0, 0, 0], np.uint8), np.array([[5, 0, -1, 1, 0], [9, 3, 2, 2, 7]], np.int32),
         np.array([2, 1, 1, 2], np.int32))
    b = (np.array([0, 0, 1, 1, 0, 0, 0, 0], np.uint8), np.array([[40, 2, -1, 1, 0]], np.int32),
         np.array([1, 1, 0, 1], np.int32))
    live, hits, counts = slabs.combine_radiation([a, b])
    assert live.tolist() == [1, 0, 1, 1, 0, 0, 0, 0] and len(live) == cap
    assert hits[:, 0].tolist() == [5, 9, 40]
    assert counts.tolist() == [3, 2, 1]
    tot = slabs.combine_totals([np.arange(6.0), np.ones(6)])
    assert tot.tolist() == [1, 2, 3, 4, 5, 6]


def _dist_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(rank)
        cap = 16
        live = (rng.random(cap) < 0.3).astype(np.uint8)
        k = 2 + rank
        hits = np.c_[1000 * rank + np.arange(k), rng.integers(0, cap, (k, 2)), np.ones(k), np.zeros(k)].astype(np.int32)
        counts = np.array([k, k, 0, k], np.int32)
        got = slabs.combine_radiation_dist(live, hits, counts)
        top = np.full((slabs.GHOST, 4), 10.0 * rank + 1, np.float32)
        bot = np.full((slabs.GHOST, 4), 10.0 * rank + 2, np.float32)
        north, south = slabs.exchange_rows_dist(top, bot)
        q.put((rank, (live, hits, counts), got, north[0, 0], south[0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_exchange_like_one_process():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dist_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scans = [r[1] for r in res]
    live, hits, counts = slabs.combine_radiation(scans)
    for _, _, got, north, south in res:
        assert np.array_equal(got[0], live) and np.array_equal(got[1], hits) and np.array_equal(got[2], counts)
    # rank 0's north ghost rows are rank 1's last own rows (the torus wraps), its south ghost rows
    # rank 1's first own rows; and the other way round
    assert (res[0][3], res[0][4]) == (12.0, 11.0)
    assert (res[1][3], res[1][4]) == (2.0, 1.0)
