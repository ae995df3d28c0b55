"""Row-slab decomposition of one world (logical ranks).

The substrate update is synchronous and local (Section "System Design": every cell is updated
from its neighbourhood in discrete steps), so one world can be split into horizontal slabs of
rows, one substrate per slab. A slab substrate holds its own rows plus GHOST copied rows above
and below; before every step the ghost rows are refreshed from the neighbouring slabs' own rows
(a step's new state depends on the old state within two rows; radiation's merge partner is one
row away, and the third ghost row's post-step state is exact). Radiation is global: every slab
scans its own rows (which slots own a cell, which cells are hit), the scans are combined (OR of
the liveness flags, the hit lists concatenated in slab order = global cell order, counts summed)
and every slab applies the same combined result to its copy of the genome table. The results are
bit-identical to one substrate holding the whole world.

Host bookkeeping (partition, ghost-row sources, the combine) is plain Python, shared by the
single-process form (``SlabWorld``: several substrates on one device) and the multi-process form
(``combine_radiation_dist`` / ``exchange_rows_dist`` over a torch.distributed process group).
All arithmetic of the step stays in the CUDA library.
"""
from __future__ import annotations

import numpy as np

GHOST = 3        # ghost rows above and below a slab's own rows


def partition_rows(height: int, n_ranks: int):
    """Contiguous row ranges [y0, y1) of n_ranks slabs, sizes differing by at most one, each at
    least GHOST rows (so that a slab's ghost rows come from its two neighbours' own rows)."""
    if n_ranks < 1 or height < GHOST * n_ranks:
        raise ValueError(f"{height} rows cannot be split into {n_ranks} slabs of at least {GHOST} rows")
    base, extra = divmod(height, n_ranks)
    out, y = [], 0
    for r in range(n_ranks):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def slab_height(y0: int, y1: int) -> int:
    """Rows of a slab substrate: its own rows and GHOST ghost rows on each side."""
    return (y1 - y0) + 2 * GHOST


def ghost_copies(parts, r: int):
    """The row copies that refresh slab r's ghost rows: (dst_row, src_rank, src_row, n_rows), with
    rows local to the slabs' substrates (own rows start at local row GHOST). North ghost rows are
    the last GHOST own rows of the slab above (the torus wraps: slab 0's are the last slab's), south
    ghost rows the first GHOST own rows of the slab below."""
    n = len(parts)
    up, down = (r - 1) % n, (r + 1) % n
    hu = parts[up][1] - parts[up][0]
    hr = parts[r][1] - parts[r][0]
    return [(0, up, GHOST + hu - GHOST, GHOST), (GHOST + hr, down, GHOST, GHOST)]


def combine_radiation(scans):
    """Combines the slabs' radiation scans, given in slab order as (live [cap] uint8, hits [k][5]
    int32, counts [4] int32): the OR of the liveness flags, the hit lists concatenated (slab order
    is global cell order), and the summed counts (hits, mutation hits, merge hits)."""
    live = np.zeros_like(scans[0][0])
    for lv, _, _ in scans:
        live |= lv
    hits = np.concatenate([h.reshape(-1, 5) for _, h, _ in scans]).astype(np.int32)
    counts = np.sum([c[:3] for _, _, c in scans], axis=0).astype(np.int32)
    return live, hits, counts


def combine_totals(per_slab):
    """Global FP64 totals (E, I, C0..C3) from the slabs' own-row totals, added in slab order."""
    tot = np.zeros(6)
    for t in per_slab:
        tot = tot + np.asarray(t, np.float64)
    return tot


# ------------------------------------------------------------------ one process, many slabs

class SlabWorld:
    """One world as n_ranks row slabs on the current device (logical ranks in one process)."""

    def __init__(self, world, n_ranks: int, path=None, stream=None):
        from . import coral
        self.coral = coral
        self.world = world
        self.parts = partition_rows(world.height, n_ranks)
        self.path = coral.BF16_GROUPED if path is None else path
        self.radiation_every = int(world.physics.get("radiation_every", 0))
        W = world.width
        self.subs = []
        for (y0, y1) in self.parts:
            rows = np.r_[np.arange(y0 - GHOST, y0), np.arange(y0, y1), np.arange(y1, y1 + GHOST)] % world.height
            p = coral.params_from_world(world, self.path)
            s = coral.Substrate(p, W, slab_height(y0, y1), world.capacity, stream)
            s.load_state(np.ascontiguousarray(world.E[rows]), np.ascontiguousarray(world.I[rows]),
                         np.ascontiguousarray(world.C[:, rows]), np.ascontiguousarray(world.G[rows]),
                         np.ascontiguousarray(world.R[rows]))
            s.load_genomes(genes=world.genes, dense=world.dense, n=world.n_genomes)
            if world.genes is not None:
                s.generate_weights()
            s.slab_set(GHOST, GHOST + (y1 - y0), y0 * W)
            self.subs.append(s)

    def set_step(self, t):
        for s in self.subs:
            s.set_step(t)

    def exchange(self):
        for r, s in enumerate(self.subs):
            for dst_row, src, src_row, n in ghost_copies(self.parts, r):
                s.copy_rows_from(dst_row, self.subs[src], src_row, n)

    def step(self, n=1):
        for _ in range(int(n)):
            self.exchange()
            for s in self.subs:
                s.step(1)
            t = self.subs[0].get_step() - 1
            if self.radiation_every and (t + 1) % self.radiation_every == 0:
                # no exchange first: a merge partner is at most one row from the own rows, and
                # the ghost row next to them holds its exact post-step state
                live, hits, counts = combine_radiation([s.slab_radiation_scan() for s in self.subs])
                for s in self.subs:
                    s.slab_radiation_apply(live, hits, counts)

    def read_channels(self):
        """The whole world's planes, assembled from the slabs' own rows."""
        parts = []
        for (y0, y1), s in zip(self.parts, self.subs):
            d = s.read_channels()
            parts.append({k: (v[:, GHOST:GHOST + (y1 - y0)] if k == "C" else v[GHOST:GHOST + (y1 - y0)])
                          for k, v in d.items()})
        out = {}
        for k in parts[0]:
            out[k] = np.concatenate([p[k] for p in parts], axis=1 if k == "C" else 0)
        return out

    def read_genomes(self):
        return self.subs[0].read_genomes()

    def totals(self):
        return combine_totals([s.slab_totals() for s in self.subs])

    def close(self):
        for s in self.subs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ one slab per process

def combine_radiation_dist(live, hits, counts, group=None):
    """combine_radiation across the ranks of a torch.distributed group (rank order = slab order):
    an all-reduce (max) of the liveness flags, an all-gather of the hit counts and the padded hit
    lists, and an all-reduce (sum) of the counts. Returns what combine_radiation returns."""
    import torch
    import torch.distributed as dist
    lv = torch.from_numpy(np.asarray(live, np.int32).copy())
    dist.all_reduce(lv, op=dist.ReduceOp.MAX, group=group)
    n = torch.tensor([len(hits)], dtype=torch.int64)
    world = dist.get_world_size(group)
    ns = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    m = max(int(x.item()) for x in ns)
    pad = torch.zeros((max(m, 1), 5), dtype=torch.int32)
    if len(hits):
        pad[:len(hits)] = torch.from_numpy(np.asarray(hits, np.int32).reshape(-1, 5))
    got = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(got, pad, group=group)
    allh = np.concatenate([g[:int(k.item())].numpy() for g, k in zip(got, ns)]).astype(np.int32)
    c = torch.from_numpy(np.asarray(counts[:3], np.int64).copy())
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    return lv.numpy().astype(np.uint8), allh.reshape(-1, 5), c.numpy().astype(np.int32)


def exchange_rows_dist(top_rows, bottom_rows, group=None):
    """Ghost-row exchange between neighbouring ranks of a torch.distributed group (one slab per
    rank, slab order = rank order, the torus wraps): sends this slab's first GHOST own rows
    (top_rows) to the rank above and its last GHOST own rows (bottom_rows) to the rank below;
    returns (north ghost rows from the rank above, south ghost rows from the rank below). Rows are
    float32 arrays of equal shape."""
    import torch
    import torch.distributed as dist
    r, n = dist.get_rank(group), dist.get_world_size(group)
    up, down = (r - 1) % n, (r + 1) % n
    top = torch.from_numpy(np.ascontiguousarray(top_rows))
    bot = torch.from_numpy(np.ascontiguousarray(bottom_rows))
    north, south = torch.empty_like(bot), torch.empty_like(top)
    if n == 1:
        return bot.numpy().copy(), top.numpy().copy()
    # tags tell the two messages apart when the rank above is also the rank below (two ranks):
    # 1 = my first own rows, the receiver's south ghost rows; 2 = my last own rows, its north
    reqs = [dist.isend(top, up, group=group, tag=1), dist.isend(bot, down, group=group, tag=2),
            dist.irecv(north, up, group=group, tag=2), dist.irecv(south, down, group=group, tag=1)]
    for q in reqs:
        q.wait()
    return north.numpy(), south.numpy()
