"""Seeded synthetic worlds: the inputs that both the CUDA library and the CPU oracle step.

This module generates inputs only. It holds none of the method's arithmetic: no sensing,
no network, no physics, no radiation. Everything it draws comes from numpy's seeded
generator, and every array it returns is float32 / int32 / uint8, so the CUDA path and the
FP64 oracle see exactly the same values.

Workload recipes (the paper prints no workload; these stand in for its qualitative
1024x1024 / 512-organism runs, Section "Experiment"):

* ``tiny``-style worlds for parity tests: any side, any genome count, Voronoi layout.
* ``cfg1`` 64x64 torus, 8 genomes in Voronoi blobs, direct 54->10 nets, weights N(0, 0.3).
* ``cfg2`` 1024x1024 torus, 64 Voronoi genomes, CPPN genes N(0, 1), 54->32->10 nets,
  mutation p=1e-4 per cell every 50 steps.
* ``cfg3`` 4096x4096 torus, 1024 genomes with Zipf(1.2) cell counts laid out as contiguous
  segments of a Hilbert curve, 54->64->10 CPPN nets, merge and mutation every 20 steps.

Channel initialisation (all worlds): energy U[0, 1], infrastructure U[0, 0.5], four
communication channels N(0, 0.1), rotation 0 unless ``random_rotation`` is asked for.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

N_SENSORS = 6          # energy, infrastructure, com0..com3
N_INPUTS = 54          # 9 kernel offsets x 6 sensor channels
N_OUTPUTS = 10         # com0..com3, invest, liquidate, explore0..explore3
N_GENES = 18           # 3 hidden CPPN nodes x 5 inputs + 3 hidden->output weights

# Physics constants shared by every preset (each is a reading of a paper passage the
# paper leaves without numbers; the readings are listed with the oracle).
DEFAULT_PHYSICS = dict(
    k_inv=0.1, k_liq=0.1, k_exp=0.5, k_flow=0.2,
    e_day=0.005, e_night=0.005, day_period=200,
    rotation=1, sigma_mut=0.05,
)

PRESETS = {
    "cfg1": dict(width=64, height=64, n_genomes=8, layout="voronoi", hidden=0,
                 net="direct", radiation_every=0, p_mut=0.0, p_merge=0.0, steps=100,
                 capacity=8),
    "cfg2": dict(width=1024, height=1024, n_genomes=64, layout="voronoi", hidden=32,
                 net="cppn", radiation_every=50, p_mut=1e-4, p_merge=0.0, steps=1000,
                 capacity=8192),
    "cfg3": dict(width=4096, height=4096, n_genomes=1024, layout="hilbert_zipf",
                 zipf_s=1.2, hidden=64, net="cppn", radiation_every=20, p_mut=1e-4,
                 p_merge=1e-4, steps=500, capacity=65536),
}


def net_floats(hidden: int) -> int:
    """Floats in one dense net: W1[H][54], b1[H], W2[10][H], b2[10]; H=0 is W[10][54], b[10]."""
    if hidden == 0:
        return N_OUTPUTS * N_INPUTS + N_OUTPUTS
    return hidden * N_INPUTS + hidden + N_OUTPUTS * hidden + N_OUTPUTS


@dataclass
class World:
    width: int
    height: int
    E: np.ndarray            # [H][W] float32
    I: np.ndarray            # [H][W] float32
    C: np.ndarray            # [4][H][W] float32
    G: np.ndarray            # [H][W] int32, genome slot of each cell
    R: np.ndarray            # [H][W] uint8 in {0,1,2,3}
    n_genomes: int
    hidden: int
    capacity: int
    genes: np.ndarray | None = None   # [n][18] float32 CPPN genes (net == "cppn")
    dense: np.ndarray | None = None   # [n][net_floats] float32 direct nets (net == "direct")
    physics: dict = field(default_factory=dict)
    seed: int = 0
    steps: int = 1
    name: str = ""

    @property
    def n_cells(self) -> int:
        return self.width * self.height


def _torus_voronoi(width, height, n, rng):
    """Genome of each cell = nearest of n distinct seed points (integer torus distance^2,
    ties to the lower seed index)."""
    flat = rng.choice(width * height, size=n, replace=False)
    sx, sy = flat % width, flat // width
    G = np.empty((height, width), np.int32)
    xs = np.arange(width)
    for y in range(height):
        dy = np.abs(y - sy)
        dy = np.minimum(dy, height - dy)[:, None]                 # [n][1]
        dx = np.abs(xs[None, :] - sx[:, None])
        dx = np.minimum(dx, width - dx)                           # [n][W]
        d2 = dx * dx + dy * dy
        G[y] = np.argmin(d2, axis=0)                              # first minimum = lower seed
    return G


def _torus_voronoi_tree(width, height, n, rng):
    """The same layout as _torus_voronoi (same seed draw, integer torus distance^2, ties to the
    lower seed index), found with a periodic k-d tree: the two nearest seeds of each cell, and
    a scan of every seed for the few cells where those two are at the same distance."""
    from scipy.spatial import cKDTree
    flat = rng.choice(width * height, size=n, replace=False)
    sx, sy = flat % width, flat // width
    G = np.zeros(width * height, np.int32)
    if n == 1:
        return G.reshape(height, width)
    tree = cKDTree(np.stack([sx, sy], 1).astype(np.float64), boxsize=[width, height])
    chunk = 1 << 20
    for c0 in range(0, width * height, chunk):
        c = np.arange(c0, min(width * height, c0 + chunk))
        x, y = c % width, c // width
        _, idx = tree.query(np.stack([x, y], 1).astype(np.float64), k=2, workers=-1)
        dx = np.abs(x[:, None] - sx[idx])
        dx = np.minimum(dx, width - dx)
        dy = np.abs(y[:, None] - sy[idx])
        dy = np.minimum(dy, height - dy)
        d2 = dx * dx + dy * dy
        g = idx[:, 0].copy()
        for j in np.nonzero(d2[:, 1] == d2[:, 0])[0]:
            ex = np.abs(x[j] - sx)
            ex = np.minimum(ex, width - ex)
            ey = np.abs(y[j] - sy)
            ey = np.minimum(ey, height - ey)
            g[j] = np.argmin(ex * ex + ey * ey)
        G[c] = g
    return G.reshape(height, width)


def zipf_counts(total: int, n: int, s: float) -> np.ndarray:
    """Cell counts n_k proportional to k^-s (k = 1..n), rounded by largest remainder so that
    they sum to ``total``; remainder ties go to the lower rank."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    share = total * w / w.sum()
    base = np.floor(share).astype(np.int64)
    rest = total - int(base.sum())
    frac = share - base
    order = np.lexsort((np.arange(n), -frac))                    # largest fraction first
    base[order[:rest]] += 1
    return base


def hilbert_d2xy(order: int, d: np.ndarray):
    """Textbook Hilbert-curve index -> (x, y) on a 2^order square (vectorised): at level s
    (1, 2, 4, ...) take the next two bits (rx, ry) of d; when ry = 0 reflect (if rx = 1) and
    transpose the coordinates gathered so far; then add s*rx, s*ry."""
    t = np.asarray(d, np.int64).copy()
    x = np.zeros(t.shape, np.int64)
    y = np.zeros(t.shape, np.int64)
    for level in range(order):
        s = 1 << level
        rx = (t >> 1) & 1
        ry = (t ^ rx) & 1
        swap = ry == 0
        flip = swap & (rx == 1)
        xf = np.where(flip, s - 1 - x, x)
        yf = np.where(flip, s - 1 - y, y)
        x = np.where(swap, yf, xf) + s * rx
        y = np.where(swap, xf, yf) + s * ry
        t >>= 2
    return x, y


def hilbert_curve(order: int):
    """(x, y) of every index 0 .. 4^order - 1 of the Hilbert curve, computed as the low
    half-order curve (a table) carried through the high levels, whose reflections and
    transpositions act on the low coordinates as one affine map per high index."""
    lo = order // 2
    hi_levels = order - lo
    ux, uy = hilbert_d2xy(lo, np.arange(1 << (2 * lo)))          # low table
    hi = np.arange(1 << (2 * hi_levels), dtype=np.int64)
    # x = fx * (swapped ? uy : ux) + ox,  y = fy * (swapped ? ux : uy) + oy
    swapped = np.zeros(hi.shape, bool)
    fx = np.ones(hi.shape, np.int64); fy = np.ones(hi.shape, np.int64)
    ox = np.zeros(hi.shape, np.int64); oy = np.zeros(hi.shape, np.int64)
    t = hi.copy()
    for level in range(lo, order):
        s = 1 << level
        rx = (t >> 1) & 1
        ry = (t ^ rx) & 1
        swap = ry == 0
        flip = swap & (rx == 1)
        fx = np.where(flip, -fx, fx); ox = np.where(flip, s - 1 - ox, ox)
        fy = np.where(flip, -fy, fy); oy = np.where(flip, s - 1 - oy, oy)
        swapped = swapped ^ swap
        fx, fy = np.where(swap, fy, fx), np.where(swap, fx, fy)
        ox, oy = np.where(swap, oy, ox), np.where(swap, ox, oy)
        ox = ox + s * rx
        oy = oy + s * ry
        t >>= 2
    sw = swapped[:, None]
    x = fx[:, None] * np.where(sw, uy[None, :], ux[None, :]) + ox[:, None]
    y = fy[:, None] * np.where(sw, ux[None, :], uy[None, :]) + oy[:, None]
    return x.ravel(), y.ravel()


def _hilbert_zipf(width, height, n, s):
    """Genome k owns the k-th contiguous run of a Hilbert curve, run lengths Zipf(s)."""
    order = max(1, int(np.ceil(np.log2(max(width, height)))))
    side = 1 << order
    x, y = hilbert_curve(order)
    keep = (x < width) & (y < height)
    x, y = x[keep], y[keep]
    counts = zipf_counts(width * height, n, s)
    owner = np.repeat(np.arange(n, dtype=np.int32), counts)
    G = np.empty((height, width), np.int32)
    G[y, x] = owner
    return G


def make_world(preset: str | None = None, seed: int = 0, **overrides) -> World:
    """Build a seeded world. ``preset`` is one of PRESETS (or None for a custom world given
    entirely by keyword arguments: width, height, n_genomes, layout, hidden, net, ...)."""
    cfg = dict(PRESETS[preset]) if preset else dict(
        width=16, height=16, n_genomes=4, layout="voronoi", hidden=0, net="direct",
        radiation_every=0, p_mut=0.0, p_merge=0.0, steps=1, capacity=None)
    cfg.update(overrides)
    width, height, n = int(cfg["width"]), int(cfg["height"]), int(cfg["n_genomes"])
    hidden = int(cfg["hidden"])
    if width < 1 or height < 1 or n < 1 or n > width * height:
        raise ValueError("bad world size")
    rng = np.random.default_rng(np.random.SeedSequence([seed, width, height, n, hidden]))

    E = rng.uniform(0.0, 1.0, (height, width)).astype(np.float32)
    I = rng.uniform(0.0, 0.5, (height, width)).astype(np.float32)
    C = rng.normal(0.0, 0.1, (4, height, width)).astype(np.float32)
    if cfg.get("random_rotation"):
        R = rng.integers(0, 4, (height, width)).astype(np.uint8)
    else:
        R = np.zeros((height, width), np.uint8)

    layout = cfg.get("layout", "voronoi")
    if layout == "voronoi":
        # the same layout; the k-d tree search for large grids (equal to the plain one, tested)
        G = (_torus_voronoi_tree if width * height * n > 10**8 else _torus_voronoi)(width, height, n, rng)
    elif layout == "hilbert_zipf":
        G = _hilbert_zipf(width, height, n, float(cfg.get("zipf_s", 1.2)))
    elif layout == "random":
        G = rng.integers(0, n, (height, width)).astype(np.int32)
    else:
        raise ValueError(f"unknown layout {layout}")

    genes = dense = None
    if cfg.get("net", "direct") == "cppn":
        genes = rng.normal(0.0, 1.0, (n, N_GENES)).astype(np.float32)
    else:
        std = float(cfg.get("weight_std", 0.3))
        dense = rng.normal(0.0, std, (n, net_floats(hidden))).astype(np.float32)

    capacity = cfg.get("capacity") or n
    physics = dict(DEFAULT_PHYSICS)
    for k in list(physics) + ["radiation_every", "p_mut", "p_merge"]:
        if k in cfg:
            physics[k] = cfg[k]
    physics.setdefault("radiation_every", 0)
    physics.setdefault("p_mut", 0.0)
    physics.setdefault("p_merge", 0.0)
    return World(width, height, E, I, C, G.astype(np.int32), R, n, hidden, int(capacity),
                 genes=genes, dense=dense, physics=physics, seed=seed,
                 steps=int(cfg.get("steps", 1)), name=preset or "custom")


def make_batch_worlds(n_worlds: int = 256, side_min: int = 128, side_max: int = 2048,
                      genomes=(16, 256), hidden: int = 32, seed: int = 0):
    """Independent square worlds for batched stepping: side log-uniform in [side_min, side_max],
    genome count uniform in the given range, CPPN nets 54->hidden->10, no radiation. Channels
    are drawn in float32 (same distributions as make_world); genomes sit in per-cell Voronoi
    blobs."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, n_worlds, side_min, side_max, 4]))
    sides = np.rint(np.exp(rng.uniform(np.log(side_min), np.log(side_max), n_worlds))).astype(int)
    counts = rng.integers(genomes[0], genomes[1] + 1, n_worlds)
    return [make_square_world(int(sides[k]), int(counts[k]), hidden, seed * 100003 + k, f"batch{k}")
            for k in range(n_worlds)]


def make_square_world(side: int, n_genomes: int, hidden: int = 32, seed: int = 0, name: str = "") -> World:
    """One side x side world with n_genomes CPPN genomes in Voronoi blobs (per cell, as
    make_world), no radiation; channels drawn in float32 with make_world's distributions."""
    s, n = int(side), int(n_genomes)
    r = np.random.default_rng(np.random.SeedSequence([seed, s, n, hidden, 6]))
    E = r.random((s, s), dtype=np.float32)
    I = (0.5 * r.random((s, s), dtype=np.float32)).astype(np.float32)
    C = (0.1 * r.standard_normal((4, s, s), dtype=np.float32)).astype(np.float32)
    G = _torus_voronoi_tree(s, s, min(n, s * s), r)
    genes = r.normal(0.0, 1.0, (n, N_GENES)).astype(np.float32)
    phys = dict(DEFAULT_PHYSICS, radiation_every=0, p_mut=0.0, p_merge=0.0)
    return World(s, s, E, I, C, G, np.zeros((s, s), np.uint8), n, hidden, n, genes=genes,
                 physics=phys, seed=seed, steps=1, name=name or f"square{s}")


class LazySquareWorld:
    """A serving request's world, described by its size up front (for admission) and built by
    make_square_world on first use (materialize), so that a long request list holds no state."""

    def __init__(self, side: int, n_genomes: int, hidden: int, seed: int, name: str):
        self.width = self.height = int(side)
        self.n_genomes = self.capacity = int(n_genomes)
        self.hidden, self.seed, self.name = int(hidden), int(seed), name

    @property
    def n_cells(self) -> int:
        return self.width * self.height

    def materialize(self) -> World:
        return make_square_world(self.width, self.n_genomes, self.hidden, seed=self.seed, name=self.name)


def request_world_factory(side_range=(128, 4096), genomes_range=(8, 1024), hidden: int = 32, lazy: bool = False):
    """make_world(rng, k) for serving requests: side log-uniform in side_range, genome count
    uniform in genomes_range (capped by the cell count); lazy: a LazySquareWorld."""
    def make(rng, k):
        side = int(np.rint(np.exp(rng.uniform(np.log(side_range[0]), np.log(side_range[1])))))
        n = min(int(rng.integers(genomes_range[0], genomes_range[1] + 1)), side * side)
        seed = int(rng.integers(1 << 30))
        if lazy:
            return LazySquareWorld(side, n, hidden, seed, f"req{k}")
        return make_square_world(side, n, hidden, seed=seed, name=f"req{k}")
    return make


def sample_cells(world: World, n: int, seed: int = 1) -> np.ndarray:
    """Seeded sample of distinct flat cell indices (for per-cell checks at full size)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, world.n_cells, 7]))
    return np.sort(rng.choice(world.n_cells, size=min(n, world.n_cells), replace=False))
