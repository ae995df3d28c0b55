"""Parity at the full benchmark size (4096 x 4096 torus, 1024 Zipf genomes, 54->64->10 CPPN
nets) in the launch configuration bench.py times: one GPU step compared with the oracle on a
stratified sample of cells the oracle computes one by one (the tiles with several genomes, the
torus seams, the edges of the CTAs' tile runs and pool chunks, and a uniform remainder), every
float plane, and a full-size radiation event compared bit-exactly."""
import numpy as np
import pytest

from oracle import coral_oracle as O
from oracle import philox as P
from paper_2406_09654_gb300 import coral, worlds
from parity import BF16_TAU, BF16_TOL, FP32_TAU, FP32_TOL, band_mask_cells, decision_split, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cfg3():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()
    return worlds.make_world("cfg3", seed=0)


# The BF16 kernel's work split (its tile shape and tile pool): 32 x 4-cell tiles in row-major
# tile order; each CTA first walks a contiguous run of n_tiles // 2 // ctas tiles, then claims
# 4-tile chunks of the rest. Halos that wrap around the torus, or whose 40-wide copy box would
# leave the grid, come by cp.async instead of TMA.
TILE_W, TILE_H, CHUNK = 32, 4, 4


def stratified_cells(w, ctas, seed=11):
    """Cells the sampled parity checks: every cell of every tile holding 3 or more genomes and of
    up to 48 tiles holding 2 (tiles with several genomes run several tensor-core rounds),
    1,500 cells of the tiles whose halo is copied by cp.async (torus seams), 16 cells of the
    first and last tile of 24 CTA runs and 24 pool chunks, and 3,000 cells drawn uniformly."""
    rng = np.random.default_rng(seed)
    W, H = w.width, w.height
    tx, ty = W // TILE_W, H // TILE_H
    G = w.G.reshape(ty, TILE_H, tx, TILE_W).transpose(0, 2, 1, 3).reshape(ty * tx, TILE_H * TILE_W)
    Gs = np.sort(G, axis=1)
    n_gen = 1 + np.sum(Gs[:, 1:] != Gs[:, :-1], axis=1)
    parts = []

    def tile_cells(t, k=None):
        y0, x0 = (t // tx) * TILE_H, (t % tx) * TILE_W
        c = ((y0 + np.arange(TILE_H))[:, None] * W + x0 + np.arange(TILE_W)[None, :]).ravel()
        return c if k is None else rng.choice(c, k, replace=False)

    multi = np.nonzero(n_gen >= 3)[0]
    two = np.nonzero(n_gen == 2)[0]
    for t in np.concatenate([multi, rng.choice(two, min(48, two.size), replace=False)]):
        parts.append(tile_cells(int(t)))
    x0 = (np.arange(tx * ty) % tx) * TILE_W
    y0 = (np.arange(tx * ty) // tx) * TILE_H
    seam = np.nonzero((x0 < 4) | (x0 + TILE_W + 4 > W) | (y0 == 0) | (y0 + TILE_H + 1 > H))[0]
    parts.append(np.concatenate([tile_cells(t) for t in seam]))
    parts[-1] = rng.choice(parts[-1], 1500, replace=False)
    per = tx * ty // 2 // ctas
    pool0 = per * ctas
    runs = rng.choice(ctas, 24, replace=False)
    chunks = rng.choice((tx * ty - pool0) // CHUNK, 24, replace=False)
    for t in np.concatenate([runs * per, runs * per + per - 1, pool0 + CHUNK * chunks, pool0 + CHUNK * chunks + CHUNK - 1]):
        parts.append(tile_cells(int(t), 16))
    parts.append(worlds.sample_cells(w, 3000, seed=seed))
    return np.unique(np.concatenate(parts)), (int(multi.size), int(two.size))


PLANES = ("E", "I", "C0", "C1", "C2", "C3")


def plane_errors(g, o, cells, mask):
    """[R16] per-plane normwise errors at the sampled cells; I outside the decision band."""
    errs = {}
    for name in PLANES:
        ref = o["E"] if name == "E" else o["I"] if name == "I" else o["C"][int(name[1])]
        got = g[name].ravel()[cells].astype(np.float64)
        m = mask if name == "I" else np.zeros_like(mask)
        errs[name] = float(np.max(np.abs(got - ref)[~m]) / np.max(np.abs(ref)))
    return errs


def gpu_step(w, path, t, before=0):
    """One GPU step t of world w after `before` GPU steps from t - before; returns the state the
    step started from (as an oracle state), its result and the pass-1 CTA count."""
    with coral.substrate_for_world(w, path) as sub:
        sub.set_step(t - before)
        sub.step(before)
        s0 = sub.read_channels()
        sub.step(1)
        g = sub.read_channels()
        ctas = sub.launch_config()["grid_pass1"]
    st = O.State(w.width, w.height, s0["E"].ravel().astype(np.float64), s0["I"].ravel().astype(np.float64),
                 s0["C"].reshape(4, -1).astype(np.float64), s0["G"].ravel().astype(np.int64),
                 s0["R"].ravel().astype(np.int64))
    return st, g, ctas


@pytest.mark.parametrize("t,before,max_band", [(6, 6, 0.05), (0, 0, 0.10)])
def test_fullsize_bf16_sampled_parity(cfg3, t, before, max_band):
    """Step 6 from the state the GPU reached after steps 0..5 (both sides start from it), and
    step 0 from the raw initial state, whose communication channels are N(0, 0.1) noise: there
    every CPPN net sees inputs near its bias point and a genome's explore actuators are nearly
    equal over its blob, so more decisions sit in the band."""
    w = cfg3
    st, g, ctas = gpu_step(w, coral.BF16_GROUPED, t, before)
    cells, n_multi = stratified_cells(w, ctas)
    _, nets, gen, p = oracle_setup(w)
    _, nets_b, _, p_b = oracle_setup(w, net_precision="bf16")
    o = O.step_cells(st, nets, t, p, cells)
    ob = O.step_cells(st, nets_b, t, p_b, cells)
    gG, gR = g["G"].ravel()[cells], g["R"].ravel()[cells]
    # against the BF16-operand oracle, outside its 5e-3 band
    mb = band_mask_cells(st, ob, cells, 5e-3, p.rotation)
    errs_b = plane_errors(g, ob, cells, mb)
    assert np.sum((gG != ob["G"]) & ~mb) == 0 and np.sum((gR != ob["R"]) & ~mb) == 0
    assert max(errs_b.values()) <= 3e-3, errs_b
    # against the FP64 oracle: outside the fixed 3e-2 band, and outside the band the BF16
    # rounding accounts for (decisions the two oracles take differently, plus mb)
    m_fixed = band_mask_cells(st, o, cells, BF16_TAU, p.rotation)
    split, outcome = decision_split(st, o["pass1"]["dir"], ob["pass1"]["dir"], o["G"], ob["G"], o["R"], ob["R"])
    m = split[cells] | outcome | mb
    errs = plane_errors(g, o, cells, m)
    for mask in (m_fixed, m):
        assert np.sum((gG != o["G"]) & ~mask) == 0 and np.sum((gR != o["R"]) & ~mask) == 0
    assert max(errs.values()) <= BF16_TOL, errs
    print(f"4096^2 BF16 step {t}: {cells.size} cells (tiles with >= 3 / 2 genomes in the world: {n_multi}); "
          f"vs BF16-operand oracle {errs_b}, band {mb.mean():.4f}; vs FP64 oracle {errs}, band {m.mean():.4f}, "
          f"fixed 3e-2 band {m_fixed.mean():.4f}")
    assert mb.mean() <= max_band and m.mean() <= max_band


def test_fullsize_fp32_sampled_parity(cfg3):
    w = cfg3
    st, g, ctas = gpu_step(w, coral.FP32_PERCELL, 150)
    cells, _ = stratified_cells(w, ctas)
    _, nets, gen, p = oracle_setup(w)
    o = O.step_cells(st, nets, 150, p, cells)
    mask = band_mask_cells(st, o, cells, FP32_TAU, p.rotation)
    errs = plane_errors(g, o, cells, mask)
    bad_G = int(np.sum((g["G"].ravel()[cells] != o["G"]) & ~mask))
    bad_R = int(np.sum((g["R"].ravel()[cells] != o["R"]) & ~mask))
    print("fp32 vs FP64 oracle at 4096^2 (night step):", cells.size, "cells", errs, "band", mask.mean())
    assert bad_G == 0 and bad_R == 0 and max(errs.values()) <= FP32_TOL
    assert mask.mean() <= 0.05


def test_fullsize_radiation_event_bit_exact(cfg3):
    """Exploration off keeps G at the initial layout through the physics, so the radiation
    event after step 0 (every step here) sees the same G on both sides at full size."""
    w = cfg3
    w.physics = dict(w.physics, k_exp=0.0, radiation_every=1)
    try:
        p = O.Params.from_world(w)
        st = O.State.from_world(w)
        gen = O.Genomes.from_genes(w.genes, w.capacity)
        new, gen2, slots, ev = O.radiation(st, gen, 0, p)
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as sub:
            sub.step(1)
            G = sub.read_channels(coral.CH_G)["G"].ravel()
            genes, parent = sub.read_genomes()
            s = sub.read_stats(0, 1)[0]
        assert s["n_mut"] == ev["n_mut"] and s["n_merge"] == ev["n_merge"] and s["n_born"] == ev["n_assigned"]
        assert ev["n_hits"] > 1000
        assert np.array_equal(G, new.G)
        assert np.array_equal(parent[:w.capacity], gen2.parent)
        for k in slots[:200]:
            assert np.allclose(genes[k], gen2.genes[k], rtol=0, atol=2e-6)
    finally:
        w.physics = dict(w.physics, k_exp=0.5, radiation_every=20)


def test_fullsize_bucketing_sort(cfg3):
    """The bucketing sort of the full-size world's GenomeIndex (the sort bench.py times). A
    permutation whose keys are non-decreasing and whose cell ids increase within each key is
    the stable sort, so these properties check every output; counts against a plain bincount."""
    G = cfg3.G.ravel().astype(np.int64)
    with coral.Substrate(coral.params_from_world(cfg3), cfg3.width, cfg3.height, cfg3.capacity) as sub:
        sub.load_state(cfg3.E, cfg3.I, cfg3.C, cfg3.G, cfg3.R)
        counts, perm = sub.read_perm()
    n = G.size
    assert np.array_equal(np.sort(perm), np.arange(n))
    k = G[perm]
    assert np.all(np.diff(k) >= 0)
    same = k[1:] == k[:-1]
    assert np.all(np.diff(perm.astype(np.int64))[same] > 0)
    assert np.array_equal(counts, np.bincount(G, minlength=cfg3.capacity))
