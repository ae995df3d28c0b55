"""Parity at the full benchmark size (4096 x 4096 torus, 1024 Zipf genomes, 54->64->10 CPPN
nets) in the launch configuration bench.py times: one GPU step compared with the FP64 oracle on
a seeded sample of cells the oracle computes one by one, and a full-size radiation event
compared bit-exactly."""
import numpy as np
import pytest

from oracle import coral_oracle as O
from oracle import philox as P
from paper_2406_09654_gb300 import coral, worlds
from parity import BF16_TAU, BF16_TOL, FP32_TAU, FP32_TOL, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cfg3():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()
    return worlds.make_world("cfg3", seed=0)


def sampled_errors(w, path, net_precision, tau, t=0):
    st, nets, gen, p = oracle_setup(w, net_precision=net_precision)
    cells = worlds.sample_cells(w, 3000, seed=11)
    o = O.step_cells(st, nets, t, p, cells)
    with coral.substrate_for_world(w, path) as sub:
        sub.set_step(t)
        sub.step(1)
        g = sub.read_channels()
    # cells whose own explore decision, a neighbour's, or their takeover compare was a near-tie
    mask = (o["margin_explore_nb"] < tau) | (o["tmargin"] < tau)
    errs = {}
    for name, ref in (("E", o["E"]), ("I", o["I"]), ("C0", o["C"][0]), ("C3", o["C"][3])):
        got = g[name].ravel()[cells].astype(np.float64)
        m = mask if name == "I" else np.zeros_like(mask)
        errs[name] = float(np.max(np.abs(got - ref)[~m]) / np.max(np.abs(ref)))
    bad_G = int(np.sum((g["G"].ravel()[cells] != o["G"]) & ~mask))
    bad_R = int(np.sum((g["R"].ravel()[cells] != o["R"]) & ~mask))
    return errs, bad_G, bad_R, int(mask.sum())


def test_fullsize_bf16_sampled_parity(cfg3):
    errs, bg, br, band = sampled_errors(cfg3, coral.BF16_GROUPED, "fp64", BF16_TAU)
    print("bf16 vs FP64 oracle at 4096^2:", errs, "band", band)
    assert bg == 0 and br == 0 and max(errs.values()) <= BF16_TOL
    errs, bg, br, band = sampled_errors(cfg3, coral.BF16_GROUPED, "bf16", 5e-3)
    print("bf16 vs BF16-operand oracle at 4096^2:", errs, "band", band)
    assert bg == 0 and br == 0 and max(errs.values()) <= 3e-3


def test_fullsize_fp32_sampled_parity(cfg3):
    errs, bg, br, band = sampled_errors(cfg3, coral.FP32_PERCELL, "fp64", FP32_TAU, t=150)
    print("fp32 vs FP64 oracle at 4096^2 (night step):", errs, "band", band)
    assert bg == 0 and br == 0 and max(errs.values()) <= FP32_TOL


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
