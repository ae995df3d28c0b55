"""GPU parity of the BF16 tensor-core (tcgen05) network path against the oracle.

Two references:
  * the oracle with BF16 network operands (x, W1 with b1, h, W2 rounded to bfloat16, exact
    sums) — the arithmetic the tensor-core path defines; what remains is FP32 accumulation
    order and the hardware tanh (relative error below 2^-10.9), so the tolerance is 3e-3 and
    the decision band 5e-3 (in units of the explore actuators);
  * the FP64 oracle (exact network) — the stated contract: per-channel normwise error <= 2e-2.
    Its integer outputs are compared outside two bands, each of which must hold on its own:
    the fixed band of reading R14 (every decision within 3e-2 of flipping), and the band the
    BF16 rounding itself accounts for (cells whose decision the FP64 and BF16-operand oracles
    take differently, plus the 5e-3 band of the BF16-operand oracle). The second is the narrow one and is gated
    at 5% of the cells; the first is reported with its breakdown (with CPPN nets the four
    explore actuators come from neighbouring output nodes of one smooth CPPN and are within
    3e-2 of each other for 8-19% of the cells, so that band holds a fifth of the grid).
"""
import numpy as np
import pytest

from oracle import coral_oracle as O
from paper_2406_09654_gb300 import coral, worlds
from parity import (BF16_TAU, BF16_TOL, band_breakdown, band_mask, compare_step, decision_split,
                    oracle_setup, round32, state_arrays)

pytestmark = pytest.mark.gpu

BF16_OP_TOL = 3e-3
BF16_OP_TAU = 5e-3
MAX_BAND = 0.05           # largest share of cells in the band a test accepts


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()
    assert coral.bf16_available(), "the tcgen05 path must be available on this GPU"


def forced(world, steps, tol, tau, t0=0, net_precision="fp64", max_band_frac=MAX_BAND, warm=0, fma_cutoff=0):
    """Oracle-forced steps: each step starts from the oracle's state on both sides (after `warm`
    oracle-only steps from t0). Returns the worst per-channel errors, the share of cells in the
    band (over all compared steps) and, for the FP64 contract, the fixed band's breakdown."""
    st, nets, gen, p = oracle_setup(world, net_precision=net_precision)
    if net_precision == "fp64":
        _, nets_b, _, p_b = oracle_setup(world, net_precision="bf16")
    sub = coral.substrate_for_world(world, coral.BF16_GROUPED)
    sub.set_fma_cutoff(fma_cutoff)
    worst, band, fixed = {}, 0, []
    try:
        st = round32(st)
        for t in range(t0, t0 + warm):
            st = round32(O.step(st, nets, t, p)[0])
        for t in range(t0 + warm, t0 + warm + steps):
            sub.load_state(*state_arrays(st))
            sub.set_step(t)
            sub.step(1)
            g = sub.read_channels()
            new, info = O.step(st, nets, t, p)
            if net_precision == "fp64":
                # fixed band of reading R14 at tau, then the band the BF16 rounding accounts for
                fixed.append(band_breakdown(st, info, tau, p.rotation))
                mask_r14 = band_mask(st, info, tau, p.rotation)
                _, bad_G, bad_R = compare_step(g, new, mask_r14, tol)
                assert bad_G == 0 and bad_R == 0, ("outside the fixed band", t, bad_G, bad_R)
                new_b, info_b = O.step(st, nets_b, t, p_b)
                split, outcome = decision_split(st, info["dir"], info_b["dir"], new.G, new_b.G, new.R, new_b.R)
                # the GPU is within BF16_OP_TAU of the BF16-operand oracle: outside that
                # oracle's band and where both oracles decide alike, it decides as they do
                mask = split | outcome | band_mask(st, info_b, BF16_OP_TAU, p.rotation)
            else:
                mask = band_mask(st, info, tau, p.rotation)
            band += int(mask.sum())
            errs, bad_G, bad_R = compare_step(g, new, mask, tol)
            assert bad_G == 0 and bad_R == 0, (t, bad_G, bad_R)
            for k, v in errs.items():
                worst[k] = max(worst.get(k, 0.0), v)
            assert max(errs.values()) <= tol, (t, errs)
            st = round32(new)
    finally:
        sub.close()
    frac = band / (steps * world.n_cells)
    assert frac <= max_band_frac, (frac, max_band_frac)
    return worst, frac, fixed


@pytest.mark.parametrize("W,H,n,hidden,layout", [(64, 64, 8, 0, "voronoi"), (96, 40, 6, 32, "voronoi"),
                                                 (37, 29, 5, 64, "voronoi"), (33, 7, 3, 16, "voronoi"),
                                                 (64, 64, 9, 48, "voronoi"), (40, 24, 50, 64, "random"),
                                                 # widths that are not a multiple of 4 (padded rows)
                                                 (130, 70, 10, 64, "voronoi"), (141, 43, 8, 32, "random"),
                                                 (103, 37, 6, 16, "voronoi")])
def test_bf16_matches_bf16_operand_oracle(W, H, n, hidden, layout):
    w = worlds.make_world(width=W, height=H, n_genomes=n, hidden=hidden, layout=layout,
                          net="cppn" if hidden else "direct", seed=W + H + hidden, random_rotation=True)
    # 50 genomes scattered cell by cell: several of their CPPNs give near-equal explore
    # actuators (4% of the cells within 5e-3), and each such explorer sets aside its
    # candidate targets too, so this adversarial layout's band is about 12% of the grid
    limit = 0.15 if n == 50 else MAX_BAND
    worst, frac, _ = forced(w, 3, BF16_OP_TOL, BF16_OP_TAU, t0=98, net_precision="bf16", max_band_frac=limit)
    print(W, H, hidden, layout, "worst", worst, "band fraction", round(frac, 4))


@pytest.mark.parametrize("hidden", [0, 32, 64])
def test_bf16_within_stated_tolerance_of_fp64_oracle(hidden):
    w = worlds.make_world(width=128, height=96, n_genomes=12, hidden=hidden,
                          net="cppn" if hidden else "direct", seed=5 + hidden)
    worst, frac, fixed = forced(w, 3, BF16_TOL, BF16_TAU, warm=1)
    print("hidden", hidden, "worst per-channel error vs FP64 oracle", worst, "band fraction", round(frac, 4),
          "fixed 3e-2 band", {k: round(float(np.mean([f[k] for f in fixed])), 4) for k in fixed[0]})


@pytest.mark.parametrize("hidden", [32, 64])
def test_bf16_first_step_from_raw_initial_state(hidden):
    """Step 0 starts from the raw initial state: the communication channels are N(0, 0.1) noise
    and every CPPN net sees inputs near its bias point, so the explore actuators of a genome are
    nearly equal over its whole blob; BF16 rounding then moves 0.3-6% of the decisions, and the
    band is 11-15% of the grid (it falls below 1% from step 1 on)."""
    w = worlds.make_world(width=128, height=96, n_genomes=12, hidden=hidden, net="cppn", seed=5 + hidden)
    worst, frac, _ = forced(w, 1, BF16_TOL, BF16_TAU, max_band_frac=0.2)
    print("hidden", hidden, "step 0: worst", worst, "band fraction", round(frac, 4))


def test_bf16_minimum_torus_and_single_genome():
    w = worlds.make_world(width=3, height=3, n_genomes=1, hidden=64, net="cppn", seed=1)
    # nine cells: one near-tie is already 11% of the grid
    forced(w, 2, BF16_OP_TOL, BF16_OP_TAU, net_precision="bf16", max_band_frac=1.0)


def test_bf16_radiation_and_determinism():
    w = worlds.make_world(width=160, height=96, n_genomes=20, hidden=64, net="cppn", seed=4,
                          radiation_every=3, p_mut=2e-3, p_merge=2e-3, capacity=600)
    outs, stats = [], []
    for _ in range(2):
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as sub:
            sub.step(10)
            outs.append(sub.read_channels())
            s = sub.read_stats(8, 1)[0]
            assert s["n_born"] > 0 and s["n_live"] > 20
            stats.append(sub.read_stats(0, 10))
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    # tiles are shared out dynamically among the CTAs; the totals stay bit-identical
    assert stats[0] == stats[1]


OPERAND_WORLDS = [(64, 64, 8, 0, "voronoi"), (96, 40, 6, 32, "voronoi"), (37, 29, 5, 64, "voronoi"),
                  (33, 7, 3, 16, "voronoi"), (64, 64, 9, 48, "voronoi"), (40, 24, 50, 64, "random"),
                  (130, 70, 10, 64, "voronoi"), (141, 43, 8, 32, "random"), (103, 37, 6, 16, "voronoi")]


@pytest.mark.parametrize("W,H,n,hidden,layout", OPERAND_WORLDS)
def test_fma_small_genome_path_matches_bf16_operand_oracle(W, H, n, hidden, layout):
    """The worlds of the test above with cutoff 128: every later genome round of a tile runs on
    the warp-level FMA path (a tile's first round stays on the tensor cores), with the
    tensor-core path's operands (BF16 inputs, weights and hidden values, FP32 sums); the same
    tolerance and band gates."""
    w = worlds.make_world(width=W, height=H, n_genomes=n, hidden=hidden, layout=layout,
                          net="cppn" if hidden else "direct", seed=W + H + hidden, random_rotation=True)
    limit = 0.15 if n == 50 else MAX_BAND
    worst, frac, _ = forced(w, 3, BF16_OP_TOL, BF16_OP_TAU, t0=98, net_precision="bf16", max_band_frac=limit,
                            fma_cutoff=128)
    print(W, H, hidden, layout, "worst", worst, "band fraction", round(frac, 4))


def test_fma_cutoff_is_validated():
    w = worlds.make_world(width=16, height=16, n_genomes=2, hidden=16, net="cppn", seed=1)
    with coral.substrate_for_world(w, coral.BF16_GROUPED) as sub:
        for bad in (-1, 129):
            with pytest.raises(coral.CoralError) as e:
                sub.set_fma_cutoff(bad)
            assert e.value.code == coral.E_INVALID
        sub.set_fma_cutoff(0)
        sub.set_fma_cutoff(128)


def test_fma_path_is_taken_and_close_to_tensor_core_path():
    """One step of a cell-by-cell random world with the small-genome path off and on: the FMA
    sums run in another order than the tensor core's, so some outputs differ in their last
    bits (the path did run), all within the BF16-operand tolerance."""
    w = worlds.make_world(width=40, height=24, n_genomes=50, hidden=64, layout="random", net="cppn", seed=128)
    outs = []
    for cut in (0, 128):
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as sub:
            sub.set_step(98)
            sub.set_fma_cutoff(cut)
            sub.step(1)
            outs.append(sub.read_channels())
    a, b = outs
    assert any(not np.array_equal(a[k], b[k]) for k in ("C0", "C1", "C2", "C3"))
    for k in ("C0", "C1", "C2", "C3"):
        assert np.max(np.abs(a[k] - b[k])) <= BF16_OP_TOL * max(1.0, float(np.max(np.abs(a[k]))))
