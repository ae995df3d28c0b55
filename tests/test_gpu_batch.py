"""Batched stepping of many worlds of different sizes (one launch per pass, CUDA graph
replays): every world's result must be bit-identical to stepping it alone, and the autotuner
must leave the worlds' states untouched."""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def mixed_worlds(n=7, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        W = int(rng.integers(3, 300))
        H = int(rng.integers(3, 200))
        g = int(rng.integers(1, min(40, W * H)))
        out.append(worlds.make_world(width=W, height=H, n_genomes=g, hidden=32, net="cppn", seed=100 + k,
                                     random_rotation=bool(k % 2)))
    out.append(worlds.make_world(width=256, height=128, n_genomes=30, hidden=32, net="cppn", seed=7))
    return out


def test_batched_equals_alone_bit_exact():
    ws = mixed_worlds()
    alone = []
    for w in ws:
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as s:
            s.step(5)
            alone.append((s.read_channels(), s.read_stats(4, 1)[0]))
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        with coral.Batch(subs) as b:
            b.step(2)
            b.step(3)
        for (ref, st), s in zip(alone, subs):
            got = s.read_channels()
            for k in ref:
                assert np.array_equal(ref[k], got[k]), k
            bs = s.read_stats(4, 1)[0]
            assert bs["step"] == 4 and bs["n_explore"] == st["n_explore"]
            assert bs["sum_E"] == pytest.approx(st["sum_E"], rel=1e-12)
            # the C' totals are exact sums, whatever the split of tiles among CTAs
            assert bs["sum_C"] == st["sum_C"]
            assert s.get_step() == 5
    finally:
        for s in subs:
            s.close()


def test_batch_tuner_restores_state_and_mixes_with_single_steps():
    ws = mixed_worlds(5, seed=3)
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        with coral.Batch(subs) as b:
            choice = b.tune(trial_steps=2)
            assert choice["pass1_ctas_per_sm"] in (3, 4, 5, 6) and choice["pass2_ctas_per_sm"] in (1, 2, 3)
            assert choice["fma_cutoff"] in (0, 1, 2, 4, 8)
            b.set_fma_cutoff(0)                      # the steps below: the tensor-core path only
            subs[0].step(1)                          # one world steps alone in between
            b.step(2)
        for w, s, extra in zip(ws, subs, [1, 0, 0, 0, 0]):
            with coral.substrate_for_world(w, coral.BF16_GROUPED) as ref:
                ref.step(2 + extra)
                a, g = ref.read_channels(), s.read_channels()
                for k in a:
                    assert np.array_equal(a[k], g[k]), k
    finally:
        for s in subs:
            s.close()


def test_batch_rejects_mixed_configurations():
    a = worlds.make_world(width=16, height=16, n_genomes=2, hidden=32, net="cppn", seed=1)
    c = worlds.make_world(width=16, height=16, n_genomes=2, hidden=16, net="cppn", seed=1)
    s1 = coral.substrate_for_world(a, coral.BF16_GROUPED)
    s2 = coral.substrate_for_world(c, coral.BF16_GROUPED)
    s3 = coral.substrate_for_world(a, coral.FP32_PERCELL)
    try:
        for pair in ([s1, s2], [s1, s3]):
            with pytest.raises(coral.CoralError) as e:
                coral.Batch(pair)
            assert e.value.code == coral.E_INVALID
    finally:
        for s in (s1, s2, s3):
            s.close()


def test_batched_worlds_match_oracle():
    """Two worlds inside a batch of five, one oracle-forced step: both sides start from the
    state the oracle reached after one step and step t = 1 (the other worlds run their own
    states alongside)."""
    from oracle import coral_oracle as O
    from parity import check_bf16_step, oracle_setup, round32, state_arrays
    ws = mixed_worlds(3, seed=9) + [worlds.make_world(width=96, height=64, n_genomes=7, hidden=32, net="cppn", seed=21),
                                    worlds.make_world(width=130, height=70, n_genomes=9, hidden=32, net="cppn", seed=22,
                                                      random_rotation=True)]
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        starts = []
        for w, s in zip(ws[3:], subs[3:]):
            st, nets, gen, p = oracle_setup(w)
            st = round32(O.step(round32(st), nets, 0, p)[0])
            s.load_state(*state_arrays(st))
            starts.append(st)
        for s in subs:
            s.set_step(1)
        with coral.Batch(subs) as b:
            b.step(1)
        for w, s, st in zip(ws[3:], subs[3:], starts):
            _, nets, _, p = oracle_setup(w)
            _, nets_b, _, p_b = oracle_setup(w, net_precision="bf16")
            _, errs, frac = check_bf16_step(s.read_channels(), st, 1, nets, p, nets_b, p_b)
            print(w.width, w.height, errs, "band", round(frac, 4))
            assert frac <= 0.05
    finally:
        for s in subs:
            s.close()


def radiating_worlds(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k, every in enumerate([2, 0, 3, 1, 2]):
        W = int(rng.integers(20, 200))
        H = int(rng.integers(12, 120))
        out.append(worlds.make_world(width=W, height=H, n_genomes=int(rng.integers(2, 20)), hidden=32, net="cppn",
                                     seed=300 + k, radiation_every=every, p_mut=6e-3, p_merge=6e-3,
                                     capacity=400, random_rotation=bool(k % 2)))
    return out


def test_batched_radiation_equals_alone_bit_exact():
    """Worlds with their own radiation schedules (every 1, 2, 3 steps, or none) inside one batch,
    over several epochs and two step calls: state, genome tables and stats as stepping alone; the
    tuner in between (graphs only) leaves the genome tables as they are."""
    ws = radiating_worlds()
    alone = []
    for w in ws:
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as s:
            s.step(7)
            alone.append((s.read_channels(), s.read_genomes(), s.read_stats(0, 7)))
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        with coral.Batch(subs) as b:
            b.step(3)
            b.tune(trial_steps=1)
            b.step(4)
        born = 0
        for (ref, (genes, parent), stats), s in zip(alone, subs):
            got = s.read_channels()
            for k in ref:
                assert np.array_equal(ref[k], got[k]), k
            g2, p2 = s.read_genomes()
            assert np.array_equal(genes, g2) and np.array_equal(parent, p2)
            bs = s.read_stats(0, 7)
            for a, c in zip(stats, bs):
                for k in ("n_mut", "n_merge", "n_born", "n_skipped", "n_live", "n_explore"):
                    assert a[k] == c[k], (k, a, c)
            born += sum(a["n_born"] for a in stats)
        assert born > 0
    finally:
        for s in subs:
            s.close()


def test_batched_radiation_matches_oracle():
    """Exploration off keeps G fixed through the physics, so each radiation event of a batched
    world sees the same G as the oracle's: hit set, slots, parents and G bit-exact, genes within
    FP32 rounding, event counts equal; a world without radiation runs alongside."""
    from oracle import coral_oracle as O
    from parity import oracle_setup
    ws = [worlds.make_world(width=96, height=64, n_genomes=10, hidden=32, net="cppn", seed=21, radiation_every=1,
                            p_mut=4e-3, p_merge=8e-3, capacity=200),
          worlds.make_world(width=51, height=37, n_genomes=6, hidden=32, net="cppn", seed=22, radiation_every=1,
                            p_mut=1e-2, p_merge=1e-2, capacity=120, random_rotation=True),
          worlds.make_world(width=40, height=30, n_genomes=4, hidden=32, net="cppn", seed=23)]
    for w in ws[:2]:
        w.physics["k_exp"] = 0.0
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        refs = []
        for w in ws[:2]:
            st, nets, gen, p = oracle_setup(w)
            refs.append([st, gen, p])
        with coral.Batch(subs) as b:
            for t in range(3):
                b.step(1)
                for ref, s in zip(refs, subs[:2]):
                    st, gen, p = ref
                    st, gen, slots, ev = O.radiation(st, gen, t, p)
                    ref[0], ref[1] = st, gen
                    G = s.read_channels(coral.CH_G)["G"].ravel()
                    genes, parent = s.read_genomes()
                    c = s.read_stats(t, 1)[0]
                    assert np.array_equal(G, st.G), t
                    assert np.array_equal(parent, gen.parent), t
                    assert np.max(np.abs(genes - gen.genes)) <= 1e-6 * max(1.0, np.max(np.abs(gen.genes)))
                    assert c["n_mut"] == ev["n_mut"] and c["n_merge"] == ev["n_merge"]
                    assert c["n_born"] == ev["n_assigned"] and c["n_skipped"] == ev["n_skipped"]
        assert sum(r[1].parent[r[1].parent >= 0].size for r in refs) > 0
    finally:
        for s in subs:
            s.close()


def test_batched_fma_path_equals_alone():
    """With the small-genome path on (cutoff 8), each batched world is bit-identical to the same
    world stepped alone with that cutoff (both run the same kernel body)."""
    ws = [worlds.make_square_world(side, n, 32, seed=side + n) for side, n in ((96, 40), (200, 150), (64, 9))]
    ws.append(worlds.make_world(width=77, height=50, n_genomes=25, hidden=32, layout="random", net="cppn", seed=3))
    alone = []
    for w in ws:
        with coral.substrate_for_world(w, coral.BF16_GROUPED) as s:
            s.set_fma_cutoff(8)
            s.step(4)
            alone.append(s.read_channels())
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    try:
        with coral.Batch(subs) as b:
            b.set_fma_cutoff(8)
            b.step(4)
        for ref, s in zip(alone, subs):
            got = s.read_channels()
            for k in ref:
                assert np.array_equal(ref[k], got[k]), k
    finally:
        for s in subs:
            s.close()
