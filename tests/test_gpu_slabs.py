"""One world stepped as row slabs (logical ranks: several substrates on one GPU, ghost rows
exchanged by device copies, radiation combined across the slabs) against the same world in one
substrate: the state, the genome table and the radiation decisions must be bit-identical, and
the own-row FP64 totals combined over the slabs must match the whole world's."""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, slabs, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def whole(w, path, steps):
    with coral.substrate_for_world(w, path) as s:
        s.step(steps)
        ch = s.read_channels()
        genes, parent = s.read_genomes()
        stats = s.read_stats(0, steps)
        tot = s.slab_totals()
    return ch, genes, parent, stats, tot


@pytest.mark.parametrize("path", [coral.BF16_GROUPED, coral.FP32_PERCELL])
@pytest.mark.parametrize("ranks", [1, 2, 3, 4])
def test_slabs_bit_identical_to_one_substrate(path, ranks):
    w = worlds.make_world(width=96, height=61, n_genomes=9, hidden=32, net="cppn", seed=17, random_rotation=True,
                          radiation_every=2, p_mut=3e-3, p_merge=3e-3, capacity=300)
    steps = 7
    ref, genes, parent, stats, tot = whole(w, path, steps)
    assert sum(s["n_born"] for s in stats) > 0          # radiation created genomes
    with slabs.SlabWorld(w, ranks, path) as sw:
        sw.step(steps)
        got = sw.read_channels()
        g2, p2 = sw.read_genomes()
        per = [s.read_stats(steps - 1, 1)[0] for s in sw.subs]
        t2 = sw.totals()
    for k in ("E", "I", "C", "G", "R"):
        assert np.array_equal(ref[k], got[k]), k
    assert np.array_equal(genes, g2) and np.array_equal(parent, p2)
    # the radiation event counts of the last event are global: every slab holds them
    for s in per:
        for k in ("n_mut", "n_merge", "n_born", "n_skipped", "n_live"):
            assert s[k] == stats[-1][k], k
    np.testing.assert_allclose(t2, tot, rtol=1e-12)


def test_slab_radiation_with_exhausted_slots():
    """More hits than free slots: the skipped hits are the same ones in both forms."""
    w = worlds.make_world(width=64, height=48, n_genomes=6, hidden=16, net="cppn", seed=5,
                          radiation_every=1, p_mut=0.03, p_merge=0.02, capacity=40)
    ref, genes, parent, stats, _ = whole(w, coral.BF16_GROUPED, 3)
    assert stats[0]["n_skipped"] > 0
    with slabs.SlabWorld(w, 3) as sw:
        sw.step(3)
        got = sw.read_channels()
        g2, p2 = sw.read_genomes()
    assert np.array_equal(ref["G"], got["G"]) and np.array_equal(genes, g2) and np.array_equal(parent, p2)
