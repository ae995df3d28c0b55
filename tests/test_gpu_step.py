"""GPU parity of the substrate step through the C ABI against the FP64 oracle.

Each test seeds a world, runs the oracle and the CUDA library on the same inputs and
compares element by element: GenomeIndex and rotation bit-exact outside the decision band,
float channels within the per-channel normwise tolerance."""
import numpy as np
import pytest

from oracle import coral_oracle as O
from paper_2406_09654_gb300 import coral, worlds
from parity import (FP32_TAU, FP32_TOL, band_mask, compare_step, oracle_setup, rel_err,
                    round32, state_arrays)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def forced_steps(world, path, steps, tol, tau, t0=0, max_band_frac=0.05, **pkw):
    """Oracle-forced parity: at every step both sides start from the oracle's state (rounded
    to float32); the GPU's next state is compared with the oracle's next state. The cells set
    aside by the decision band may be at most max_band_frac of all compared cells."""
    st, nets, gen, p = oracle_setup(world, **pkw)
    sub = coral.substrate_for_world(world, path)
    worst = {}
    banded = 0
    try:
        st = round32(st)
        for t in range(t0, t0 + steps):
            sub.load_state(*state_arrays(st))
            sub.set_step(t)
            sub.step(1)
            g = sub.read_channels()
            new, info = O.step(st, nets, t, p)
            mask = band_mask(st, info, tau, p.rotation)
            banded += int(mask.sum())
            errs, bad_G, bad_R = compare_step(g, new, mask, tol)
            assert bad_G == 0 and bad_R == 0, (t, bad_G, bad_R)
            for k, v in errs.items():
                worst[k] = max(worst.get(k, 0.0), v)
            assert max(errs.values()) <= tol, (t, errs)
            st = round32(new)
    finally:
        sub.close()
    assert banded <= max_band_frac * steps * world.n_cells, banded
    return worst, banded


def test_cfg1_fp32_forced_100_steps():
    w = worlds.make_world("cfg1", seed=0)
    worst, banded = forced_steps(w, coral.FP32_PERCELL, 100, FP32_TOL, FP32_TAU)
    print("cfg1 worst per-channel error", worst, "band cells", banded)


FREE_TAU = 2e-6   # about 5x the FP32 path's observed per-step error on cfg1


def test_cfg1_fp32_free_running_100_steps():
    """Free-running: both sides step from the initial state with no re-loading. Compared
    step by step until the oracle meets a decision within FREE_TAU of flipping (then the
    trajectories may legitimately part); the step reached is printed."""
    w = worlds.make_world("cfg1", seed=0)
    st, nets, gen, p = oracle_setup(w)
    sub = coral.substrate_for_world(w, coral.FP32_PERCELL)
    first_band = None
    try:
        for t in range(100):
            new, info = O.step(st, nets, t, p)
            sub.step(1)
            mask = band_mask(st, info, FREE_TAU, p.rotation)
            if mask.any():
                first_band = t
                break
            g = sub.read_channels()
            errs, bad_G, bad_R = compare_step(g, new, mask, FP32_TOL)
            assert bad_G == 0 and bad_R == 0, t
            assert max(errs.values()) <= FP32_TOL, (t, errs)
            st = new
    finally:
        sub.close()
    print("free-running cfg1: identical within tolerance up to step",
          100 if first_band is None else first_band)
    assert first_band is None or first_band >= 5


@pytest.mark.parametrize("W,H,n,hidden,rot", [(3, 3, 1, 0, 1), (3, 5, 2, 16, 1), (37, 29, 7, 32, 1),
                                              (64, 48, 9, 48, 0), (130, 67, 13, 64, 1)])
def test_fp32_shapes_and_hidden_sizes(W, H, n, hidden, rot):
    w = worlds.make_world(width=W, height=H, n_genomes=n, hidden=hidden, net="cppn" if hidden else "direct",
                          seed=W * 7 + H, random_rotation=True, rotation=rot)
    # on the 3x3 and 3x5 tori a single near-tie is 7-11% of the grid
    forced_steps(w, coral.FP32_PERCELL, 4, FP32_TOL, FP32_TAU, t0=97, max_band_frac=0.05 if W * H > 15 else 0.25)


def test_fp32_day_night_boundary_and_stats():
    w = worlds.make_world(width=40, height=24, n_genomes=5, hidden=32, net="cppn", seed=11)
    st, nets, gen, p = oracle_setup(w)
    sub = coral.substrate_for_world(w, coral.FP32_PERCELL)
    try:
        st = round32(st)
        for t in (99, 100, 199, 200):
            sub.load_state(*state_arrays(st))
            sub.set_step(t)
            sub.step(1)
            new, info = O.step(st, nets, t, p)
            s = sub.read_stats(t, 1)[0]
            tot = O.totals(new)
            assert s["step"] == t
            assert s["sum_E"] == pytest.approx(tot["E"], rel=2e-6)
            mask = band_mask(st, info, FP32_TAU, p.rotation)
            if not mask.any():
                assert s["sum_I"] == pytest.approx(tot["I"], rel=2e-6)
                assert s["n_explore"] == info["n_explore"] and s["n_takeover"] == info["n_takeover"]
            for k in range(4):
                assert s["sum_C"][k] == pytest.approx(tot["C"][k], rel=2e-6)
            st = round32(new)
    finally:
        sub.close()


def test_degenerate_no_infrastructure_no_flow():
    w = worlds.make_world(width=16, height=16, n_genomes=3, hidden=0, seed=5)
    w.I[:] = 0.0
    forced_steps(w, coral.FP32_PERCELL, 3, FP32_TOL, FP32_TAU)


def test_determinism_two_runs_identical():
    w = worlds.make_world(width=96, height=80, n_genomes=12, hidden=32, net="cppn", seed=3,
                          radiation_every=5, p_mut=3e-3, p_merge=3e-3, capacity=512)
    outs = []
    for _ in range(2):
        with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
            sub.step(12)
            outs.append(sub.read_channels())
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_checkpoint_resume_matches_uninterrupted():
    w = worlds.make_world(width=64, height=40, n_genomes=6, hidden=16, net="cppn", seed=8,
                          radiation_every=4, p_mut=5e-3, p_merge=5e-3, capacity=256)
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as a:
        a.step(10)
        full = a.read_channels()
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as b:
        b.step(5)
        ck = b.read_channels()
        genes, parent = b.read_genomes()
        t = b.get_step()
    with coral.Substrate(coral.params_from_world(w), w.width, w.height, w.capacity) as c:
        c.load_state(ck["E"], ck["I"], ck["C"], ck["G"], ck["R"])
        c.load_genomes(genes=genes, n=w.capacity)
        c.generate_weights()
        c.set_step(t)
        c.step(5)
        res = c.read_channels()
    for k in full:
        assert np.array_equal(full[k], res[k]), k


def test_cppn_generated_weights_match_direct_evaluation():
    for hidden in (0, 16, 32, 64):
        w = worlds.make_world(width=8, height=8, n_genomes=6, hidden=hidden, net="cppn", seed=hidden)
        with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
            for g in range(6):
                got = sub.read_weights(g)
                W1, b1, W2, b2 = O.cppn_weights(w.genes[g].astype(np.float64), hidden)
                ref = np.concatenate([W1.ravel(), b1.ravel()] + ([] if hidden == 0 else [W2.ravel(), b2.ravel()]))
                assert rel_err(got, ref) <= 2e-6, (hidden, g, rel_err(got, ref))


def test_dense_nets_round_trip():
    w = worlds.make_world(width=8, height=8, n_genomes=4, hidden=32, seed=2)
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
        for g in range(4):
            assert np.array_equal(sub.read_weights(g), w.dense[g])


@pytest.mark.parametrize("W,H,cap,layout", [(50, 40, 300, "random"), (64, 64, 8, "voronoi"),
                                            (33, 31, 70000, "random"), (3, 3, 1, "voronoi"),
                                            (300, 250, 300, "random"), (300, 250, 70000, "random"),
                                            (257, 255, 4000, "voronoi")])
def test_bucket_counting_sort_bit_exact(W, H, cap, layout):
    n = min(cap, 200)
    w = worlds.make_world(width=W, height=H, n_genomes=max(1, min(n, W * H)), layout=layout, seed=W, capacity=cap)
    if cap == 70000:
        w.G = (w.G * 347 + 65000) % cap      # keys above 2^16: three digit passes
        w.G = w.G.astype(np.int32)
    with coral.Substrate(coral.params_from_world(w), W, H, cap) as sub:
        sub.load_state(w.E, w.I, w.C, w.G, w.R)
        counts, perm = sub.read_perm()
    c_ref, off_ref, perm_ref = O.bucket(w.G.ravel(), cap)
    assert np.array_equal(counts, c_ref) and np.array_equal(perm, perm_ref)


def test_radiation_bit_exact_without_exploration():
    """k_exp = 0 keeps G fixed through the physics, so the radiation event (after step 0,
    M = 1) sees the same G on both sides: hit set, slots, parents, G and genes must agree."""
    w = worlds.make_world(width=96, height=64, n_genomes=10, hidden=16, net="cppn", seed=21,
                          radiation_every=1, p_mut=4e-3, p_merge=8e-3, capacity=200)
    w.physics["k_exp"] = 0.0
    st, nets, gen, p = oracle_setup(w)
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
        for t in range(3):
            sub.step(1)
            new, info = O.step(st, nets, t, p)
            new, gen, slots, ev = O.radiation(new, gen, t, p)
            O.nets_from_genomes(gen, p.hidden, slots, nets)
            g = sub.read_channels()
            genes, parent = sub.read_genomes()
            s = sub.read_stats(t, 1)[0]
            assert np.array_equal(g["G"].ravel(), new.G), t
            assert np.array_equal(parent, gen.parent), t
            assert rel_err(genes, gen.genes) <= 1e-6
            assert s["n_mut"] == ev["n_mut"] and s["n_merge"] == ev["n_merge"]
            assert s["n_born"] == ev["n_assigned"] and s["n_skipped"] == ev["n_skipped"]
            for slot in slots[:5]:
                W1, b1, W2, b2 = O.cppn_weights(gen.genes[slot], 16)
                ref = np.concatenate([W1.ravel(), b1, W2.ravel(), b2])
                assert rel_err(sub.read_weights(slot), ref) <= 1e-5
            st = round32(new)
            sub.load_state(*state_arrays(st))
            sub.set_step(t + 1)


def test_radiation_capacity_exhaustion_counts_skips():
    w = worlds.make_world(width=64, height=64, n_genomes=4, hidden=16, net="cppn", seed=2,
                          radiation_every=1, p_mut=0.02, capacity=20)
    w.physics["k_exp"] = 0.0
    st, nets, gen, p = oracle_setup(w)
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
        sub.step(1)
        s = sub.read_stats(0, 1)[0]
        g = sub.read_channels(coral.CH_G)
    new, info = O.step(st, nets, 0, p)
    new, gen, slots, ev = O.radiation(new, gen, 0, p)
    assert ev["n_skipped"] > 0 and s["n_skipped"] == ev["n_skipped"] and s["n_born"] == 16
    assert np.array_equal(g["G"].ravel(), new.G)


def test_errors_are_reported():
    w = worlds.make_world(width=8, height=8, n_genomes=2, seed=1)
    p = coral.params_from_world(w)
    with pytest.raises(coral.CoralError) as e:
        coral.Substrate(p, 2, 8, 4)
    assert e.value.code == coral.E_INVALID
    with coral.Substrate(p, 8, 8, 4) as sub:
        with pytest.raises(coral.CoralError) as e:
            sub.step(1)
        assert e.value.code == coral.E_STATE
        bad = w.G.copy(); bad[0, 0] = 9
        sub.load_state(w.E, w.I, w.C, bad, w.R)
        with pytest.raises(coral.CoralError) as e:
            sub.sync()
        assert e.value.code == coral.E_INVALID
        sub.load_state(G=w.G)
        sub.sync()


def test_genome_distances_and_lineage_after_radiation():
    w = worlds.make_world(width=96, height=64, n_genomes=10, hidden=16, net="cppn", seed=21,
                          radiation_every=1, p_mut=4e-3, p_merge=8e-3, capacity=200)
    with coral.substrate_for_world(w, coral.FP32_PERCELL) as sub:
        sub.step(3)
        genes, parent = sub.read_genomes()
        born = [s for s in range(200) if parent[s] >= 0]
        slots = np.array(list(range(10)) + born[:20], np.int32)
        d = sub.genome_distances(slots)
    for i, a in enumerate(slots):
        for k, b in enumerate(slots):
            assert d[i, k] == pytest.approx(O.genetic_distance(genes[a], genes[b]), rel=1e-5, abs=1e-7)
    for s in born:
        anc = O.lineage(parent, s)
        assert anc[0] == s and parent[anc[-1]] == -1 and anc[-1] < 10
