"""The allocation-free bucketing entry point (coral_bucket_noalloc), called through the C ABI.

It exists for callers that cannot allocate device memory when they need the sort (inside a
stream capture they do not own, or in loops where an allocator call is not allowed). Its
result must equal the regular entry point's (coral_read_perm) and the oracle's stable counting
sort exactly: the sort is integer work, so the tolerance is zero. Two calls in a row check that
the shared scratch array's leftover contents from the first call do not leak into the second.
"""
import numpy as np
import pytest

from oracle import coral_oracle as O
from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def regular_entry_point(w):
    with coral.Substrate(coral.params_from_world(w), w.width, w.height, w.capacity) as sub:
        sub.load_state(w.E, w.I, w.C, w.G, w.R)
        return sub.read_perm()


def noalloc(G_host, capacity):
    import torch
    G = torch.from_numpy(np.ascontiguousarray(G_host, np.int32).ravel()).cuda()
    counts = torch.full((capacity,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((G.numel(),), -7, dtype=torch.int32, device="cuda")
    coral.bucket_noalloc(G, capacity, counts, perm, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return counts.cpu().numpy(), perm.cpu().numpy()


def test_noalloc_bucket_matches_regular_entry_point_and_oracle_twice():
    cases = [worlds.make_world(width=640, height=480, n_genomes=200, layout="random", seed=3, capacity=300),
             worlds.make_world(width=256, height=200, n_genomes=40, layout="voronoi", seed=4, capacity=40)]
    for w in cases:                          # second call: smaller input over the first's leftovers
        counts, perm = noalloc(w.G, w.capacity)
        ref_counts, ref_perm = regular_entry_point(w)
        assert np.array_equal(counts, ref_counts) and np.array_equal(perm, ref_perm)
        o_count, _, o_perm = O.bucket(w.G, w.capacity)
        assert np.array_equal(counts, o_count) and np.array_equal(perm, o_perm)


def test_noalloc_bucket_keys_out_of_range():
    """Keys outside [0, capacity) are not counted (valid slots' counts stay exact) and perm is
    still a permutation of the cells, as the header documents."""
    rng = np.random.default_rng(8)
    G = rng.integers(0, 200, 50_000).astype(np.int32)
    bad = rng.choice(G.size, 700, replace=False)
    G[bad[:400]] = 200 + rng.integers(0, 1000, 400)       # above capacity
    G[bad[400:]] = -rng.integers(1, 50, 300)              # negative
    counts, perm = noalloc(G, 200)
    ok = (G >= 0) & (G < 200)
    assert np.array_equal(counts, np.bincount(G[ok], minlength=200))
    assert counts.sum() == G.size - 700
    assert np.array_equal(np.sort(perm), np.arange(G.size))


def test_noalloc_bucket_rejects_sizes_beyond_its_scratch():
    import torch
    G = torch.zeros(coral.NOALLOC_MAX_CELLS + 1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    perm = torch.zeros(coral.NOALLOC_MAX_CELLS + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(coral.CoralError) as e:
        coral.bucket_noalloc(G, 4, counts, perm)
    assert e.value.code == coral.E_INVALID and "1048576" in str(e.value)
    with pytest.raises(coral.CoralError) as e:
        coral.bucket_noalloc(G[:10], coral.NOALLOC_MAX_CAPACITY + 1, counts, perm[:10])
    assert e.value.code == coral.E_INVALID
