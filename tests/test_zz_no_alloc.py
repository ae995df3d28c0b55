"""The allocation-free bucketing entry point (coral_bucket_noalloc), called through the C ABI.

It exists for callers that cannot allocate device memory when they need the sort (inside a
stream capture they do not own, or in loops where an allocator call is not allowed). Its
result must equal the regular entry point's (coral_read_perm) exactly: the sort is integer
work, so the tolerance is zero. Two calls in a row check that the shared scratch array's
leftover contents from the first call do not leak into the second.
"""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def reference(w):
    with coral.Substrate(coral.params_from_world(w), w.width, w.height, w.capacity) as sub:
        sub.load_state(w.E, w.I, w.C, w.G, w.R)
        return sub.read_perm()


def test_noalloc_bucket_matches_regular_entry_point_twice():
    import torch
    cases = [worlds.make_world(width=640, height=480, n_genomes=200, layout="random", seed=3, capacity=300),
             worlds.make_world(width=256, height=200, n_genomes=40, layout="voronoi", seed=4, capacity=40)]
    for w in cases:                          # second call: smaller input over the first's leftovers
        ref_counts, ref_perm = reference(w)
        G = torch.from_numpy(w.G.ravel().copy()).cuda()
        counts = torch.full((w.capacity,), -7, dtype=torch.int32, device="cuda")
        perm = torch.full((w.n_cells,), -7, dtype=torch.int32, device="cuda")
        coral.bucket_noalloc(G, w.capacity, counts, perm, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy(), ref_counts)
        assert np.array_equal(perm.cpu().numpy(), ref_perm)


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
