"""Host copies of the state: pageable host arrays go through the packed staging path (one
contiguous copy, re-pitched on the device in the spare state buffer), pinned ones through
pitched 2-D copies. Both give the same bytes, and neither changes later steps or the totals
(the spare buffer's row padding is zero again afterwards)."""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


@pytest.mark.parametrize("W,H", [(37, 29), (130, 70), (64, 48)])
@pytest.mark.parametrize("path", [coral.BF16_GROUPED, coral.FP32_PERCELL])
def test_pageable_and_pinned_copies_agree_and_leave_steps_unchanged(W, H, path):
    import torch
    w = worlds.make_world(width=W, height=H, n_genomes=4, hidden=32, net="cppn", seed=W + H)
    with coral.substrate_for_world(w, path) as a, coral.substrate_for_world(w, path) as b:
        a.step(1)
        r = a.read_channels()                                   # pageable: staged
        C = np.stack([r[f"C{k}"] for k in range(4)])
        a.load_state(r["E"], r["I"], C, r["G"], r["R"])         # pageable: staged
        a.set_step(1)
        a.step(2)
        b.step(3)
        ra = a.read_channels()
        pinned = torch.empty(coral.STATE_BYTES * w.n_cells, dtype=torch.uint8).pin_memory()
        b.read_channels(coral.CH_ALL, out=pinned)               # pinned: pitched 2-D copies
        want = np.concatenate([ra[k].view(np.uint8).ravel() for k in ("E", "I", "C0", "C1", "C2", "C3", "G", "R")])
        assert np.array_equal(pinned.numpy(), want)
        ta, tb = a.slab_totals(), b.slab_totals()
        assert np.array_equal(ta, tb)
        ref = [ra["E"], ra["I"], ra["C0"], ra["C1"], ra["C2"], ra["C3"]]
        assert np.allclose(ta, [float(np.sum(p, dtype=np.float64)) for p in ref], rtol=1e-12, atol=1e-9)
