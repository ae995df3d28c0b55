"""Host-to-host job stepping (coral_step_jobs): several states copied in, stepped and copied
out with the copies overlapping the steps give exactly what loading, stepping and reading each
state in turn gives."""
import numpy as np
import pytest
import torch

from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def packed(w, seed):
    """A packed state (CH_ALL order) of world w's shape with its own seeded values."""
    rng = np.random.default_rng(seed)
    n = w.n_cells
    E = rng.uniform(0, 1, n).astype(np.float32)
    I = rng.uniform(0, 0.5, n).astype(np.float32)
    C = rng.normal(0, 0.1, 4 * n).astype(np.float32)
    G = rng.integers(0, w.n_genomes, n).astype(np.int32)
    R = rng.integers(0, 4, n).astype(np.uint8)
    buf = torch.empty(coral.STATE_BYTES * n, dtype=torch.uint8, pin_memory=True)
    v = buf.numpy()
    v[:24 * n] = np.concatenate([E, I, C]).view(np.uint8)
    v[24 * n:28 * n] = G.view(np.uint8)
    v[28 * n:] = R
    return buf


def unpack(buf, n):
    v = buf.numpy() if hasattr(buf, "numpy") else buf
    f = v[:24 * n].view(np.float32)
    return f[:n], f[n:2 * n], f[2 * n:].reshape(4, n), v[24 * n:28 * n].view(np.int32), v[28 * n:]


@pytest.mark.parametrize("path,radiation", [(coral.BF16_GROUPED, 0), (coral.FP32_PERCELL, 3)])
def test_jobs_match_sequential_load_step_read(path, radiation):
    w = worlds.make_world(width=96, height=64, n_genomes=9, hidden=32, net="cppn", seed=21,
                          radiation_every=radiation, p_mut=4e-3, p_merge=4e-3, capacity=512)
    n = w.n_cells
    ins = [packed(w, 100 + k) for k in range(5)]
    outs = [torch.empty_like(b).pin_memory() for b in ins]
    steps, t0 = 4, 197                                   # crosses the day/night boundary
    with coral.substrate_for_world(w, path) as sub:
        sub.step_jobs(ins, outs, steps, t0)
        assert sub.get_step() == t0 + steps
    with coral.substrate_for_world(w, path) as ref:
        for k, b in enumerate(ins):
            E, I, C, G, R = unpack(b, n)
            ref.load_state(E, I, C.reshape(4, w.height, w.width), G, R)
            ref.set_step(t0)
            ref.step(steps)
            want = ref.read_channels(coral.CH_ALL, out=np.empty(coral.STATE_BYTES * n, np.uint8))
            assert np.array_equal(outs[k].numpy(), want), f"job {k}"


def test_jobs_shared_buffers_and_invalid_input():
    w = worlds.make_world(width=64, height=48, n_genomes=5, hidden=16, net="cppn", seed=4)
    n = w.n_cells
    good = packed(w, 1)
    out = torch.empty_like(good).pin_memory()
    with coral.substrate_for_world(w, coral.BF16_GROUPED) as sub:
        sub.step_jobs([good] * 4, [out] * 4, 2, 0)       # one shared input and output buffer
        single = torch.empty_like(good).pin_memory()
        sub.step_jobs([good], [single], 2, 0)
        assert np.array_equal(out.numpy(), single.numpy())
        bad = good.clone().pin_memory()
        bad.numpy()[24 * n:28 * n].view(np.int32)[7] = w.capacity   # GenomeIndex out of range
        with pytest.raises(coral.CoralError) as e:
            sub.step_jobs([good, bad], [out, single], 1, 0)
        assert e.value.code == coral.E_INVALID
