"""The world server on the GPU: requests arriving while others run are stepped in the same
batched launches, and every result is bit-identical to stepping that world alone."""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, serving, worlds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def test_served_results_equal_solo_runs():
    f = worlds.request_world_factory((16, 160), (2, 40))
    reqs = serving.poisson_requests(10, 400.0, f, (3, 25), seed=4)
    srv = serving.WorldServer(serving.CoralBackend(), budget_bytes=8 << 30, chunk_steps=3)
    done, rep = srv.run(reqs)
    assert rep["served"] == 10
    assert rep["mean_resident_worlds"] > 1.0          # work of several requests overlapped
    for c in done:
        r = reqs[c.rid]
        with coral.substrate_for_world(r.world, coral.BF16_GROUPED) as s:
            s.step(r.steps)
            ref = s.read_channels()
        for k in ref:
            assert np.array_equal(ref[k], c.result[k]), (c.rid, k)


def test_served_worlds_match_oracle():
    """Two one-step requests inside a served mix, compared with the oracle: each starts from the
    state the oracle reached after one step of its world (the server steps it as step 0; the
    oracle steps the same state as step 0)."""
    from oracle import coral_oracle as O
    from parity import check_bf16_step, oracle_setup, round32, state_arrays
    f = worlds.request_world_factory((16, 160), (2, 40))
    reqs = serving.poisson_requests(8, 400.0, f, (3, 12), seed=5)
    starts = {}
    for k, (W, H, seed) in enumerate([(96, 64, 31), (120, 88, 32)]):
        w = worlds.make_world(width=W, height=H, n_genomes=6, hidden=32, net="cppn", seed=seed)
        st, nets, _, p = oracle_setup(w)
        st = round32(O.step(round32(st), nets, 0, p)[0])
        w.E, w.I, w.C, w.G, w.R = state_arrays(st)
        rid = 100 + k
        reqs.append(serving.Request(reqs[2 + 3 * k].arrival, rid, w, 1))
        starts[rid] = (w, st)
    srv = serving.WorldServer(serving.CoralBackend(), budget_bytes=8 << 30, chunk_steps=3)
    done, rep = srv.run(reqs)
    assert rep["served"] == len(reqs)
    got = {c.rid: c.result for c in done}
    for rid, (w, st) in starts.items():
        _, nets, _, p = oracle_setup(w)
        _, nets_b, _, p_b = oracle_setup(w, net_precision="bf16")
        _, errs, frac = check_bf16_step(got[rid], st, 0, nets, p, nets_b, p_b)
        print(rid, errs, "band", round(frac, 4))
        assert frac <= 0.05
