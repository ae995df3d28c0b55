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
