"""Failure detection on the GPU without a fault: a bounded device-side wait on a barrier that
nothing arrives on runs out, the kernel reports a timeout status, releases its tensor memory,
and the context keeps working."""
import time

import numpy as np
import pytest

from paper_2406_09654_gb300 import coral, worlds

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2406_09654_gb300 import build
    build.build()
    t0 = time.perf_counter()
    assert coral.selftest_wait_timeout(2000) == coral.E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert coral.selftest_wait_timeout(500) == coral.E_TIMEOUT       # again: TMEM was released
    w = worlds.make_world(width=64, height=32, n_genomes=3, hidden=32, net="cppn", seed=2)
    with coral.substrate_for_world(w, coral.BF16_GROUPED) as s:
        s.step(2)
        g = s.read_channels()
    assert np.all(np.isfinite(g["E"])) and g["G"].max() < 3
