"""The device Philox4x32-10 (the function the radiation kernels draw their hit words, partner
directions, crossover bits and mutation normals from) against the published known-answer
vectors of the generator (Salmon et al., SC'11; Random123's kat_vectors), through the C ABI."""
import numpy as np
import pytest

from paper_2406_09654_gb300 import coral
from test_oracle_pins import philox_kat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09654_gb300 import build
    build.build()
    coral.lib()


def test_device_philox_known_answer_vectors():
    kat = philox_kat()
    ctr = np.array([c for c, _, _ in kat], np.uint32)
    key = np.array([k for _, k, _ in kat], np.uint32)
    out = coral.philox4x32_10(ctr, key)
    assert out.tolist() == [o for _, _, o in kat]


def test_device_philox_equals_oracle_on_radiation_counters():
    from oracle import philox as P
    cells = np.arange(5000, dtype=np.uint64) * 977
    ref = P.draw(cells, 19, P.STREAM_MERGE, 0, 3, 0x0123456789ABCDEF)
    ctr = np.stack([cells.astype(np.uint32), np.full(5000, 19, np.uint32),
                    np.full(5000, P.STREAM_MERGE << 24, np.uint32), np.full(5000, 3, np.uint32)], 1)
    key = np.tile(np.array([0x89ABCDEF, 0x01234567], np.uint32), (5000, 1))
    out = coral.philox4x32_10(ctr, key)
    for w in range(4):
        assert np.array_equal(out[:, w], ref[w])
