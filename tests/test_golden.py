"""The oracle against its stored results on two small seeded worlds (tests/golden): any change
to the oracle's arithmetic shows up here and must be justified by the passage it follows."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_stored_small_worlds():
    stored = json.load(open(os.path.join(HERE, "golden", "oracle_small_worlds.json")))
    now = _maker().build()
    assert set(stored) == set(now)
    for name in stored:
        a, b = stored[name]["oracle"], now[name]["oracle"]
        # integer state and decisions: exact
        assert a["G"] == b["G"] and a["R"] == b["R"], name
        assert a.get("parent") == b.get("parent"), name
        for ta, tb in zip(a["totals"], b["totals"]):
            assert ta["t"] == tb["t"] and ta["n_explore"] == tb["n_explore"] and ta["n_takeover"] == tb["n_takeover"]
            np.testing.assert_allclose([ta["E"], ta["I"], *ta["C"]], [tb["E"], tb["I"], *tb["C"]], rtol=1e-9)
        # FP64 planes: equal up to summation order of the host's BLAS
        np.testing.assert_allclose(a["E"], b["E"], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(a["I"], b["I"], rtol=1e-9, atol=1e-12)
