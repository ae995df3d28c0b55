"""CPU checks of the C ABI library: it loads and exports every entry point declared in
include/coral.h; the compute-free calls behave as documented. No GPU is used."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_09654_gb300 import build, coral
    build.build()
    return coral.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "coral.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(coral_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("coral_substrate_create", "coral_genome_table_load", "coral_cppn_generate_weights",
              "coral_step", "coral_read_channels"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2406_09654_gb300 import coral
    out = subprocess.run(["nm", "-D", "--defined-only", coral.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (coral_\w+)", out))
    for n in declared():
        assert n in exported, n
        assert hasattr(lib, n)


def test_defaults_and_net_floats(lib):
    from paper_2406_09654_gb300 import coral
    p = coral.default_params()
    assert (p.hidden, p.path, p.day_period, p.rotation) == (0, 0, 200, 1)
    assert p.k_inv == pytest.approx(0.1) and p.k_exp == pytest.approx(0.5)
    assert p.k_flow == pytest.approx(0.2) and p.sigma_mut == pytest.approx(0.05)
    assert p.seed == 0 and p.p_mut == 0.0 and p.p_merge == 0.0
    assert coral.net_floats(0) == 550 and coral.net_floats(64) == 64 * 54 + 64 + 640 + 10


def test_invalid_arguments_fail_before_any_device_work(lib):
    from paper_2406_09654_gb300 import coral
    p = coral.default_params()
    for w, h, cap in ((2, 8, 4), (8, 2, 4), (8, 8, 0), (70000, 70000, 4)):
        with pytest.raises(coral.CoralError) as e:
            coral.Substrate(p, w, h, cap)
        assert e.value.code == coral.E_INVALID
    p.hidden = 20
    with pytest.raises(coral.CoralError) as e:
        coral.Substrate(p, 8, 8, 4)
    assert e.value.code == coral.E_INVALID
    assert lib.coral_step(None, 1) == coral.E_INVALID
    assert lib.coral_step_jobs(None, 1, None, None, 1, 0) == coral.E_INVALID
    assert b"NULL" in lib.coral_last_error(None)


def test_radiation_probabilities_are_validated(lib):
    """p_mut and p_merge are probabilities: the library turns them into Philox thresholds and
    refuses values outside [0, 1] (checked before any device work)."""
    from paper_2406_09654_gb300 import coral
    for field, bad in (("p_mut", -0.1), ("p_mut", 1.5), ("p_merge", float("nan")), ("p_merge", 2.0)):
        p = coral.default_params()
        setattr(p, field, bad)
        with pytest.raises(coral.CoralError) as e:
            coral.Substrate(p, 8, 8, 4)
        assert e.value.code == coral.E_INVALID and "p_mut and p_merge" in str(e.value)


def test_selftest_rejects_bad_arguments(lib):
    from paper_2406_09654_gb300 import coral
    import ctypes
    st = ctypes.c_int32(0)
    assert lib.coral_selftest_wait_timeout(None, 0, ctypes.byref(st)) == coral.E_INVALID
    assert lib.coral_selftest_wait_timeout(None, 10, None) == coral.E_INVALID
