"""The C-ABI library builds, loads and exports every entry point that
include/fz.h declares (CPU-only: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fz_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libfz():
    from paper_2407_20474_gb300 import _build
    _build.build()
    import paper_2407_20474_gb300 as fz
    return fz.lib()


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ("fz_count", "fz_build_memo", "fz_enumerate", "fz_plan_create",
                 "fz_plan_enumerate", "fz_plan_unrank"):
        assert must in names


def test_every_declared_symbol_is_exported(libfz):
    import paper_2407_20474_gb300 as fz
    names = declared_functions()
    missing = [n for n in names if not hasattr(libfz, n)]
    assert not missing, missing
    assert sorted(fz.EXPORTS) == names


def test_status_strings_and_version(libfz):
    import paper_2407_20474_gb300 as fz
    assert fz.fz_version() >= 100
    assert fz.status_string(fz.FZ_EINVAL) == "FZ_EINVAL"
    assert fz.status_string(fz.FZ_ENOSPC) == "FZ_ENOSPC"


def test_argument_errors_need_no_gpu(libfz):
    """Invalid arguments are rejected before any device work."""
    import paper_2407_20474_gb300 as fz
    with pytest.raises(fz.FzError) as e:
        fz.fz_count((3, 0, 5), 10)
    assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.fz_count((3, 5), -1)
    assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.fz_count(tuple(range(1, 18)), 10)
    assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.fz_memo_rows((4, 0), 10)
    assert e.value.status == fz.FZ_EINVAL
