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


def test_missing_or_broken_library_fails_loudly(tmp_path):
    """No CPU fallback: a missing or unloadable libfz.so raises FzError."""
    import subprocess
    import sys
    broken = tmp_path / "libfz_broken.so"
    broken.write_text("not a shared object")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_2407_20474_gb300 as fz\n"
        "for path in (%r, %r):\n"
        "    fz.LIB_PATH = path; fz._lib = None\n"
        "    try:\n"
        "        fz.fz_count((3, 5), 10)\n"
        "    except fz.FzError as e:\n"
        "        assert e.status == fz.FZ_ECUDA, e\n"
        "        print('raised', e)\n"
        "    else:\n"
        "        raise SystemExit('no error for ' + path)\n"
        % (ROOT, str(tmp_path / "missing.so"), str(broken)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("raised") == 2


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor: the binding's size checks read only these."""

    def __init__(self, numel, itemsize, contiguous=True, cuda=True):
        self._n, self._s, self._c, self.is_cuda = numel, itemsize, contiguous, cuda

    def data_ptr(self):
        return 0x1000

    def numel(self):
        return self._n

    def element_size(self):
        return self._s

    def is_contiguous(self):
        return self._c


def test_binding_checks_device_buffer_sizes():
    """Calls that write a caller buffer of implied size through a raw pointer
    reject, before any library call, a tensor that is too short, has the
    wrong element size, is not contiguous or is not on the device."""
    import paper_2407_20474_gb300 as fz
    bad = [_FakeDeviceTensor(100, 8), _FakeDeviceTensor(101, 4),
           _FakeDeviceTensor(101, 8, contiguous=False), _FakeDeviceTensor(101, 8, cuda=False)]
    for t in bad:
        with pytest.raises(fz.FzError) as e:
            fz.fz_count_upto_noalloc((3, 5), 100, t)
        assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.fz_count_table((3, 5), 10, _FakeDeviceTensor(3 * 11 - 1, 8))
    assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.fz_build_memo_into((3, 5), 10, _FakeDeviceTensor(11, 8), _FakeDeviceTensor(9, 4), 5)
    assert e.value.status == fz.FZ_EINVAL
    assert fz._devbuf(_FakeDeviceTensor(101, 8), 8, 101, "counts") == 0x1000
