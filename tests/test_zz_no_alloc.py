"""The allocation-free counting entry point (fz_count_upto_noalloc).

It exists for callers that cannot call cudaMalloc (inside stream capture, in
loops that must not wait on the allocator, or when another allocator owns the
device memory): its scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test.  The output must equal the allocating entry point
fz_count_upto exactly (counts are integers), on two calls in a row, and the
oracle's counts (the coefficients of prod 1/(1 - x^g_i)), saturated at
2^64 - 1 as the library documents.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fz():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20474_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return m


def _noalloc(fz, g, n_max):
    out = torch.full((n_max + 1,), -1, dtype=torch.int64, device="cuda")
    fz.fz_count_upto_noalloc(g, n_max, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def test_two_calls_in_a_row_match_the_allocating_call(fz):
    cases = [((5, 8, 11, 14), 500), ((2, 3, 5), fz.FZ_NOALLOC_MAX_N),
             ((56, 90, 96, 127, 146, 178), 39064), ((1,) * 16, 3000)]
    for g, n_max in cases:
        ref = fz.fz_count_upto(g, n_max)
        first = _noalloc(fz, g, n_max)
        second = _noalloc(fz, g, n_max)
        assert np.array_equal(first, ref), g
        assert np.array_equal(second, ref), g
        assert np.array_equal(first, _oracle_saturated(g, n_max)), g


def _oracle_saturated(g, n_max):
    """The oracle's |Z(r, g)|, r = 0..n_max, saturated at 2^64 - 1."""
    exact = oracle.count_upto(g, n_max)
    if exact.dtype != object:
        return exact.astype(np.uint64)
    top = (1 << 64) - 1
    return np.array([min(int(v), top) for v in exact], dtype=np.uint64)


def test_oracle_saturation_reading():
    """The saturated oracle row is exact below 2^64 and saturates above."""
    row = _oracle_saturated((1,) * 16, 3000)
    assert int(row[0]) == 1 and int(row[1]) == 16
    assert int(row[-1]) == (1 << 64) - 1


def test_limit_is_enforced(fz):
    out = torch.zeros(fz.FZ_NOALLOC_MAX_N + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.fz_count_upto_noalloc((3, 5), fz.FZ_NOALLOC_MAX_N + 1, out)
    assert e.value.status == fz.FZ_EINVAL
