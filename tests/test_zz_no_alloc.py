"""The allocation-free counting entry point (fz_count_upto_noalloc).

It exists for callers that cannot call cudaMalloc (inside stream capture, in
loops that must not wait on the allocator, or when another allocator owns the
device memory): its scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test.  The output must equal the allocating entry point
fz_count_upto exactly (counts are integers), on two calls in a row.
"""
import numpy as np
import pytest

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


def test_limit_is_enforced(fz):
    out = torch.zeros(fz.FZ_NOALLOC_MAX_N + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.fz_count_upto_noalloc((3, 5), fz.FZ_NOALLOC_MAX_N + 1, out)
    assert e.value.status == fz.FZ_EINVAL
