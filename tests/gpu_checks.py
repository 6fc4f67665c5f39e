"""Checks of GPU output that hold at any size (plain torch ops, test-side only).

A list is exactly Z(n, g) in descending lexicographic order iff
  (1) every row is a non-negative solution of sum a_i g_i = n,
  (2) consecutive rows are strictly decreasing lexicographically, and
  (3) it has |Z(n, g)| rows (taken from the oracle).
(1)+(2) make it a strictly sorted list of distinct members of Z(n, g); (3)
then forces it to be all of Z(n, g).
"""
import torch


def check_sorted_solutions(rows: torch.Tensor, g, n: int, chunk: int = 1 << 25):
    """Assert (1) and (2) on a CUDA int32 tensor of shape (N, d)."""
    N, d = rows.shape
    assert d == len(g)
    gt = torch.tensor([int(x) for x in g], dtype=torch.int64, device=rows.device)
    start = 0
    while start < N:
        stop = min(N, start + chunk)
        x = rows[start:min(N, stop + 1)].to(torch.int64)
        assert bool((x >= 0).all()), "negative coordinate near row %d" % start
        s = (x * gt).sum(dim=1)
        bad = torch.nonzero(s != n)
        assert bad.numel() == 0, "row %d does not sum to n" % (start + int(bad[0, 0]))
        if x.shape[0] > 1:
            diff = x[:-1] - x[1:]
            nz = diff != 0
            dup = torch.nonzero(~nz.any(dim=1))
            assert dup.numel() == 0, "duplicate rows at %d" % (start + int(dup[0, 0]))
            first = nz.to(torch.int8).argmax(dim=1, keepdim=True)
            lead = diff.gather(1, first).squeeze(1)
            inv = torch.nonzero(lead <= 0)
            assert inv.numel() == 0, "order broken at row %d" % (start + int(inv[0, 0]))
        start = stop


def check_csr_segments(offsets: torch.Tensor, rows: torch.Tensor, g, counts,
                       chunk_elems: int = 64):
    """Every CSR segment m holds |Z(m, g)| = counts[m] rows, each a solution
    for m, strictly descending (offsets: uint64/int64 CUDA tensor, top+1)."""
    off = offsets.to(torch.int64).cpu().tolist()
    top = len(off) - 1
    assert off[0] == 0
    for m in range(top):
        assert off[m + 1] - off[m] == int(counts[m]), "segment %d size" % m
    gt = torch.tensor([int(x) for x in g], dtype=torch.int64, device=rows.device)
    x = rows.to(torch.int64)
    # sums: one pass over all rows against their segment's element
    seg = torch.repeat_interleave(
        torch.arange(top, device=rows.device, dtype=torch.int64),
        torch.tensor([off[m + 1] - off[m] for m in range(top)], device=rows.device))
    assert bool((x >= 0).all())
    assert bool(((x * gt).sum(dim=1) == seg).all()), "a memo row does not sum to its element"
    if x.shape[0] > 1:
        same = seg[:-1] == seg[1:]
        diff = x[:-1] - x[1:]
        nz = diff != 0
        first = nz.to(torch.int8).argmax(dim=1, keepdim=True)
        lead = diff.gather(1, first).squeeze(1)
        ok = (~same) | (nz.any(dim=1) & (lead > 0))
        assert bool(ok.all()), "memo segment not strictly descending"


_M64 = (1 << 64) - 1
_K0 = 0x9E3779B97F4A7C15 - (1 << 64)  # the oracle's row-digest constants, as int64
_K1 = 0x632BE59BD9B4E019
_LSR2 = (1 << 62) - 1


def rows_digest(rows: torch.Tensor, rank0: int = 0, chunk: int = 1 << 22) -> int:
    """The oracle's order-sensitive digest (oracle.digest) of int32 rows of
    any device, row r having rank rank0 + r: the sum mod 2^64 over rows of
    h = rank * K0, then for each coordinate a, h ^= a + K1 + (h << 6) + (h >> 2)
    (unsigned 64-bit; here int64 with wrap-around, << as a product and the
    logical >> as an arithmetic one masked)."""
    N, d = rows.shape
    total = 0
    start = 0
    while start < N:
        stop = min(N, start + chunk)
        x = rows[start:stop].to(torch.int64)
        h = torch.arange(rank0 + start, rank0 + stop, dtype=torch.int64, device=rows.device)
        h = h * _K0
        for i in range(d):
            h = h ^ (x[:, i] + _K1 + h * 64 + ((h >> 2) & _LSR2))
        total = (total + int(h.sum().item())) & _M64
        start = stop
    return total
