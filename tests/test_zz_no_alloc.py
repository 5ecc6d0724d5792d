"""The allocation-free cell sort (for callers that cannot allocate device memory, e.g. code
running under another framework's memory pool or a real-time loop that must not enter the
CUDA allocator) gives exactly what the allocating entry point gives, on two calls in a row
that share its fixed in-library scratch, and rejects inputs above its fixed limits.

This file is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RCS = 2.0951 * 1.80 + 0.5


def _soa(x):
    return torch.tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=torch.float64, device="cuda")


def _bin(fn, x, box):
    n = len(x)
    cap = 4096
    cell = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    start = torch.full((cap + 1,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nc = fn(_soa(x), n, box, RCS, cell, start, perm, cap)
    torch.cuda.synchronize()
    tot = int(np.prod(nc))
    return nc, cell.cpu().numpy(), start.cpu().numpy()[: tot + 1], perm.cpu().numpy()


def test_noalloc_cell_bin_matches_allocating_entry_point_twice():
    from paper_2103_10449_gb300 import nefe as N
    xa, ba = I.liquid(3000, 0.05425, seed=21)
    xa = xa + np.array([-40.0, 13.0, 200.0])
    xb, bb = I.diamond(6, 6, 6)
    xb = I.rattle(xb, 0.2, 22)
    for x, box in ((xa, ba), (xb, bb)):        # two calls in a row on the shared scratch
        ref = _bin(N.nefe_cell_bin, x, box)
        got = _bin(N.nefe_cell_bin_noalloc, x, box)
        assert ref[0] == got[0]
        for r, g in zip(ref[1:], got[1:]):
            assert np.array_equal(r, g)


def test_noalloc_cell_bin_rejects_sizes_above_its_limits():
    from paper_2103_10449_gb300 import nefe as N
    n = N.NOALLOC_MAX_ATOMS + 1
    x = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(N.NefeError, match="fixed maximum"):
        N.nefe_cell_bin_noalloc(x, n, (100.0, 100.0, 100.0), RCS, out, out, out, 1 << 20)
    box = (300.0, 300.0, 300.0)                 # 70^3 cells > NOALLOC_MAX_CELLS
    with pytest.raises(N.NefeError, match="fixed maximum"):
        N.nefe_cell_bin_noalloc(x, 16, box, RCS, out, out, out, 1 << 20)
