"""The allocation-free cell sort (for callers that cannot allocate device memory, e.g. code
running under another framework's memory pool or a real-time loop that must not enter the
CUDA allocator) gives exactly what the allocating entry point gives, on two calls in a row
that share its fixed in-library scratch (and the FP64 oracle's cell sort bit for bit), takes no
device memory in those calls, and rejects inputs above its fixed limits.

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


CAP = 4096


def _buffers(x):
    """Device input and output buffers of one call (allocated by torch, before any timing of
    device memory)."""
    n = len(x)
    return (_soa(x), torch.full((n,), -1, dtype=torch.int32, device="cuda"),
            torch.full((CAP + 1,), -1, dtype=torch.int32, device="cuda"),
            torch.full((n,), -1, dtype=torch.int32, device="cuda"))


def _call(fn, bufs, n, box):
    xd, cell, start, perm = bufs
    return fn(xd, n, box, RCS, cell, start, perm, CAP)


def _read(nc, bufs):
    torch.cuda.synchronize()
    tot = int(np.prod(nc))
    _, cell, start, perm = bufs
    return nc, cell.cpu().numpy(), start.cpu().numpy()[: tot + 1], perm.cpu().numpy()


def _bin(fn, x, box):
    bufs = _buffers(x)
    return _read(_call(fn, bufs, len(x), box), bufs)


def test_noalloc_cell_bin_matches_allocating_entry_point_twice():
    from oracle import oracle as O
    from paper_2103_10449_gb300 import nefe as N
    xa, ba = I.liquid(3000, 0.05425, seed=21)
    xa = xa + np.array([-40.0, 13.0, 200.0])
    xb, bb = I.diamond(6, 6, 6)
    xb = I.rattle(xb, 0.2, 22)
    cases = ((xa, ba), (xb, bb))
    refs = [_bin(N.nefe_cell_bin, x, box) for x, box in cases]
    _bin(N.nefe_cell_bin_noalloc, xb, bb)        # first call on this device: looks up the scratch address
    bufs = [_buffers(x) for x, _ in cases]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ncs = [_call(N.nefe_cell_bin_noalloc, b, len(x), box) for b, (x, box) in zip(bufs, cases)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # the two calls took no device memory
    for (x, box), ref, nc, b in zip(cases, refs, ncs, bufs):   # two calls in a row on the shared scratch
        got = _read(nc, b)
        orc = O.cell_bin(x, box, RCS)
        assert ref[0] == got[0] == tuple(int(v) for v in orc[0])
        for r, g, o in zip(ref[1:], got[1:], orc[1:]):
            assert np.array_equal(r, g)
            assert np.array_equal(g, o)           # bit-exact against the FP64 oracle


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
