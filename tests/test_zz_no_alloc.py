"""rsos_width_noalloc: the width measurement for callers that cannot allocate
device memory (fixed budgets, real-time loops, lattice-only buffers).  Its
exact sums must equal rsos_width's on the same lattice, on two calls in a row
(the shared scratch array keeps the previous call's contents).  Collected last
so that a failure here never hides the other tests."""
import numpy as np
import pytest

import paper_1605_02620_gb300 as R

pytestmark = pytest.mark.gpu


def _to128(lo, hi):
    return [(int(h) << 64) + (int(l) & 0xFFFFFFFFFFFFFFFF) for l, h in zip(lo, hi)]


@pytest.mark.parametrize("L,N,S,tiling,tile", [(256, 2, 64, 0, 8), (4096, 1, 64, 0, 8), (512, 4, 96, 0, 8),
                                                (256, 1, 64, 1, (6, 10)), (100, 3, 32, 1, (7, 9))])
def test_noalloc_width_equals_rsos_width_on_two_calls(L, N, S, tiling, tile):
    import torch
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=tile, seed=123, series_capacity=4, tiling=tiling)
    nbytes = R.rsos_required_bytes(p)
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    B = 2 if N <= 1 else (3 if N <= 3 else 4)
    NW = (S + 31) // 32
    # site records per lattice: L * L, or with a (+1) tiling L rows of
    # T * ceil(L / T) records (T = tile_x: rows padded to whole column classes)
    T = tile[0] if isinstance(tile, tuple) else tile
    records = L * T * ((L + T - 1) // T) if tiling else L * L
    h00_off = (B * records * NW * 4 + 255) // 256 * 256
    out = torch.zeros(S * 4, dtype=torch.int64, device="cuda")
    h = R.rsos_init(p, dev_buf=base, dev_bytes=nbytes)
    try:
        for n_sweeps in (7, 13):
            R.rsos_sweep(h, n_sweeps)
            s1, s2, _, _ = R.rsos_width(h, S)
            out.fill_(-1)
            R.rsos_width_noalloc(p, base, base + h00_off, out.data_ptr())
            torch.cuda.synchronize()
            v = out.cpu().numpy().reshape(S, 4)
            assert _to128(v[:, 0], v[:, 1]) == [int(x) for x in s1]
            assert _to128(v[:, 2], v[:, 3]) == [int(x) for x in s2]
    finally:
        R.rsos_free(h)


def test_noalloc_rejects_what_it_cannot_hold():
    p = R.rsos_params(L=65536, N=4, surfaces=64, tile=8)
    with pytest.raises(R.RsosError) as e:
        R.rsos_width_noalloc(p, 256, 512, 1024)
    assert e.value.status == R.RSOS_ERANGE
    with pytest.raises(R.RsosError) as e:
        R.rsos_width_noalloc(R.rsos_params(L=64, N=1, surfaces=1), 256, 512, 1024)
    assert e.value.status == R.RSOS_EINVAL
