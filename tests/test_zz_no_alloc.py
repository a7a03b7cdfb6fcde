"""pic_bin_tiles_noalloc, the binning entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against pic_bin_tiles on the same input, twice in a
row (the fixed scratch keeps the previous call's contents, which must not leak
into the next result).  This file is collected last on purpose: when it fails
in a run that stops at the first failure, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, torch, nx, tile, cells):
    n = cells.shape[0]
    nt = int(np.prod([nx[d] // tile[d] for d in range(3)]))
    counts = torch.full((nt,), -7, dtype=torch.int32, device="cuda")
    start = torch.full((nt,), -7, dtype=torch.int64, device="cuda")
    perm = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    nxa = (C.c_int * 3)(*nx)
    ta = (C.c_int * 3)(*tile)
    code = lib.pic_bin_tiles_noalloc(nxa, ta, n, C.c_void_p(cells.data_ptr()), C.c_void_p(counts.data_ptr()),
                                     C.c_void_p(start.data_ptr()), C.c_void_p(perm.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, counts.cpu().numpy(), start.cpu().numpy(), perm[:n].cpu().numpy()


def test_noalloc_binning_matches_allocating_entry_point_twice():
    import torch
    import paper_1503_00276_gb300 as pg
    from paper_1503_00276_gb300 import _capi

    lib = _capi.load()
    rng = np.random.default_rng(42)
    cases = [((64, 32, 16), (8, 8, 4), 200003), ((48, 16, 1), (8, 4, 1), 77777), ((256, 128, 8), (2, 2, 2), 150001)]
    for nx, tile, n in cases:
        cells = np.stack([rng.integers(0, nx[d], n) for d in range(3)], axis=1).astype(np.int32)
        dev = torch.from_numpy(cells).cuda()
        ref_c, ref_s, ref_p = (t.cpu().numpy() for t in pg.bin_tiles(nx, tile, dev))
        for _ in range(2):  # two calls in a row share the fixed scratch
            code, cnt, st, perm = _call_noalloc(lib, torch, nx, tile, dev)
            assert code == 0, lib.pic_last_error()
            np.testing.assert_array_equal(cnt, ref_c)
            np.testing.assert_array_equal(st, ref_s)
            # both list the particles tile by tile in increasing index
            np.testing.assert_array_equal(perm, ref_p)
    # a request needing more than the fixed scratch is refused before any work
    big = torch.zeros((_capi.BIN_NOALLOC_SCRATCH_BYTES // 4 + 1024, 3), dtype=torch.int32, device="cuda")
    code, cnt, _, _ = _call_noalloc(lib, torch, (64, 32, 16), (8, 8, 4), big)
    assert code == -1 and b"fixed" in lib.pic_last_error()
    assert np.all(cnt == -7)
