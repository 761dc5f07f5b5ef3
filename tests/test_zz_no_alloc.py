"""The allocation-free entry point against the allocating one.

pg_sort_photons_noalloc is for callers that cannot allocate device memory
(their host application owns every allocation, or they must not block on the
driver's allocator).  Its scratch is a static device array inside libpg.so.
Through the C ABI it must produce the same Morton codes and sort permutation
as pg_build_grid, on two calls in a row (the second call reuses the scratch
the first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LO, HI = [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]


def _reference(ctx, d_ph, n, D):
    g = pg.pg_build_grid(ctx, d_ph, n, LO, HI, D, 0, 1000)
    out = pg.export_grid(g)
    g.free()
    return out["codes"], out["perm"]


def test_noalloc_sort_matches_build_grid_twice():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ctx = pg.Context()
    stream = torch.cuda.current_stream().cuda_stream
    # Different inputs in a row: a large one (several sort tiles, ragged
    # tail, 4 radix passes), a smaller one with a different depth (3
    # passes), an empty call, and depth 16 at the size limit (48-bit codes,
    # 6 passes: the largest use of the scratch), so stale scratch from one
    # call would show up in the next.
    for n, D, seed in [(300_001, 10, 901), (77_777, 6, 902), (0, 10, 903), (pg.PG_NOALLOC_MAX_PHOTONS, 16, 904)]:
        if n == 0:
            pg.pg_sort_photons_noalloc(0, 0, LO, HI, D, 0, 0, stream)  # nothing to do, no pointers needed
            continue
        ph = synth.photons(n, 7, seed)
        d_ph = torch.from_numpy(ph).cuda()
        codes = torch.empty(n, dtype=torch.int64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        pg.pg_sort_photons_noalloc(d_ph, n, LO, HI, D, codes, perm, stream)
        torch.cuda.synchronize()
        ref_codes, ref_perm = _reference(ctx, d_ph, n, D)
        assert np.array_equal(codes.cpu().numpy().view(np.uint64), ref_codes)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), ref_perm)
    # Beyond the stated maximum: a clear error, nothing launched.
    with pytest.raises(pg.PgError) as e:
        pg.pg_sort_photons_noalloc(0, pg.PG_NOALLOC_MAX_PHOTONS + 1, LO, HI, 10, 0, 0, stream)
    assert e.value.status == 9
    ctx.destroy()
