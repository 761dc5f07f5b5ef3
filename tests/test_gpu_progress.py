"""Progressive iterations (Sec. 7.1, 7.2; Algorithm 1) through the C ABI
against the oracle's Progressive form.

After every iteration: the leaf table, the updated-leaf list and the
leaf-indexed energy and count planes (current and previous) bit for bit;
after every reconstruct: the maps of the updated leaves at the FP32 CNN gate,
every other leaf's map unchanged bit for bit, validity flags exact; sampling
through the state's grid and tables: leaves exact and bins as in the plain
sampling test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LO = [0.0, 0.0, 0.0]
HI = [1.0, 1.0, 1.0]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = pg.Context()
    yield c
    c.destroy()


def _batches(first, iters, seed):
    """Doubling batches (Sec. 7.2: 2^t N_p photons in iteration t)."""
    sizes = [first << t for t in range(iters)]
    ph = synth.photons(sum(sizes), 12, seed)
    ends = np.cumsum(sizes)
    return [ph[e - n:e] for n, e in zip(sizes, ends)]


def _check_fp32_maps(y, yr):
    """The FP32 CNN gate of the single-shot path (see tests/test_gpu_parity.py)."""
    P = y.reshape(len(y), -1).astype(np.float64)
    Pr = yr.reshape(len(yr), -1)
    P = P / P.sum(axis=1, keepdims=True)
    Pr = Pr / Pr.sum(axis=1, keepdims=True)
    assert np.all(np.abs(P - Pr) <= 1e-5 * Pr + 1e-7 * Pr.max(axis=1, keepdims=True))


@pytest.mark.parametrize("refine,c,D,min_depth,H,W,first,iters,rule,R", [
    (2, 300.0, 5, 1, 16, 16, 20_000, 4, 0, 0),
    (1, 500.0, 4, 0, 32, 32, 30_000, 3, 0, 0),
    (0, 500.0, 6, 2, 8, 16, 25_000, 3, 0, 0),
    (2, 200.0, 6, 0, 16, 16, 20_000, 4, 1, 6),   # the paper's rule: 6^3 voxels, trees of depth 6
    (0, 500.0, 8, 0, 8, 16, 20_000, 3, 1, 5),
])
def test_iterations_match_oracle(ctx, refine, c, D, min_depth, H, W, first, iters, rule, R):
    batches = _batches(first, iters, 700 + refine + 10 * rule)
    normals = [synth.wall_normals(b) for b in batches] if rule else [None] * iters
    total = sum(len(b) for b in batches)
    st = pg.pg_progress_create(ctx, LO, HI, D, min_depth, H, W, total, split_c=c, refine_iterations=refine,
                               grid_rule=rule, resolution=R or 100)
    pr = O.Progressive(LO, HI, D, min_depth, H, W, total, split_c=c, refine_iterations=refine,
                       grid_rule="kd" if rule else "octree", R=R)
    blob = synth.net_blob(synth.ARCH_TINY3, (16,), 710)
    net = pg.pg_net_load(ctx, blob)
    onet = O.parse_net(blob)
    prev_maps = None
    for t, (b, nb) in enumerate(zip(batches, normals)):
        # Odd iterations pass the batch from host memory.
        src = b if t % 2 else torch.from_numpy(b).cuda()
        pg.pg_progress_add_photons(ctx, st, src, len(b), nb)
        pr.add_photons(b, nb)
        ctx.sync()
        assert pr.status == 0
        assert st.info(pg.PG_INFO_ITERATION) == t + 1 and st.info(pg.PG_INFO_N_PHOTONS) == sum(map(len, batches[:t + 1]))
        g, h, m, _ = pg.pg_progress_view(st)
        eg = pg.export_grid(g)
        assert eg["L"] == pr.grid["L"]
        if rule:
            ek = pg.export_kd(g)
            assert np.array_equal(ek["node_link"], pr.grid["node_link"])
            assert np.array_equal(ek["leaf_cell"].astype(np.int64), pr.grid["leaf_cell"].astype(np.int64))
        else:
            assert np.array_equal(eg["leaf_code"], pr.grid["leaf_code"])
        assert np.array_equal(eg["leaf_depth"], pr.grid["leaf_depth"])
        # Map slots: refined leaves in leaf order, later newcomers appended.
        A = len(pr.slot_leaf)
        assert eg["A"] == A and np.array_equal(eg["active"][:A].astype(np.int64), np.array(pr.slot_leaf, np.int64))
        assert np.array_equal(eg["slot_of_leaf"].astype(np.int64), pr.slot_of_leaf)
        upd = pg.export_progress_updated(st).astype(np.int64)
        assert np.array_equal(upd, pr.updated_slots)
        eh = pg.export_hist(h)
        rows = np.array(pr.slot_leaf, np.int64)
        for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
            assert np.array_equal(eh[k], getattr(pr, k)[rows]), (t, k)

        pg.pg_progress_reconstruct(ctx, st, net, pg.PG_FP32)
        ctx.sync()
        _, _, m, tab = pg.pg_progress_view(st)
        tables = pr.reconstruct(onet)
        y = pg.export_map(m)
        assert y.shape[0] == A
        if len(upd):
            _check_fp32_maps(y[upd], pr.maps[rows[upd]])
        if t >= refine and prev_maps is not None:  # slots not updated keep their maps
            other = np.setdiff1d(np.arange(prev_maps.shape[0]), upd)
            assert np.array_equal(y[other], prev_maps[other])
        prev_maps = y
        et = pg.export_tables(tab)
        assert np.array_equal(et["valid"], tables["valid"][rows])

    # Guided sampling through the state's grid and tables (the oracle's tables
    # are leaf-indexed; leaves without a slot fall back on both sides).
    q = 50_000
    pos = synth.query_positions(q, 720)
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    leaf = torch.empty(q, dtype=torch.int32, device="cuda")
    bins = torch.empty(q, dtype=torch.int32, device="cuda")
    g, _, _, tab = pg.pg_progress_view(st)
    pg.pg_sample_dirs(ctx, g, tab, torch.from_numpy(pos).cuda(), q, 99, 0, dirs, pdf, leaf, bins)
    ctx.sync()
    s = O.sample(pr.grid, np.arange(pr.grid["L"], dtype=np.int32), tables, pos, 99, 0)
    assert np.array_equal(leaf.cpu().numpy().view(np.uint32), s["leaf"])
    assert (bins.cpu().numpy().view(np.uint32) == s["bin"]).mean() >= 1 - 1e-3
    st.free()


def test_errors_and_borrowed_handles(ctx):
    b = _batches(5_000, 3, 730)
    st = pg.pg_progress_create(ctx, LO, HI, 4, 1, 8, 8, 20_000, split_c=100.0, refine_iterations=1)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_TINY3, (16,), 731))
    with pytest.raises(pg.PgError) as e:  # no grid before the first refining iteration
        pg.pg_progress_reconstruct(ctx, st, net, pg.PG_FP32)
    assert e.value.status == 1
    # The paper's rule: normals with every refining batch or with none.
    kst = pg.pg_progress_create(ctx, LO, HI, 6, 0, 8, 8, 20_000, split_c=100.0, refine_iterations=2, grid_rule=1,
                                resolution=4)
    pg.pg_progress_add_photons(ctx, kst, torch.from_numpy(b[0]).cuda(), len(b[0]),
                               torch.from_numpy(synth.wall_normals(b[0])).cuda())
    with pytest.raises(pg.PgError) as e:
        pg.pg_progress_add_photons(ctx, kst, torch.from_numpy(b[1]).cuda(), len(b[1]))
    assert e.value.status == 1
    kst.free()
    pg.pg_progress_add_photons(ctx, st, torch.from_numpy(b[0]).cuda(), len(b[0]))
    g, h, m, tab = pg.pg_progress_view(st)
    assert tab is None
    # pg_free leaves borrowed handles alone.
    pg._lib.pg_free(g.ptr)
    assert pg.export_grid(g)["A"] == pg.export_hist(h)["pow_cur"].shape[0]
    # The photon total is bounded by max_photons.
    with pytest.raises(pg.PgError) as e:
        pg.pg_progress_add_photons(ctx, st, torch.from_numpy(b[2]).cuda(), 16_000)
    assert e.value.status == 1
    # A non-finite position in a binned batch is reported and changes nothing.
    before = pg.export_hist(h)["cnt_cur"].sum()
    bad = b[1].copy()
    bad[17, 0] = np.nan
    with pytest.raises(pg.PgError) as e:
        pg.pg_progress_add_photons(ctx, st, torch.from_numpy(bad).cuda(), len(bad))
    assert e.value.status == 8
    assert st.info(pg.PG_INFO_ITERATION) == 1 and pg.export_hist(h)["cnt_cur"].sum() == before
    # A power above (2^63 - 1) / max_photons in fixed point overflows.
    big = b[1].copy()
    big[3, 6] = 1.0e6  # 2^32 * 1e6 > (2^63 - 1) / 20000
    pg.pg_progress_add_photons(ctx, st, torch.from_numpy(big).cuda(), len(big))
    with pytest.raises(pg.PgError) as e:
        ctx.sync()
    assert e.value.status == 4
    st.free()
