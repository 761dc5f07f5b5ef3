"""Scene batches: every scene of a batched call matches the same scene alone.

Each scene's grid, histograms, BF16 maps and guided samples inside a batch
are compared bit for bit with the scene processed on its own, and two of the
scenes inside the batch are compared with the FP64 oracle directly (grid,
histograms and sampling bit for bit, pdfs within the FP32 bound).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

D, THR, H, W = 6, 300, 32, 32


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = pg.Context()
    yield c
    c.destroy()


def _scenes():
    sizes = [20_000, 0, 517, 9_001, 3]
    los = [[0, 0, 0], [-1, -1, -1], [0.25, 0.1, 0.0], [-2.0, 0.0, 1.0], [0, 0, 0]]
    his = [[1, 1, 1], [1, 1, 1], [1.25, 1.1, 1.0], [2.0, 3.0, 3.0], [1, 1, 1]]
    phs = []
    for s, n in enumerate(sizes):
        ph = synth.photons(n, 3, 500 + s)
        lo, hi = np.array(los[s], np.float32), np.array(his[s], np.float32)
        ph[:, :3] = lo + ph[:, :3] * (hi - lo)
        phs.append(ph)
    return sizes, los, his, phs


def test_batched_grid_hist_maps_and_samples_match_single_scenes(ctx):
    sizes, los, his, phs = _scenes()
    S = len(sizes)
    begin = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    n = int(begin[-1])
    allph = np.ascontiguousarray(np.concatenate(phs))
    d_all = torch.from_numpy(allph).cuda()
    gb = pg.pg_build_grid_batched(ctx, d_all, n, begin, los, his, D, 0, THR)
    SL = gb.info(pg.PG_INFO_SCENE_LEVELS)
    assert gb.info(pg.PG_INFO_N_SCENES) == S and SL == 1
    B = pg.export_grid(gb)
    n_prev = np.array([sz // 2 for sz in sizes], np.uint32)
    hb = pg.pg_splat_photons_batched(ctx, gb, d_all, n, n_prev, H, W)
    HB = pg.export_hist(hb)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_TINY3, (16,), 601))
    mb = pg.pg_reconstruct(ctx, hb, net, pg.PG_BF16)
    tb = pg.pg_build_cdf(ctx, mb)
    YB = pg.export_map(mb)
    # Queries: scene-grouped, scene s gets its own Philox stream id.
    qs = [4096, 7, 0, 1000, 33]
    qbeg = np.concatenate([[0], np.cumsum(qs)]).astype(np.uint32)
    pos = []
    for s, q in enumerate(qs):
        p = synth.query_positions(q, 700 + s)
        lo, hi = np.array(los[s], np.float32), np.array(his[s], np.float32)
        pos.append((lo + p * (hi - lo)).astype(np.float32))
    pos_all = np.ascontiguousarray(np.concatenate(pos))
    streams = np.array([11, 22, 33, 44, 55], np.uint32)
    Q = int(qbeg[-1])
    dirs = torch.empty(Q, 3, device="cuda")
    pdf = torch.empty(Q, device="cuda")
    leaf = torch.empty(Q, dtype=torch.int32, device="cuda")
    bins = torch.empty(Q, dtype=torch.int32, device="cuda")
    pg.pg_sample_dirs_batched(ctx, gb, tb, torch.from_numpy(pos_all).cuda(), qbeg, Q, 99, streams, dirs, pdf, leaf, bins)
    ev = torch.empty(Q, device="cuda")
    pg.pg_eval_pdf_batched(ctx, gb, tb, torch.from_numpy(pos_all).cuda(), dirs, qbeg, Q, ev)
    ctx.sync()
    dirs, pdf, leaf, bins, ev = (dirs.cpu().numpy(), pdf.cpu().numpy(), leaf.cpu().numpy().view(np.uint32),
                                 bins.cpu().numpy().view(np.uint32), ev.cpu().numpy())

    shift = 3 * D
    mask = (1 << shift) - 1
    leaf0 = act0 = 0
    scene_leaf0 = []
    for s in range(S):
        scene_leaf0.append(leaf0)
        gs = pg.pg_build_grid(ctx, torch.from_numpy(phs[s]).cuda() if sizes[s] else 0, sizes[s], los[s], his[s],
                              D, 0, THR)
        G = pg.export_grid(gs)
        L = G["L"]
        sel = slice(leaf0, leaf0 + L)
        assert np.all((B["leaf_code"][sel] >> np.uint64(shift)) == s)
        assert np.array_equal(B["leaf_code"][sel] & np.uint64(mask), G["leaf_code"])
        assert np.array_equal(B["leaf_depth"][sel] - SL, G["leaf_depth"])
        assert np.array_equal(B["leaf_begin"][sel] - begin[s], G["leaf_begin"])
        assert np.array_equal(B["leaf_end"][sel] - begin[s], G["leaf_end"])
        assert np.array_equal(B["perm"][begin[s]:begin[s + 1]] - begin[s], G["perm"])
        assert np.array_equal(B["leaf_of"][begin[s]:begin[s + 1]] - leaf0, G["leaf_of"])
        A = G["A"]
        hs = pg.pg_splat_photons(ctx, gs, torch.from_numpy(phs[s]).cuda() if sizes[s] else 0, sizes[s],
                                 int(n_prev[s]), H, W)
        HS = pg.export_hist(hs)
        for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
            assert np.array_equal(HB[k][act0:act0 + A], HS[k]), k
        if A:
            ms = pg.pg_reconstruct(ctx, hs, net, pg.PG_BF16)
            assert np.array_equal(YB[act0:act0 + A], pg.export_map(ms))
            ts = pg.pg_build_cdf(ctx, ms)
        if qs[s] and A:
            q = qs[s]
            d2 = torch.empty(q, 3, device="cuda")
            p2 = torch.empty(q, device="cuda")
            l2 = torch.empty(q, dtype=torch.int32, device="cuda")
            b2 = torch.empty(q, dtype=torch.int32, device="cuda")
            pg.pg_sample_dirs(ctx, gs, ts, torch.from_numpy(pos[s]).cuda(), q, 99, int(streams[s]), d2, p2, l2, b2)
            e2 = torch.empty(q, device="cuda")
            pg.pg_eval_pdf(ctx, gs, ts, torch.from_numpy(pos[s]).cuda(), d2, q, e2)
            ctx.sync()
            r = slice(qbeg[s], qbeg[s + 1])
            assert np.array_equal(dirs[r], d2.cpu().numpy())
            assert np.array_equal(pdf[r], p2.cpu().numpy())
            assert np.array_equal(bins[r], b2.cpu().numpy().view(np.uint32))
            lb, ls = leaf[r], l2.cpu().numpy().view(np.uint32)
            assert np.array_equal(lb >> 31, ls >> 31)
            assert np.array_equal((lb & 0x7FFFFFFF) - leaf0, ls & 0x7FFFFFFF)
            assert np.array_equal(ev[r], e2.cpu().numpy())
        leaf0 += L
        act0 += A
    # Scene slots beyond S (8^SL > S) hold single empty leaves at the end.
    assert B["L"] == leaf0 + (8 ** SL - S)
    lb = gb.export(pg.PG_GRID_SCENE_LEAF_BEGIN, np.uint32, S + 1)
    assert lb.tolist() == scene_leaf0 + [leaf0]
    assert B["A"] == act0


def test_batched_scenes_against_the_oracle(ctx):
    """Scenes 0 and 3 of the batch (20,000 and 9,001 photons, different
    domains) against the oracle run on each scene alone: the scene's leaves,
    permutation and leaf assignment, all four histogram planes, and the guided
    samples and pdf evaluations of the scene's queries on the batch's own
    maps (bins identical for >= 1 - 1e-4 of the queries, FP32 pdfs within
    1e-5 relative above FP32's normal range)."""
    sizes, los, his, phs = _scenes()
    S = len(sizes)
    begin = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    n = int(begin[-1])
    d_all = torch.from_numpy(np.ascontiguousarray(np.concatenate(phs))).cuda()
    gb = pg.pg_build_grid_batched(ctx, d_all, n, begin, los, his, D, 0, THR)
    SL = gb.info(pg.PG_INFO_SCENE_LEVELS)
    B = pg.export_grid(gb)
    n_prev = np.array([sz // 2 for sz in sizes], np.uint32)
    hb = pg.pg_splat_photons_batched(ctx, gb, d_all, n, n_prev, H, W)
    HB = pg.export_hist(hb)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_TINY3, (16,), 602))
    mb = pg.pg_reconstruct(ctx, hb, net, pg.PG_BF16)
    tb = pg.pg_build_cdf(ctx, mb)
    YB = pg.export_map(mb).astype(np.float64)
    qs = [3000, 0, 0, 2000, 0]
    qbeg = np.concatenate([[0], np.cumsum(qs)]).astype(np.uint32)
    pos = []
    for s_, q in enumerate(qs):
        p = synth.query_positions(q, 710 + s_)
        lo, hi = np.array(los[s_], np.float32), np.array(his[s_], np.float32)
        pos.append((lo + p * (hi - lo)).astype(np.float32))
    pos_all = np.ascontiguousarray(np.concatenate(pos))
    streams = np.array([5, 6, 7, 8, 9], np.uint32)
    Q = int(qbeg[-1])
    dirs = torch.empty(Q, 3, device="cuda")
    pdf = torch.empty(Q, device="cuda")
    leaf = torch.empty(Q, dtype=torch.int32, device="cuda")
    bins = torch.empty(Q, dtype=torch.int32, device="cuda")
    d_pos = torch.from_numpy(pos_all).cuda()
    pg.pg_sample_dirs_batched(ctx, gb, tb, d_pos, qbeg, Q, 77, streams, dirs, pdf, leaf, bins)
    ev_dirs = np.ascontiguousarray(np.concatenate([synth.query_directions(q, 720 + s_) for s_, q in enumerate(qs)]))
    ev = torch.empty(Q, device="cuda")
    pg.pg_eval_pdf_batched(ctx, gb, tb, d_pos, torch.from_numpy(ev_dirs).cuda(), qbeg, Q, ev)
    ctx.sync()
    dirs, pdf, leaf, bins, ev = (dirs.cpu().numpy(), pdf.cpu().numpy(), leaf.cpu().numpy().view(np.uint32),
                                 bins.cpu().numpy().view(np.uint32), ev.cpu().numpy().astype(np.float64))
    shift = np.uint64(3 * D)
    scene_of_leaf = (B["leaf_code"] >> shift).astype(np.int64)
    active = np.zeros(B["L"], bool)
    active[B["active"]] = True
    for s_ in (0, 3):
        ref = O.build_grid(phs[s_], los[s_], his[s_], D, 0, THR)
        leaf0 = int(np.argmax(scene_of_leaf == s_))
        L = ref["L"]
        sel = slice(leaf0, leaf0 + L)
        assert np.all(scene_of_leaf[sel] == s_)
        assert np.array_equal(B["leaf_code"][sel] & np.uint64((1 << (3 * D)) - 1), ref["leaf_code"])
        assert np.array_equal(B["leaf_depth"][sel] - SL, ref["leaf_depth"])
        assert np.array_equal(B["leaf_begin"][sel] - begin[s_], ref["leaf_begin"])
        assert np.array_equal(B["leaf_end"][sel] - begin[s_], ref["leaf_end"])
        assert np.array_equal(B["perm"][begin[s_]:begin[s_ + 1]] - begin[s_], ref["perm"])
        assert np.array_equal(B["leaf_of"][begin[s_]:begin[s_ + 1]] - leaf0, ref["leaf_of"])
        act, slot = O.active_leaves(ref)
        act0 = int(active[:leaf0].sum())
        A = act.size
        assert np.array_equal(np.nonzero(active[sel])[0], act)
        h = O.hist_for_active(O.splat(phs[s_], ref, int(n_prev[s_]), H, W), act)
        for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
            assert np.array_equal(HB[k][act0:act0 + A], h[k]), (s_, k)
        # Sampling and evaluation of the scene's queries on the batch's maps.
        tabs = O.tables_from_map(YB[act0:act0 + A])
        r = slice(qbeg[s_], qbeg[s_ + 1])
        o = O.sample(ref, slot, tabs, pos[s_], 77, int(streams[s_]))
        lb = leaf[r]
        assert np.array_equal(lb >> 31, o["leaf"] >> 31)
        assert np.array_equal((lb & 0x7FFFFFFF) - leaf0, o["leaf"] & 0x7FFFFFFF)
        same = bins[r] == o["bin"]
        assert same.mean() >= 1 - 1e-4
        # FP32 pdfs within 1e-5 relative; maps of this random net reach P below
        # FP32's normal range (1.2e-38) on some bins, where an FP32 value keeps
        # only its absolute spacing, hence the 1e-35 floor (HW / 4 pi = 81.5).
        nz = same & (o["pdf"] > 0)
        assert np.all(np.abs(pdf[r][nz] - o["pdf"][nz]) <= 1e-5 * o["pdf"][nz] + 1e-35)
        e = O.eval_pdf(ref, slot, tabs, pos[s_], ev_dirs[r])
        assert np.all(np.abs(ev[r] - e) <= 1e-5 * e + 1e-35)
    for hd in (tb, mb, hb, gb, net):
        hd.free()


def test_batched_argument_checks(ctx):
    ph = synth.photons(100, 1, 9)
    d = torch.from_numpy(ph).cuda()
    with pytest.raises(pg.PgError) as e:  # offsets must end at n
        pg.pg_build_grid_batched(ctx, d, 100, np.array([0, 50, 99], np.uint32), [[0, 0, 0]] * 2, [[1, 1, 1]] * 2,
                                 4, 0, 10)
    assert e.value.status == 1
    with pytest.raises(pg.PgError) as e:  # depth must be shared
        pg.pg_build_grid_batched(ctx, d, 100, np.array([0, 50, 100], np.uint32), [[0, 0, 0]] * 2, [[1, 1, 1]] * 2,
                                 17, 0, 10)
    assert e.value.status in (1, 9)


def test_batched_overflow_bound_is_per_scene(ctx):
    # Two one-photon scenes of power 2^30: 2^62 in fixed point each, within
    # (2^63-1)/1 for each scene alone, over (2^63-1)/2 for the two together.
    ph = synth.photons(2, 1, 5)
    ph[:, 6] = 2.0 ** 30
    d = torch.from_numpy(ph).cuda()
    begin = np.array([0, 1, 2], np.uint32)
    g = pg.pg_build_grid_batched(ctx, d, 2, begin, [[0, 0, 0]] * 2, [[1, 1, 1]] * 2, 3, 0, 10)
    h = pg.pg_splat_photons_batched(ctx, g, d, 2, np.zeros(2, np.uint32), 8, 8, 32)
    ctx.sync()
    hb = pg.export_hist(h)
    assert hb["pow_cur"].sum(axis=1).tolist() == [1 << 62, 1 << 62]
    g1 = pg.pg_build_grid(ctx, d, 2, [0, 0, 0], [1, 1, 1], 3, 0, 10)
    pg.pg_splat_photons(ctx, g1, d, 2, 0, 8, 8, 32)
    with pytest.raises(pg.PgError) as e:
        ctx.sync()
    assert e.value.status == 4
