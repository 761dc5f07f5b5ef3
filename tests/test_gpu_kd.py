"""The paper's grid rule (Sec. 7.1; Sec. 8: 100^3 voxels, binary trees of
depth <= 8, V_thr = 0.5) through the C ABI against the oracle.

Bit for bit: voxel of every photon, sort permutation, the trees (split axes,
split values, links), leaf table, leaf of every photon, active leaves and
histograms.  Guided sampling and evaluation on the grid: leaves bit for bit
and the plain sampling test's bounds.  At the paper's sizes (4M photons,
100^3 voxels, wall normals) the tree is checked node by node on a sample of
internal nodes against its own photons, and every photon is located by a
walk down its voxel's tree.
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


def _normals(kind, ph, seed):
    if kind == "wall":
        return synth.wall_normals(ph)
    if kind == "few":
        rng = np.random.default_rng(seed)
        return synth.uniform_sphere(rng, 6)[rng.integers(0, 6, ph.shape[0])].astype(np.float32)
    return None


def _build(ctx, ph, nrm, R, depth, thr, vthr=0.5, host=False):
    n = ph.shape[0]
    if host:
        return pg.pg_build_grid_kd(ctx, ph, nrm, n, LO, HI, R, depth, thr, vthr)
    d = torch.from_numpy(ph).cuda() if n else None
    dn = torch.from_numpy(nrm).cuda() if nrm is not None else None
    return pg.pg_build_grid_kd(ctx, d, dn, n, LO, HI, R, depth, thr, vthr)


CASES = [(200_000, 16, 8, 300, None, 51), (150_000, 10, 8, 2000, "wall", 52), (50_000, 4, 3, 50, "few", 53),
         (30_000, 1, 8, 100, "wall", 54), (0, 3, 8, 10, None, 55)]


@pytest.mark.parametrize("n,R,depth,thr,normals,seed", CASES)
def test_grid_bit_exact(ctx, n, R, depth, thr, normals, seed):
    ph = synth.photons(n, 12, seed)
    nrm = _normals(normals, ph, seed)
    g = _build(ctx, ph, nrm, R, depth, thr, host=(seed % 2 == 0))
    e = pg.export_kd(g)
    ref = O.build_kd_grid(ph, nrm, LO, HI, R, depth, thr, 0.5)
    assert e["L"] == ref["L"]
    assert np.array_equal(e["cells"].astype(np.int64), ref["cells"])
    for k in ("perm", "leaf_of", "leaf_depth", "leaf_begin", "leaf_end", "node_link"):
        assert np.array_equal(e[k], ref[k]), k
    assert np.array_equal(e["leaf_cell"].astype(np.int64), ref["leaf_cell"].astype(np.int64))
    internal = ref["node_link"] >= 0
    assert np.array_equal(e["node_axis"][internal], ref["node_axis"][internal])
    assert np.array_equal(e["node_tau"], ref["node_tau"])
    act, slot = O.active_leaves(ref)
    assert e["A"] == act.size
    assert np.array_equal(pg.export_grid(g)["slot_of_leaf"], slot)
    if n:
        h = pg.export_hist(pg.pg_splat_photons(ctx, g, torch.from_numpy(ph).cuda(), n, n // 2, 16, 16))
        hr = O.splat(ph, ref, n // 2, 16, 16)
        for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
            assert np.array_equal(h[k], hr[k][act]), k


def test_sample_eval_and_mis_on_the_grid(ctx):
    n, R, H, W = 120_000, 12, 32, 32
    ph = synth.photons(n, 12, 61)
    nrm = synth.wall_normals(ph)
    g = _build(ctx, ph, nrm, R, 8, 400)
    ref = O.build_kd_grid(ph, nrm, LO, HI, R, 8, 400, 0.5)
    act, slot = O.active_leaves(ref)
    A = act.size
    rng = np.random.default_rng(62)
    y = rng.lognormal(0, 2, (A, H, W)).astype(np.float32)
    y[1] = 0.0  # an invalid map
    t = pg.pg_build_cdf(ctx, pg.pg_map_import(ctx, torch.from_numpy(y).cuda(), A, H, W))
    tabs = O.tables_from_map(y.astype(np.float64))
    q = 60_000
    pos = synth.query_positions(q, 63)
    d_pos = torch.from_numpy(pos).cuda()
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    leaf = torch.empty(q, dtype=torch.int32, device="cuda")
    bins = torch.empty(q, dtype=torch.int32, device="cuda")
    pg.pg_sample_dirs(ctx, g, t, d_pos, q, 17, 2, dirs, pdf, leaf, bins)
    ctx.sync()
    s = O.sample(ref, slot, tabs, pos, 17, 2)
    assert np.array_equal(leaf.cpu().numpy().view(np.uint32), s["leaf"])
    same = bins.cpu().numpy().view(np.uint32) == s["bin"]
    assert same.mean() >= 1 - 1e-4
    err = np.abs(dirs.cpu().numpy().astype(np.float64) - s["dir"])
    stz = np.sqrt(np.maximum(1e-12, 1.0 - s["dir"][:, 2] ** 2))
    assert np.all(err[same, 2] <= 2.4e-7) and np.all(err[same, :2] <= (1e-6 + 2.4e-7 / stz[same])[:, None])
    ud = synth.query_directions(q, 64)
    out = torch.empty(q, device="cuda")
    pg.pg_eval_pdf(ctx, g, t, d_pos, torch.from_numpy(ud).cuda(), q, out)
    ctx.sync()
    er = O.eval_pdf(ref, slot, tabs, pos, ud)
    assert np.all(np.abs(out.cpu().numpy() - er) <= 1e-5 * er)
    # MIS statistics land in the leaves the tree walk finds.
    m = pg.pg_mis_create(ctx, g)
    strat = (rng.random(q) < 0.5).astype(np.uint8)
    contrib = rng.random(q).astype(np.float32)
    pg.pg_mis_accumulate(ctx, m, g, d_pos, torch.from_numpy(strat).cuda(), torch.from_numpy(contrib).cuda(), q)
    ctx.sync()
    lq, _ = O.kd_locate(ref, pos)
    st = O.mis_accumulate(ref["L"], lq, strat, contrib.astype(np.float64))
    em = pg.export_mis(m)
    assert np.array_equal(em["q_b"].astype(np.int64), st["q_b"]) and np.array_equal(em["q_g"].astype(np.int64),
                                                                                     st["q_g"])


def _node_ranges(e):
    """Photon range of every node, from the leaf ranges (children after parents)."""
    link = e["node_link"]
    N = link.size
    b = np.zeros(N, np.int64)
    en = np.zeros(N, np.int64)
    leaf = link < 0
    b[leaf] = e["leaf_begin"][~link[leaf]]
    en[leaf] = e["leaf_end"][~link[leaf]]
    for v in np.nonzero(~leaf)[0][::-1]:
        b[v] = b[link[v]]
        en[v] = en[link[v] + 1]
    return b, en


def test_paper_sizes_sampled(ctx):
    """4,194,304 photons, 100^3 voxels, depth 8, M_thr = 500, V_thr = 0.5."""
    n = 4_194_304
    ph = synth.photons(n, 64, synth.SCALE.seed)
    nrm = synth.wall_normals(ph)
    g = _build(ctx, ph, nrm, 100, 8, 500)
    e = pg.export_kd(g)
    L = e["L"]
    assert e["leaf_begin"][0] == 0 and e["leaf_end"][-1] == n
    assert np.array_equal(e["leaf_begin"][1:], e["leaf_end"][:-1])
    # Every photon is found in its leaf by a walk down its voxel's tree.
    dl = torch.empty(n, dtype=torch.int32, device="cuda")
    dd, dp = torch.empty(n, 3, device="cuda"), torch.empty(n, device="cuda")
    A = e["A"]
    t = pg.pg_build_cdf(ctx, pg.pg_map_import(ctx, torch.ones(A, 4, 4, device="cuda"), A, 4, 4))
    pg.pg_sample_dirs(ctx, g, t, torch.from_numpy(np.ascontiguousarray(ph[:, :3])).cuda(), n, 1, 0, dd, dp, dl)
    ctx.sync()
    assert np.array_equal(dl.cpu().numpy().view(np.uint32) & 0x7FFFFFFF, e["leaf_of"])
    # The split rule on a sample of internal nodes, recomputed from their photons.
    b, en = _node_ranges(e)
    cells_n = 100 ** 3
    internal = np.nonzero(e["node_link"] >= 0)[0]
    assert internal.size > 100
    rng = np.random.default_rng(7)
    u = 2 ** O.KD_NORMAL_BITS
    for v in rng.choice(internal, 200, replace=False):
        idx = e["perm"][b[v]:en[v]]
        P = ph[idx, :3]
        m = idx.size
        spread = P.max(axis=0) - P.min(axis=0)
        a = int(e["node_axis"][v])
        assert spread[a] == spread.max() and np.all(spread[:a] < spread[a])
        V = O.kd_normal_variance(np.rint(nrm[idx].astype(np.float64) * u).astype(np.int64).sum(axis=0).tolist(), m)
        assert m > 500 or V > 0.5
        x = np.sort(P[:, a])
        s = x[m // 2]
        tau = e["node_tau"][v]
        assert tau == (s if x[0] < s else np.nextafter(s, np.float32(np.inf)))
        nl = int((P[:, a] < tau).sum())
        assert b[e["node_link"][v]] == b[v] and en[e["node_link"][v]] == b[v] + nl
    # Leaves that could still split are at the depth limit.
    cnt = (e["leaf_end"] - e["leaf_begin"]).astype(np.int64)
    big = np.nonzero(cnt > 500)[0]
    for l in big[:200]:
        idx = e["perm"][e["leaf_begin"][l]:e["leaf_end"][l]]
        P = ph[idx, :3]
        assert e["leaf_depth"][l] == 8 or (P.max(axis=0) - P.min(axis=0)).max() == 0
    assert L >= cells_n


def test_errors(ctx):
    ph = synth.photons(1000, 2, 71)
    bad = ph.copy()
    bad[5, 2] = np.inf
    with pytest.raises(pg.PgError) as ei:
        _build(ctx, bad, None, 8, 8, 10)
    assert ei.value.status == 8
    nrm = synth.wall_normals(ph)
    nrm[3, 0] = 2.0
    with pytest.raises(pg.PgError) as ei:
        _build(ctx, ph, nrm, 8, 8, 10)
    assert ei.value.status == 8
    with pytest.raises(pg.PgError) as ei:
        _build(ctx, ph, None, 600, 8, 10)
    assert ei.value.status == 1
    with pytest.raises(pg.PgError) as ei:
        _build(ctx, ph, None, 8, 17, 10)
    assert ei.value.status == 1
    g = _build(ctx, ph, None, 8, 8, 10)
    with pytest.raises(pg.PgError) as ei:
        pg.pg_splat_photons_batched(ctx, g, torch.from_numpy(ph).cuda(), 1000, np.zeros(1, np.uint32), 8, 8)
    assert ei.value.status == 9
