"""One-sample MIS of BSDF and guide (Sec. 7.3, Eq. target_mis, mis_alpha,
mis_coef) through the C ABI against the FP64 oracle.

Statistics: counts bit for bit, FP64 sums to summation-order rounding, alpha
to one FP32 ulp (the kernel rounds its FP64 ratio once).  Sampling: the
strategy decision is the same FP32 comparison of the selection uniform with
alpha on both sides, so strategies match exactly wherever the two alphas
agree; guided directions are bit for bit pg_sample_dirs' and within the
sampling test's bounds of the oracle; Lambertian directions within 2e-6
(an FP32 frame, square roots and sincos, each a few ulps of a unit
vector); pdfs within 1e-5 relative plus 1e-6 absolute (the FP32 dot
product n.w near grazing angles).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LO = [0.0, 0.0, 0.0]
HI = [1.0, 1.0, 1.0]
H, W = 32, 32


@pytest.fixture(scope="module")
def scene():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ctx = pg.Context()
    wl = synth.TINY
    ph = synth.photons(wl.n_photons, wl.n_blobs, wl.seed)
    g = pg.pg_build_grid(ctx, torch.from_numpy(ph).cuda(), wl.n_photons, LO, HI, wl.max_depth, 0,
                         wl.split_threshold)
    ref = O.build_grid(ph, LO, HI, wl.max_depth, 0, wl.split_threshold)
    act, slot = O.active_leaves(ref)
    A = g.info(pg.PG_INFO_N_ACTIVE)
    rng = np.random.default_rng(41)
    y = rng.lognormal(0, 2, (A, H, W)).astype(np.float32)
    y[3] = 0.0  # an invalid map: its leaf samples the BSDF alone
    t = pg.pg_build_cdf(ctx, pg.pg_map_import(ctx, torch.from_numpy(y).cuda(), A, H, W))
    tabs = O.tables_from_map(y.astype(np.float64))
    yield dict(ctx=ctx, g=g, ref=ref, slot=slot, t=t, tabs=tabs)
    ctx.destroy()


def _bounce_records(q, seed):
    """Synthetic path-vertex records: positions, the strategy that sampled the
    bounce and its contribution; the guide's share grows along x so that
    alpha crosses both clamps across the scene."""
    pos = synth.query_positions(q, seed)
    rng = np.random.default_rng(seed)
    strat = (rng.random(q) < 0.5).astype(np.uint8)
    c = rng.lognormal(0.0, 1.0, q)
    c = np.where(strat == 1, c * (0.05 + 8.0 * pos[:, 0] ** 2), c).astype(np.float32)
    return pos, strat, c


def _accumulate(ctx, g, m, pos, strat, c):
    q = pos.shape[0]
    pg.pg_mis_accumulate(ctx, m, g, torch.from_numpy(pos).cuda(), torch.from_numpy(strat).cuda(),
                         torch.from_numpy(c).cuda(), q)


@pytest.fixture(scope="module")
def trained(scene):
    ctx, g, ref = scene["ctx"], scene["g"], scene["ref"]
    m = pg.pg_mis_create(ctx, g)
    e0 = pg.export_mis(m)
    assert np.all(e0["alpha"] == 0.5) and not e0["q_b"].any() and not e0["nu_g"].any()
    recs = [_bounce_records(300_000, 51), _bounce_records(123_457, 52)]
    for r in recs:
        _accumulate(ctx, g, m, *r)
    pg.pg_mis_update(ctx, m)
    ctx.sync()
    pos = np.concatenate([r[0] for r in recs])
    strat = np.concatenate([r[1] for r in recs])
    c = np.concatenate([r[2] for r in recs])
    leaf, _ = O.leaf_of_positions(ref, pos)
    st = O.mis_accumulate(ref["L"], leaf, strat, c.astype(np.float64))
    alpha = O.mis_alpha(st, np.full(ref["L"], 0.5))
    return m, st, alpha


def test_statistics_and_alpha(scene, trained):
    m, st, alpha = trained
    e = pg.export_mis(m)
    assert np.array_equal(e["q_b"].astype(np.int64), st["q_b"])
    assert np.array_equal(e["q_g"].astype(np.int64), st["q_g"])
    assert np.allclose(e["nu_b"], st["nu_b"], rtol=1e-12, atol=0)
    assert np.allclose(e["nu_g"], st["nu_g"], rtol=1e-12, atol=0)
    a32 = alpha.astype(np.float32)
    ulp = np.spacing(a32)
    assert np.all(np.abs(e["alpha"] - a32) <= ulp)
    # The workload exercises every branch of the rule.
    upd = (st["q_b"] >= 50) & (st["q_g"] >= 50)
    assert (~upd).any() and np.any(alpha[upd] == 0.2) and np.any(alpha[upd] == 0.8)
    assert np.any((alpha[upd] > 0.2) & (alpha[upd] < 0.8))


def test_update_parameters(scene):
    ctx, g, ref = scene["ctx"], scene["g"], scene["ref"]
    m = pg.pg_mis_create(ctx, g)
    r = _bounce_records(50_000, 53)
    _accumulate(ctx, g, m, *r)
    pg.pg_mis_update(ctx, m, min_count=3, alpha_lo=0.0, alpha_hi=1.0)
    e = pg.export_mis(m)
    leaf, _ = O.leaf_of_positions(ref, r[0])
    st = O.mis_accumulate(ref["L"], leaf, r[1], r[2].astype(np.float64))
    a = O.mis_alpha(st, np.full(ref["L"], 0.5), min_count=3, lo=0.0, hi=1.0).astype(np.float32)
    assert np.all(np.abs(e["alpha"] - a) <= np.spacing(a))
    for bad in ((0.5, 0.4), (-0.1, 0.8), (0.2, 1.5)):
        with pytest.raises(pg.PgError) as ei:
            pg.pg_mis_update(ctx, m, 50, *bad)
        assert ei.value.status == 1


@pytest.mark.parametrize("q,seed,stream_id", [(200_003, 61, 0), (4_097, 2 ** 40 + 3, 5), (1, 9, 2)])
def test_sample_and_eval(scene, trained, q, seed, stream_id):
    ctx, g, t, ref, slot, tabs = (scene[k] for k in ("ctx", "g", "t", "ref", "slot", "tabs"))
    m, _, alpha = trained
    a_kernel = pg.export_mis(m)["alpha"]
    a32 = alpha.astype(np.float32)
    pos = synth.query_positions(q, seed & 0xFFFF)
    nrm = synth.query_directions(q, (seed + 1) & 0xFFFF)
    d_pos, d_n = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    strat = torch.empty(q, dtype=torch.uint8, device="cuda")
    pg.pg_mis_sample(ctx, g, t, m, d_pos, d_n, q, seed, stream_id, dirs, pdf, strat)
    gd = torch.empty(q, 3, device="cuda")
    gp = torch.empty(q, device="cuda")
    gl = torch.empty(q, dtype=torch.int32, device="cuda")
    gb = torch.empty(q, dtype=torch.int32, device="cuda")
    pg.pg_sample_dirs(ctx, g, t, d_pos, q, seed, stream_id, gd, gp, gl, gb)
    ctx.sync()
    dirs, pdf, strat = dirs.cpu().numpy(), pdf.cpu().numpy(), strat.cpu().numpy()
    gd, gb = gd.cpu().numpy(), gb.cpu().numpy().view(np.uint32)

    s = O.mis_sample(ref, slot, tabs, a32.astype(np.float64), pos, nrm.astype(np.float64), seed, stream_id)
    sg = O.sample(ref, slot, tabs, pos, seed, stream_id)
    leaf, _ = O.leaf_of_positions(ref, pos)
    # Strategy: the same decision wherever both sides hold the same alpha.
    same_a = a_kernel[leaf] == a32[leaf]
    assert same_a.mean() > 0.99
    assert np.array_equal(strat[same_a], s["strategy"][same_a])
    guided = same_a & (strat == 1)
    bsdf = same_a & (strat == 0)
    if q > 1000:
        assert guided.sum() > q // 10 and bsdf.sum() > q // 10
    # Guided branch: pg_sample_dirs' direction, bit for bit, and the oracle's
    # guided sample within the plain sampling test's bounds where the bins agree.
    assert np.array_equal(dirs[strat == 1], gd[strat == 1])
    same_bin = gb == sg["bin"]
    assert same_bin.mean() >= 1 - 1e-4
    err = np.abs(dirs.astype(np.float64) - s["dir"])
    gs = guided & same_bin
    assert np.all(err[gs, 2] <= 2.4e-7)
    assert np.all(err[gs, :2] <= 1e-6)  # sin(theta) from (1 + z)(1 - z): flat at the poles too
    # Lambertian branch.
    assert np.all(err[bsdf] <= 2e-6)
    assert np.all(np.sum(nrm[bsdf].astype(np.float64) * dirs[bsdf], axis=1) >= -1e-6)
    # Mixture pdf at the sampled direction.  Both sides re-bin their own
    # direction for the guide term; a direction within the bounds above of the
    # oracle's can fall in the neighbouring bin, so a small share may differ
    # by the ratio of two bins.
    ok = np.abs(pdf - s["pdf"]) <= 1e-5 * s["pdf"] + 1e-6
    assert ok[gs].sum() >= (1 - 1e-3) * gs.sum() and ok[bsdf].sum() >= (1 - 1e-3) * bsdf.sum()
    # Evaluation: at the sampled directions it returns the sampled pdf; at
    # uniform directions it matches the oracle.
    out = torch.empty(q, device="cuda")
    pg.pg_mis_eval(ctx, g, t, m, d_pos, d_n, torch.from_numpy(dirs).cuda(), q, out)
    ctx.sync()
    assert np.allclose(out.cpu().numpy(), pdf, rtol=1e-6, atol=1e-7)
    ud = synth.query_directions(q, (seed + 2) & 0xFFFF)
    pg.pg_mis_eval(ctx, g, t, m, d_pos, d_n, torch.from_numpy(ud).cuda(), q, out)
    ctx.sync()
    er = O.mis_eval(ref, slot, tabs, a32.astype(np.float64), pos, nrm.astype(np.float64), ud)
    assert np.all((np.abs(out.cpu().numpy() - er) <= 1e-5 * er + 1e-6)[same_a])


def test_leaves_without_map_sample_the_bsdf(scene, trained):
    ctx, g, t, ref, slot, tabs = (scene[k] for k in ("ctx", "g", "t", "ref", "slot", "tabs"))
    m = trained[0]
    q = 100_000
    pos = synth.query_positions(q, 71)
    nrm = synth.query_directions(q, 72)
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    strat = torch.empty(q, dtype=torch.uint8, device="cuda")
    pg.pg_mis_sample(ctx, g, t, m, torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), q, 5, 0, dirs,
                     pdf, strat)
    ctx.sync()
    leaf, _ = O.leaf_of_positions(ref, pos)
    sl = slot[leaf]
    nomap = (sl < 0) | (tabs["valid"][np.maximum(sl, 0)] == 0)
    assert nomap.any() and (sl[nomap] == 3).any()
    strat, dirs, pdf = strat.cpu().numpy(), dirs.cpu().numpy(), pdf.cpu().numpy()
    assert np.all(strat[nomap] == 0)
    c = np.maximum(0.0, np.sum(nrm[nomap].astype(np.float64) * dirs[nomap], axis=1))
    assert np.all(np.abs(pdf[nomap] - c / np.pi) <= 1e-6)


def test_invalid_inputs_and_handles(scene):
    ctx, g, t = scene["ctx"], scene["g"], scene["t"]
    m = pg.pg_mis_create(ctx, g)
    q = 64
    pos = torch.from_numpy(synth.query_positions(q, 81)).cuda()
    nrm = synth.query_directions(q, 82)
    nrm[7, 1] = np.nan
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    strat = torch.empty(q, dtype=torch.uint8, device="cuda")
    with pytest.raises(pg.PgError) as ei:
        pg.pg_mis_sample(ctx, g, t, m, pos, torch.from_numpy(nrm).cuda(), q, 1, 0, dirs, pdf, strat)
        ctx.sync()
    assert ei.value.status == 8
    ok_n = torch.from_numpy(synth.query_directions(q, 83)).cuda()
    bad_d = synth.query_directions(q, 84)
    bad_d[3, 2] = np.inf
    with pytest.raises(pg.PgError) as ei:
        pg.pg_mis_eval(ctx, g, t, m, pos, ok_n, torch.from_numpy(bad_d).cuda(), q, pdf)
        ctx.sync()
    assert ei.value.status == 8
    assert pdf[3].item() == 0.0
    # A negative contribution is rejected and leaves the statistics alone.
    before = pg.export_mis(m)
    c = torch.ones(q, device="cuda")
    c[10] = -1.0
    with pytest.raises(pg.PgError) as ei:
        pg.pg_mis_accumulate(ctx, m, g, pos, torch.zeros(q, dtype=torch.uint8, device="cuda"), c, q)
        ctx.sync()
    assert ei.value.status == 8
    after = pg.export_mis(m)
    assert after["q_b"].sum() == before["q_b"].sum() + q - 1 and not after["q_g"].any()
    # The context stays usable; q = 0 is a no-op; a grid of another size is refused.
    pg.pg_mis_sample(ctx, g, t, m, pos, ok_n, 0, 1, 0, dirs, pdf, strat)
    ctx.sync()
    ph = synth.photons(5000, 2, 85)
    g2 = pg.pg_build_grid(ctx, torch.from_numpy(ph).cuda(), 5000, LO, HI, 2, 1, 100)
    with pytest.raises(pg.PgError) as ei:
        pg.pg_mis_accumulate(ctx, m, g2, pos, torch.zeros(q, dtype=torch.uint8, device="cuda"), c, q)
    assert ei.value.status == 1
