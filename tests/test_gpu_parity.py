"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Integer work (codes, sort permutation, grid topology, leaf assignment,
histograms, sampled bins) must match bit for bit; floating-point results
within the tolerances derived in each test.
"""
import math

import os

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


def _grid_case(ctx, ph, D, min_depth, thr, lo=LO, hi=HI):
    n = ph.shape[0]
    d = torch.from_numpy(ph).cuda() if n else torch.empty(0, 8, device="cuda")
    g = pg.pg_build_grid(ctx, d if n else 0, n, lo, hi, D, min_depth, thr)
    ref = O.build_grid(ph, lo, hi, D, min_depth, thr)
    return g, pg.export_grid(g), ref, d


def _assert_grid_equal(got, ref):
    assert got["L"] == ref["L"]
    for k in ("codes", "perm", "leaf_of", "leaf_code", "leaf_begin", "leaf_end"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["leaf_depth"], ref["leaf_depth"])
    act, slot = O.active_leaves(ref)
    assert np.array_equal(got["active"], act)
    assert np.array_equal(got["slot_of_leaf"], slot)


# ------------------------------------------------------------------ a1-a4
@pytest.mark.parametrize("n,blobs,D,min_depth,thr,seed", [
    (100_000, 8, 4, 0, 1000, synth.SEED_BASE),  # tiny workload
    (77_777, 5, 10, 0, 300, 31),                 # ragged tail of the sort tile, 4 radix passes
    (4097, 3, 6, 2, 20, 32),                     # initial regular grid
    (1000, 2, 3, 0, 0, 33),                      # split everything to max depth
    (513, 2, 16, 0, 5, 34),                      # deepest codes (48 bits, 6 passes)
    (3000, 4, 5, 0, 10 ** 9, 35),                # threshold above n: one leaf
    (1, 1, 4, 0, 0, 36),
])
def test_grid_bit_exact(ctx, n, blobs, D, min_depth, thr, seed):
    ph = synth.photons(n, blobs, seed)
    g, got, ref, _ = _grid_case(ctx, ph, D, min_depth, thr)
    _assert_grid_equal(got, ref)
    g.free()


@pytest.mark.parametrize("n,blobs,D,min_depth,thr,seed", [(100_000, 8, 4, 0, 1000, 51), (77_777, 5, 10, 0, 300, 52),
                                                       (4097, 3, 6, 2, 20, 53), (513, 2, 16, 0, 5, 54)])
def test_grid_per_level_launches_equal_the_single_launch(ctx, n, blobs, D, min_depth, thr, seed):
    # The tree as one cooperative launch (default) and as one launch per
    # level and phase: both equal the oracle's grid bit for bit.
    ph = synth.photons(n, blobs, seed)
    os.environ["PG_GRID_LEVEL_LAUNCHES"] = "1"
    try:
        g, got, ref, _ = _grid_case(ctx, ph, D, min_depth, thr)
    finally:
        del os.environ["PG_GRID_LEVEL_LAUNCHES"]
    _assert_grid_equal(got, ref)
    g2, got2, _, _ = _grid_case(ctx, ph, D, min_depth, thr)
    _assert_grid_equal(got2, ref)


def test_grid_empty_and_odd_domain(ctx):
    g, got, ref, _ = _grid_case(ctx, np.zeros((0, 8), np.float32), 3, 1, 10)
    _assert_grid_equal(got, ref)
    assert got["A"] == 0 and got["L"] == 8
    ph = synth.photons(5000, 4, 37)
    ph[:, :3] = ph[:, :3] * 7.3 - 2.1  # positions outside a shifted domain are clamped
    lo, hi = [-1.5, -0.75, 0.25], [4.0, 2.5, 3.0]
    g2, got2, ref2, _ = _grid_case(ctx, ph, 7, 0, 40, lo, hi)
    _assert_grid_equal(got2, ref2)


def test_nonfinite_position_reported(ctx):
    ph = synth.photons(100, 1, 38)
    ph[5, 1] = np.nan
    with pytest.raises(pg.PgError) as e:
        pg.pg_build_grid(ctx, torch.from_numpy(ph).cuda(), 100, LO, HI, 3, 0, 10)
    assert e.value.status == 8


# ------------------------------------------------------------------ a5
@pytest.mark.parametrize("n,D,thr,H,W,n_prev", [
    (100_000, 4, 1000, 32, 32, 50_000),
    (60_000, 5, 2000, 64, 64, 20_001),
    (30_000, 4, 3000, 128, 128, 15_000),   # two-pass (16384 bins)
    (20_000, 3, 500, 8, 16, 0),            # no previous-iteration photons
    (9_999, 3, 100, 4, 256, 9_999),
])
def test_splat_bit_exact(ctx, n, D, thr, H, W, n_prev):
    ph = synth.photons(n, 6, 40 + H)
    g, got, ref, d = _grid_case(ctx, ph, D, 0, thr)
    h = pg.pg_splat_photons(ctx, g, d, n, n_prev, H, W)
    hh = pg.export_hist(h)
    ctx.sync()
    hr = O.splat(ph, ref, n_prev, H, W)
    act, _ = O.active_leaves(ref)
    for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
        assert np.array_equal(hh[k], hr[k][act]), k
    # Eq. (photon): mass conservation, exact.
    pfx = np.rint(ph[:, 6].astype(np.float64) * 2.0 ** 32).astype(np.uint64)
    assert int(hh["pow_cur"].sum(dtype=np.uint64)) == int(pfx.sum(dtype=np.uint64))
    h.free()
    g.free()


@pytest.mark.parametrize("W", [32, 256])
def test_splat_axis_and_seam_directions(ctx, W):
    """Directions on bin edges and the phi seam: the exact rule on both sides.
    Also just either side of every edge (rotated by 1e-7 and 1e-6 rad) and
    edges scaled down, where an angle-based first guess of the column is
    most often off by one."""
    H = 16
    dirs = [[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1e-30, 0],
            [1, -1e-30, 0], [-1, -1e-30, 0], [-1, 1e-38, 0], [0.7071068, 0.7071068, 0]]
    rng = np.random.default_rng(41)
    th = 2 * np.pi * np.arange(W) / W
    edge = np.stack([np.cos(th), np.sin(th), np.zeros(W)], 1)  # exactly on rounded boundary rays
    near = [np.stack([np.cos(th + e), np.sin(th + e), np.zeros(W)], 1) for e in (-1e-6, -1e-7, 1e-7, 1e-6)]
    rand = synth.uniform_sphere(rng, 5000)
    D = np.concatenate([np.array(dirs, np.float64), edge, edge * 1e-3, *near, rand]).astype(np.float32)
    n = D.shape[0]
    ph = np.zeros((n, 8), np.float32)
    ph[:, :3] = 0.5
    ph[:, 3:6] = D
    ph[:, 6] = 1.0
    g, got, ref, d = _grid_case(ctx, ph, 1, 0, 10 ** 9)
    h = pg.pg_splat_photons(ctx, g, d, n, 0, H, W)
    hh = pg.export_hist(h)
    hr = O.splat(ph, ref, 0, H, W)
    assert np.array_equal(hh["cnt_cur"], hr["cnt_cur"])
    assert np.array_equal(hh["pow_cur"], hr["pow_cur"])


def test_splat_status_errors(ctx):
    ph = synth.photons(500, 2, 42)
    ph[7, 6] = -1.0
    g, _, _, d = _grid_case(ctx, ph, 3, 0, 50)
    pg.pg_splat_photons(ctx, g, d, 500, 0, 8, 8)
    with pytest.raises(pg.PgError) as e:
        ctx.sync()
    assert e.value.status == 8
    ph = synth.photons(4, 1, 43)
    ph[:, 6] = 2.0 ** 30
    g, _, _, d = _grid_case(ctx, ph, 2, 0, 0)
    pg.pg_splat_photons(ctx, g, d, 4, 0, 8, 8)
    with pytest.raises(pg.PgError) as e:
        ctx.sync()
    assert e.value.status == 4
    with pytest.raises(pg.PgError) as e:
        pg.pg_splat_photons(ctx, g, d, 4, 0, 12, 8)
    assert e.value.status == 5


# ------------------------------------------------------------------ a8-a12 from a given map
def _maps(A, H, W, seed):
    rng = np.random.default_rng(seed)
    y = rng.lognormal(0, 2, (A, H, W)).astype(np.float32)
    y[0, 1, :] = 0
    y[min(1, A - 1), :, 2] = 0
    if A > 3:
        y[3] = 0  # an invalid (all-zero) map
    return y


@pytest.fixture(scope="module")
def tiny_scene(ctx):
    wl = synth.TINY
    ph = synth.photons(wl.n_photons, wl.n_blobs, wl.seed)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, wl.n_photons, LO, HI, wl.max_depth, 0, wl.split_threshold)
    ref = O.build_grid(ph, LO, HI, wl.max_depth, 0, wl.split_threshold)
    act, slot = O.active_leaves(ref)
    return dict(ph=ph, d=d, g=g, ref=ref, act=act, slot=slot, wl=wl)


# Maps of at most 64 rows and 128 columns keep their rows in registers; the
# others (128x128, 64x256) stream them.
@pytest.mark.parametrize("H,W", [(32, 32), (64, 64), (16, 128), (128, 128), (4, 4), (8, 16), (64, 256)])
def test_cdf_tables(ctx, tiny_scene, H, W):
    A = tiny_scene["g"].info(pg.PG_INFO_N_ACTIVE)
    y = _maps(A, H, W, H * 1000 + W)
    m = pg.pg_map_import(ctx, torch.from_numpy(y).cuda(), A, H, W)
    t = pg.pg_build_cdf(ctx, m)
    tt = pg.export_tables(t)
    ref = O.tables_from_map(y.astype(np.float64))
    assert np.array_equal(tt["valid"], ref["valid"])
    v = ref["valid"].astype(bool)
    P, Pr = tt["P"][v].astype(np.float64), ref["P"][v]
    nz = Pr > 0
    assert np.all(P[~nz] == 0)
    assert np.max(np.abs(P[nz] - Pr[nz]) / Pr[nz]) <= 1e-5
    # Decision tables: float32 of the FP64 CDFs, last entry 1.
    dz = tt["cdf_z"][v] != ref["fz"][v]
    dp = tt["cdf_phi"][v] != ref["fphi"][v]
    assert dz.mean() <= 1e-4 and dp.mean() <= 1e-4
    assert np.max(np.abs(tt["cdf_z"][v] - ref["fz"][v])) <= 1.2e-7
    assert np.max(np.abs(tt["cdf_phi"][v] - ref["fphi"][v])) <= 1.2e-7
    assert np.all(tt["cdf_z"][:, -1] == 1.0) and np.all(tt["cdf_phi"][:, :, -1] == 1.0)


def _run_sample(ctx, g, t, pos, seed, stream_id, host=False):
    q = pos.shape[0]
    if host:
        dirs = np.empty((q, 3), np.float32)
        pdf = np.empty(q, np.float32)
        leaf = np.empty(q, np.uint32)
        bins = np.empty(q, np.uint32)
        pg.pg_sample_dirs(ctx, g, t, np.ascontiguousarray(pos), q, seed, stream_id, dirs, pdf, leaf, bins)
        ctx.sync()
        return dirs, pdf, leaf, bins
    d_pos = torch.from_numpy(pos).cuda()
    dirs = torch.empty(q, 3, device="cuda")
    pdf = torch.empty(q, device="cuda")
    leaf = torch.empty(q, dtype=torch.int32, device="cuda")
    bins = torch.empty(q, dtype=torch.int32, device="cuda")
    pg.pg_sample_dirs(ctx, g, t, d_pos, q, seed, stream_id, dirs, pdf, leaf, bins)
    ctx.sync()
    return (dirs.cpu().numpy(), pdf.cpu().numpy(), leaf.cpu().numpy().view(np.uint32),
            bins.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("H,W,q,seed,stream_id", [(32, 32, 65_536, 7, 0), (64, 64, 100_003, 2 ** 40 + 5, 3),
                                                  (128, 128, 4_099, 11, 1), (8, 4, 1, 1, 0)])
def test_sample_and_eval(ctx, tiny_scene, H, W, q, seed, stream_id):
    g, ref, slot = tiny_scene["g"], tiny_scene["ref"], tiny_scene["slot"]
    A = g.info(pg.PG_INFO_N_ACTIVE)
    y = _maps(A, H, W, 7 * H + W)
    m = pg.pg_map_import(ctx, torch.from_numpy(y).cuda(), A, H, W)
    t = pg.pg_build_cdf(ctx, m)
    tabs = O.tables_from_map(y.astype(np.float64))
    pos = synth.query_positions(q, seed & 0xFFFF)
    dirs, pdf, leaf, bins = _run_sample(ctx, g, t, pos, seed, stream_id)
    s = O.sample(ref, slot, tabs, pos, seed, stream_id)
    assert np.array_equal(leaf, s["leaf"])
    same = bins == s["bin"]
    assert same.mean() >= 1 - 1e-4
    # z = -1 + 2 (i + u2)/H is formed in FP32 (abs. error <= 2^-23).  The
    # in-plane part scales by sin(theta) = sqrt((1 + z)(1 - z)), whose factors
    # 2 (i + u2)/H and 2 (H - i - u2)/H are each formed to one rounding, so
    # its relative error stays a few ulps at the poles too; the azimuth adds a
    # few ulps of sincos: one flat bound.
    err = np.abs(dirs.astype(np.float64) - s["dir"])
    assert np.all(err[same, 2] <= 2.4e-7)
    assert np.all(err[same, :2] <= 1e-6)
    nz = same & (s["pdf"] > 0)
    assert np.max(np.abs(pdf[nz] - s["pdf"][nz]) / s["pdf"][nz], initial=0) <= 1e-5
    # Host buffers go through the same kernels.
    hd, hp, hl, hb = _run_sample(ctx, g, t, pos, seed, stream_id, host=True)
    assert np.array_equal(hb, bins) and np.array_equal(hp, pdf) and np.array_equal(hd, dirs)
    # Evaluation at uniform directions and at the sampled directions.
    ev_dirs = synth.query_directions(q, seed & 0xFFFF)
    for dd in (ev_dirs, s["dir"].astype(np.float32)):
        out = torch.empty(q, device="cuda")
        pg.pg_eval_pdf(ctx, g, t, torch.from_numpy(pos).cuda(), torch.from_numpy(np.ascontiguousarray(dd)).cuda(), q, out)
        ctx.sync()
        e = out.cpu().numpy().astype(np.float64)
        er = O.eval_pdf(ref, slot, tabs, pos, dd)
        nz = er > 0
        assert np.all(e[~nz] == 0)
        assert np.max(np.abs(e[nz] - er[nz]) / er[nz], initial=0) <= 1e-5
    # Sampled directions evaluate to their own pdf (same bin rule), away from bin edges.
    ok = (leaf >> 31) == 0
    out = torch.empty(q, device="cuda")
    pg.pg_eval_pdf(ctx, g, t, torch.from_numpy(pos).cuda(), torch.from_numpy(dirs).cuda(), q, out)
    if ok.any():
        agree = np.isclose(out.cpu().numpy()[ok], pdf[ok], rtol=1e-6)
        assert agree.mean() >= 1 - 1e-3


# ------------------------------------------------------------------ a6-a7: CNN, FP32
def _cnn_case(ctx, wl_n, blobs, D, thr, H, W, arch, widths, seed, max_check_leaves=None):
    ph = synth.photons(wl_n, blobs, seed)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, wl_n, LO, HI, D, 0, thr)
    h = pg.pg_splat_photons(ctx, g, d, wl_n, wl_n // 2, H, W)
    blob = synth.net_blob(arch, widths, seed + 1)
    net = pg.pg_net_load(ctx, blob)
    m = pg.pg_reconstruct(ctx, h, net, pg.PG_FP32)
    t = pg.pg_build_cdf(ctx, m)
    y = pg.export_map(m)
    P = pg.export_tables(t)["P"]
    ctx.sync()
    ref = O.build_grid(ph, LO, HI, D, 0, thr)
    act, _ = O.active_leaves(ref)
    hr = O.hist_for_active(O.splat(ph, ref, wl_n // 2, H, W), act)
    if max_check_leaves is not None and act.size > max_check_leaves:
        idx = np.linspace(0, act.size - 1, max_check_leaves).astype(np.int64)
    else:
        idx = np.arange(act.size)
    hsub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in hr.items()}
    yr = O.cnn_forward(O.assemble_inputs(hsub), O.parse_net(blob))
    Pr, _ = O.normalise(yr)
    return y[idx].astype(np.float64), yr, P[idx].astype(np.float64), Pr


def _check_fp32_maps(y, yr, P, Pr):
    """FP32 accumulation over K <= 3456 terms of a He-initialised net: the
    pre-activation error is about K * 2^-24 times the sum of |w x|, so a
    softplus output carries relative error ~ |x| eps for x << 0 and ~ eps
    otherwise.  Gate: per bin |dP| <= 1e-5 P + 1e-7 max(P of the leaf), and per
    leaf L1 distance <= 1e-5."""
    for a in range(P.shape[0]):
        tol = 1e-5 * Pr[a] + 1e-7 * Pr[a].max()
        assert np.all(np.abs(P[a] - Pr[a]) <= tol), (a, np.max(np.abs(P[a] - Pr[a]) - tol))
        assert np.abs(P[a] - Pr[a]).sum() <= 1e-5
    big = yr > 1e-3 * yr.max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(y[big] - yr[big]) / yr[big]) <= 1e-4


def test_cnn_tiny_fp32(ctx):
    wl = synth.TINY
    y, yr, P, Pr = _cnn_case(ctx, wl.n_photons, wl.n_blobs, wl.max_depth, wl.split_threshold, 32, 32,
                             synth.ARCH_TINY3, (16,), wl.seed)
    _check_fp32_maps(y, yr, P, Pr)


def test_cnn_unet_fp32_small(ctx):
    y, yr, P, Pr = _cnn_case(ctx, 30_000, 6, 4, 1500, 32, 32, synth.ARCH_UNET4, (32, 64, 128, 256), 51,
                             max_check_leaves=12)
    _check_fp32_maps(y, yr, P, Pr)


def test_cnn_unet_fp32_rect(ctx):
    y, yr, P, Pr = _cnn_case(ctx, 20_000, 4, 3, 2500, 16, 64, synth.ARCH_UNET4, (8, 16, 16, 32), 52)
    _check_fp32_maps(y, yr, P, Pr)


def test_budget_and_bad_args(ctx):
    small = pg.Context(hbm_budget=1 << 20)
    ph = synth.photons(100_000, 3, 60)
    with pytest.raises(pg.PgError) as e:
        pg.pg_build_grid(small, torch.from_numpy(ph).cuda(), 100_000, LO, HI, 5, 0, 100)
    assert e.value.status == 3
    assert small.bytes_in_use() == 0
    small.destroy()
    with pytest.raises(pg.PgError) as e:
        pg.pg_build_grid(ctx, torch.from_numpy(ph).cuda(), 100_000, LO, HI, 17, 0, 100)
    assert e.value.status == 1


# ------------------------------------------------------------------ a7 on tensor cores
def _kl_l1(P, Pr):
    """Per-leaf KL(P_oracle || P_gpu) and L1, the reduced-precision gates."""
    kl, l1 = [], []
    for a in range(P.shape[0]):
        p, q = Pr[a].ravel(), np.maximum(P[a].ravel(), 1e-38)
        nz = p > 0
        kl.append(float(np.sum(p[nz] * np.log(p[nz] / q[nz]))))
        l1.append(float(np.abs(p - P[a].ravel()).sum()))
    return np.array(kl), np.array(l1)


def _lp_case(ctx, n, blobs, D, thr, H, W, arch, widths, seed, prec, max_check_leaves=16, return_inputs=False,
             tune=False, force=None):
    """force: a PG_TC_FORCE launch shape for every tensor-core layer that
    supports it (e.g. "3", the tap-stacked operand mode)."""
    ph = synth.photons(n, blobs, seed)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, n, LO, HI, D, 0, thr)
    h = pg.pg_splat_photons(ctx, g, d, n, n // 2, H, W)
    blob = synth.net_blob(arch, widths, seed + 1)
    net = pg.pg_net_load(ctx, blob)
    if tune:
        pg.pg_autotune(ctx, h, net, prec)  # the reconstruction below uses the tuned launch shapes
    if force is not None:
        os.environ["PG_TC_FORCE"] = force
    try:
        m = pg.pg_reconstruct(ctx, h, net, prec)
        ctx.sync()
    finally:
        os.environ.pop("PG_TC_FORCE", None)
    t = pg.pg_build_cdf(ctx, m)
    tt = pg.export_tables(t)
    ctx.sync()
    ref = O.build_grid(ph, LO, HI, D, 0, thr)
    act, _ = O.active_leaves(ref)
    idx = np.linspace(0, act.size - 1, min(act.size, max_check_leaves)).astype(np.int64)
    hr = O.hist_for_active(O.splat(ph, ref, n // 2, H, W), act)
    hsub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in hr.items()}
    x = O.assemble_inputs(hsub)
    netp = O.parse_net(blob)
    yr = O.cnn_forward(x, netp)
    Pr, _ = O.normalise(yr)
    if return_inputs:
        return tt["P"][idx].astype(np.float64), Pr, tt["valid"][idx], x, netp
    return tt["P"][idx].astype(np.float64), Pr, tt["valid"][idx]


@pytest.mark.parametrize("arch,widths,H,W,n,D,thr", [
    (synth.ARCH_TINY3, (16,), 32, 32, 100_000, 4, 1000),
    (synth.ARCH_TINY3, (32,), 64, 64, 100_000, 4, 1000),
    (synth.ARCH_UNET4, (32, 64, 128, 256), 64, 64, 40_000, 5, 2000),
    (synth.ARCH_UNET4, (32, 64, 128, 256), 32, 32, 20_000, 4, 1500),
    (synth.ARCH_UNET4, (16, 32, 64, 128), 128, 128, 8_000, 3, 3000),
    (synth.ARCH_UNET4, (32, 64, 128, 256), 128, 128, 8_000, 3, 3000),  # the precision workload's net and maps
])
def test_cnn_bf16_kl(ctx, arch, widths, H, W, n, D, thr):
    """BF16 tensor-core network: mean KL(P_oracle || P) <= 1e-3 over leaves,
    with the default launch shapes and with autotuned ones."""
    for tune, force in ((False, None), (True, None)):
        P, Pr, valid = _lp_case(ctx, n, 6, D, thr, H, W, arch, widths, 70 + H, pg.PG_BF16, tune=tune, force=force)
        assert np.all(valid == 1)
        kl, l1 = _kl_l1(P, Pr)
        print(f"bf16 tune={tune} force={force} {arch} {widths} {H}x{W}: KL mean {kl.mean():.2e} max {kl.max():.2e}; "
              f"L1 mean {l1.mean():.2e}")
        assert kl.mean() <= 1e-3
        assert np.all(np.isfinite(kl))


def _e4m3_emulated_P(x, net):
    """The same network in float64 with every conv input and weight cast to
    E4M3 (torch.float8_e4m3fn) under a per-tensor amax/448 scale, the head's
    weights kept FP32: what per-tensor FP8 quantisation alone does."""
    F = torch.nn.functional

    def q(t):
        s = t.abs().max() / 448.0
        s = s if s > 0 else torch.tensor(1.0, dtype=torch.float64)
        return (t / s).to(torch.float8_e4m3fn).to(torch.float64) * s

    Ls = net["layers"]
    last = len(Ls) - 1

    def c(h, i):
        cout, cin, k, st, a, w, b = Ls[i]
        wt = torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2)
        h = F.conv2d(q(h), wt if i == last else q(wt), torch.from_numpy(b.astype(np.float64)), stride=st,
                     padding=k // 2)
        return F.elu(h) if a == O.ACT_ELU else (F.softplus(h) if a == O.ACT_SOFTPLUS else h)

    t = torch.from_numpy(x).permute(0, 3, 1, 2)
    if net["arch"] == O.ARCH_TINY3:
        y = c(c(c(t, 0), 1), 2)
    else:
        up = lambda h: F.interpolate(h, scale_factor=2, mode="nearest")
        e0 = c(c(t, 0), 1)
        e1 = c(c(e0, 2), 3)
        e2 = c(c(e1, 4), 5)
        e3 = c(c(e2, 6), 7)
        d2 = c(c(torch.cat([up(e3), e2], 1), 8), 9)
        d1 = c(c(torch.cat([up(d2), e1], 1), 10), 11)
        d0 = c(c(torch.cat([up(d1), e0], 1), 12), 13)
        y = c(d0, 14)
    P, _ = O.normalise(y[:, 0].numpy())
    return P


@pytest.mark.parametrize("arch,widths,H,W,n,D,thr", [
    (synth.ARCH_UNET4, (32, 64, 128, 256), 64, 64, 40_000, 5, 2000),
    (synth.ARCH_UNET4, (32, 64, 128, 256), 128, 128, 8_000, 3, 3000),
    (synth.ARCH_TINY3, (32,), 32, 32, 100_000, 4, 1000),
])
def test_cnn_fp8_kl(ctx, arch, widths, H, W, n, D, thr):
    """FP8 E4M3 network (per-tensor scales, FP32 accumulation).

    E4M3 keeps 3 mantissa bits (relative rounding error up to 2^-4) at every
    layer input and weight.  With seeded He-normal weights the head's
    pre-activations span about -115..+250, so softplus turns that noise into
    large relative changes of small bins: a float64 emulation of the same
    network with E4M3 casts (torch.float8_e4m3fn, per-tensor amax scaling)
    gives mean KL 0.021 on the 64x64 case, while BF16 gives 9e-5.  The gate
    for FP8 is therefore relative to that emulation run on the same leaves:
    mean KL <= 1.5 x the emulation's + 2e-3 (BF16 meets 1e-3 outright)."""
    P, Pr, valid, x, net = _lp_case(ctx, n, 6, D, thr, H, W, arch, widths, 80 + H, pg.PG_FP8_E4M3,
                                    return_inputs=True)
    assert np.all(valid == 1)
    kl, l1 = _kl_l1(P, Pr)
    kle, _ = _kl_l1(_e4m3_emulated_P(x, net), Pr)
    print(f"fp8 {arch} {H}x{W}: KL mean {kl.mean():.2e} max {kl.max():.2e}; L1 mean {l1.mean():.2e}; "
          f"E4M3 emulation KL mean {kle.mean():.2e}")
    assert kl.mean() <= 1.5 * kle.mean() + 2e-3
    assert np.all(np.isfinite(kl))


@pytest.mark.parametrize("H,W,n,D,thr", [(64, 64, 40_000, 5, 2000), (32, 32, 20_000, 4, 1500)])
def test_cnn_fp8_mixed(ctx, H, W, n, D, thr):
    """E4M3 inside the U-Net, BF16 at full resolution (PG_FP8_MIXED).  Its
    layers at the BF16/E4M3 boundary read one operand type and write the
    other, so the MMA kind must follow the operands.  Gate: no worse than the
    all-E4M3 form on the same leaves (whose own gate is an E4M3 emulation),
    and a mean KL that a kind mismatch (garbage maps, KL ~ 80) cannot meet."""
    arch, widths = synth.ARCH_UNET4, (32, 64, 128, 256)
    P8, Pr, _ = _lp_case(ctx, n, 6, D, thr, H, W, arch, widths, 80 + H, pg.PG_FP8_E4M3)
    Pm, Pr2, valid = _lp_case(ctx, n, 6, D, thr, H, W, arch, widths, 80 + H, pg.PG_FP8_MIXED)
    assert np.array_equal(Pr, Pr2) and np.all(valid == 1)
    k8, _ = _kl_l1(P8, Pr)
    km, _ = _kl_l1(Pm, Pr)
    print(f"fp8 mixed {H}x{W}: KL mean {km.mean():.2e} (all-E4M3 {k8.mean():.2e})")
    assert np.all(np.isfinite(km)) and km.mean() <= 1.2 * k8.mean() + 1e-3 and km.mean() < 0.1
