"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a published
known-answer vector, a closed form, a brute-force restatement of the same rule
with a different algorithm, an independent library routine, or an invariant
the paper states.  A plausible mistake in the oracle (dropped term, wrong sign
or index, transposed operand) fails one of them.
"""
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

from oracle import oracle as O
from paper_2010_01775_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LO = np.zeros(3, np.float32)
HI = np.ones(3, np.float32)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert list(O.philox4x32_10(v[0:4], v[4:6])) == v[6:10]
        n += 1
    assert n == 3


# ---------------------------------------------------------------- voxel location (a1)
def _deinterleave(code, D):
    q = [0, 0, 0]
    for b in range(D):
        for a in range(3):
            q[a] |= ((int(code) >> (3 * b + a)) & 1) << b
    return q


def test_morton_hand_values_and_roundtrip():
    lib = O.lib()
    assert lib.or_morton3(1, 0, 0, 2) == 1
    assert lib.or_morton3(0, 1, 0, 2) == 2
    assert lib.or_morton3(0, 0, 1, 2) == 4
    assert lib.or_morton3(2, 0, 0, 2) == 8
    assert lib.or_morton3(3, 3, 3, 2) == 63
    assert lib.or_morton3(1023, 0, 0, 10) == int("001" * 10, 2)
    rng = np.random.default_rng(1)
    for _ in range(200):
        D = int(rng.integers(1, 17))
        q = [int(x) for x in rng.integers(0, 2 ** D, 3)]
        code = lib.or_morton3(*q, D)
        assert _deinterleave(code, D) == q
        # Hierarchical nesting: the depth-d ancestor is the code of q >> (D - d).
        d = int(rng.integers(0, D + 1))
        assert code >> (3 * (D - d)) == lib.or_morton3(*[x >> (D - d) for x in q], d)


def test_quantisation_is_the_containing_cell():
    """q is the cell [lo + q h, lo + (q+1) h) containing x (h = (hi-lo)/2^D),
    away from float rounding at cell faces; clamped outside the domain."""
    rng = np.random.default_rng(2)
    lo = np.array([-1.5, 0.25, 3.0], np.float32)
    hi = np.array([2.5, 1.25, 7.0], np.float32)
    D = 7
    pos = (lo + (hi - lo) * rng.random((20000, 3))).astype(np.float32)
    codes, st = O.morton_codes(pos, lo, hi, D)
    assert st == 0
    h = (hi.astype(np.float64) - lo) / 2 ** D
    for i in range(pos.shape[0]):
        q = _deinterleave(codes[i], D)
        for a in range(3):
            t = (float(pos[i, a]) - float(lo[a])) / h[a]
            if abs(t - round(t)) < 1e-4:
                continue
            assert q[a] == math.floor(t)
    outside = np.array([[-9, 0.75, 100], [2.5, 1.25, 7.0]], np.float32)
    codes, st = O.morton_codes(outside, lo, hi, D)
    assert _deinterleave(codes[0], D) == [0, 2 ** (D - 1), 2 ** D - 1]
    assert _deinterleave(codes[1], D) == [2 ** D - 1] * 3
    _, st = O.morton_codes(np.array([[np.nan, 0, 0]], np.float32), lo, hi, D)
    assert st == O.ERR_INVALID_INPUT


# ---------------------------------------------------------------- grid (a2-a4)
def _brute_grid(q, D, min_depth, thr):
    """Recursive subdivision by direct membership counting over integer cells.
    Children are visited x-fastest (k = x + 2y + 4z), i.e. Morton order."""
    leaves = []

    def members(idx, c, d):
        return [i for i in idx if all((q[i][a] >> (D - d)) == c[a] for a in range(3))]

    def rec(c, d, idx):
        if len(idx) > thr and d < D:
            for k in range(8):
                cc = [2 * c[0] + (k & 1), 2 * c[1] + ((k >> 1) & 1), 2 * c[2] + ((k >> 2) & 1)]
                rec(cc, d + 1, members(idx, cc, d + 1))
        else:
            leaves.append((c, d, sorted(idx)))

    n0 = 2 ** min_depth
    cells = []
    for z in range(n0):
        for y in range(n0):
            for x in range(n0):
                cells.append([x, y, z])
    lib = O.lib()
    cells.sort(key=lambda c: lib.or_morton3(c[0], c[1], c[2], min_depth))
    all_idx = list(range(len(q)))
    for c in cells:
        rec(c, min_depth, members(all_idx, c, min_depth))
    return leaves


@pytest.mark.parametrize("n,D,min_depth,thr,seed", [
    (300, 3, 0, 20, 3), (500, 4, 1, 10, 4), (200, 2, 0, 0, 5), (400, 5, 0, 1000, 6), (0, 3, 0, 5, 7),
    (257, 4, 2, 3, 8)])
def test_grid_matches_brute_force(n, D, min_depth, thr, seed):
    ph = synth.photons(n, 3, seed)
    g = O.build_grid(ph, LO, HI, D, min_depth, thr)
    q = [_deinterleave(c, D) for c in g["codes"]]
    leaves = _brute_grid(q, D, min_depth, thr)
    assert g["L"] == len(leaves)
    lib = O.lib()
    for l, (c, d, idx) in enumerate(leaves):
        assert g["leaf_depth"][l] == d
        assert g["leaf_code"][l] == lib.or_morton3(c[0], c[1], c[2], d) << (3 * (D - d))
        got = sorted(int(p) for p in g["perm"][g["leaf_begin"][l]:g["leaf_end"][l]])
        assert got == idx
        for p in idx:
            assert g["leaf_of"][p] == l


def test_grid_invariants_tiny_workload():
    wl = synth.TINY
    ph = synth.photons(wl.n_photons, wl.n_blobs, wl.seed)
    g = O.build_grid(ph, LO, HI, wl.max_depth, 0, wl.split_threshold)
    D = wl.max_depth
    cnt = g["leaf_end"].astype(np.int64) - g["leaf_begin"]
    assert cnt.sum() == ph.shape[0]
    # Leaves partition the cube: volumes sum to one, start codes strictly increase.
    assert sum(8 ** (D - int(d)) for d in g["leaf_depth"]) == 8 ** D
    assert np.all(np.diff(g["leaf_code"].astype(np.float64)) > 0)
    # A leaf above max depth... cannot exist; below max depth it holds <= thr photons.
    assert np.all(cnt[g["leaf_depth"] < D] <= wl.split_threshold)
    # Sorted order is by code, ties by original index (a stable sort).
    key = g["codes"][g["perm"]].astype(np.float64) * 2.0 ** 20 + g["perm"]
    assert np.all(np.diff(key) > 0)
    # Single leaf when the threshold covers everything.
    g1 = O.build_grid(ph[:500], LO, HI, D, 0, 500)
    assert g1["L"] == 1 and g1["leaf_end"][0] == 500


# ---------------------------------------------------------------- direction bins
def test_axis_directions_hand_bins():
    H, W = 32, 64
    dirs = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                     [1, 1e-30, 0], [1, -1e-30, 0], [-1, -1e-30, 0]], np.float32)
    rows, cols, st = O.dir_bins(dirs, H, W)
    assert st == 0
    assert list(rows) == [16, 16, 16, 16, 31, 0, 16, 16, 16]
    assert list(cols) == [0, 16, 32, 48, 0, 0, 0, 63, 32]


def test_bins_match_atan2_away_from_edges():
    rng = np.random.default_rng(9)
    for H, W in [(32, 32), (64, 64), (128, 128), (8, 4), (64, 128)]:
        d = synth.uniform_sphere(rng, 20000).astype(np.float32)
        rows, cols, _ = O.dir_bins(d, H, W)
        phi = np.mod(np.arctan2(d[:, 1].astype(np.float64), d[:, 0]), 2 * np.pi)
        tj = phi * W / (2 * np.pi)
        ti = (d[:, 2].astype(np.float64) + 1.0) * H / 2
        okj = np.abs(tj - np.round(tj)) > 1e-4
        oki = np.abs(ti - np.round(ti)) > 1e-4
        assert np.array_equal(cols[okj], np.floor(tj[okj]).astype(np.int64) % W)
        assert np.array_equal(rows[oki], np.clip(np.floor(ti[oki]), 0, H - 1).astype(np.int64))


def test_bins_are_equal_area():
    """Uniform directions fill every bin equally (cylindrical map is
    area-preserving, Sec. 4): chi-square goodness of fit."""
    from scipy.stats import chisquare
    rng = np.random.default_rng(10)
    H, W = 16, 32
    d = synth.uniform_sphere(rng, 400000).astype(np.float32)
    rows, cols, _ = O.dir_bins(d, H, W)
    counts = np.bincount(rows * W + cols, minlength=H * W)
    assert chisquare(counts).pvalue > 1e-3


# ---------------------------------------------------------------- splat (a5)
def _brute_splat(ph, g, n_prev, H, W, F):
    rows, cols, _ = O.dir_bins(ph[:, 3:6], H, W)
    pfx = [int(v) for v in np.rint(ph[:, 6].astype(np.float64) * 2.0 ** F)]
    L = g["L"]
    pc = [[0] * (H * W) for _ in range(L)]
    cc = [[0] * (H * W) for _ in range(L)]
    pp = [[0] * (H * W) for _ in range(L)]
    cp = [[0] * (H * W) for _ in range(L)]
    for p in range(ph.shape[0]):
        l, k = int(g["leaf_of"][p]), int(rows[p] * W + cols[p])
        pc[l][k] += pfx[p]
        cc[l][k] += 1
        if p < n_prev:
            pp[l][k] += pfx[p]
            cp[l][k] += 1
    return pc, cc, pp, cp, pfx


def test_splat_matches_brute_force_and_conserves_mass():
    ph = synth.photons(3000, 4, 11)
    g = O.build_grid(ph, LO, HI, 4, 0, 100)
    H, W, F = 8, 16, 32
    h = O.splat(ph, g, 1234, H, W, F)
    assert h["status"] == 0
    pc, cc, pp, cp, pfx = _brute_splat(ph, g, 1234, H, W, F)
    assert h["pow_cur"].tolist() == pc and h["cnt_cur"].tolist() == cc
    assert h["pow_prev"].tolist() == pp and h["cnt_prev"].tolist() == cp
    # Eq. (photon): the map of a leaf sums to the power of its photons, exactly.
    assert sum(int(v) for v in h["pow_cur"].ravel()) == sum(pfx)
    assert int(h["cnt_cur"].sum()) == 3000
    # The previous-iteration channels equal the current channels of the first n_prev photons.
    h2 = O.splat(ph[:1234], O.build_grid(ph[:1234], LO, HI, 4, 0, 10 ** 9), 0, H, W, F)
    assert sum(int(v) for v in h["pow_prev"].ravel()) == sum(int(v) for v in h2["pow_cur"].ravel())


def test_single_photon_single_bin_and_status():
    ph = np.zeros((1, 8), np.float32)
    ph[0, :7] = [0.3, 0.3, 0.3, 0.0, 0.0, 1.0, 0.75]
    g = O.build_grid(ph, LO, HI, 2, 0, 0)
    h = O.splat(ph, g, 1, 4, 4)
    l = g["leaf_of"][0]
    assert np.count_nonzero(h["pow_cur"]) == 1
    assert h["pow_cur"][l, 3 * 4 + 0] == 3 << 30  # 0.75 * 2^32, top row, column 0
    bad = ph.copy()
    bad[0, 6] = np.nan
    assert O.splat(bad, g, 0, 4, 4)["status"] == O.ERR_INVALID_INPUT
    big = np.repeat(ph, 4, axis=0)
    big[:, 6] = 2.0 ** 30  # 2^62 fixed point each: four of them would overflow 2^63
    gb = O.build_grid(big, LO, HI, 2, 0, 0)
    assert O.splat(big, gb, 0, 4, 4)["status"] == O.ERR_OVERFLOW


def test_fixed_point_rounds_half_even():
    ph = np.zeros((3, 8), np.float32)
    ph[:, 3] = 1.0
    ph[:, 6] = [2.0 ** -33, 3 * 2.0 ** -33, 2.0 ** -34]  # 0.5, 1.5, 0.25 units
    g = O.build_grid(ph, LO, HI, 1, 0, 10)
    h = O.splat(ph, g, 0, 4, 4)
    assert int(h["pow_cur"].sum()) == 0 + 2 + 0


# ---------------------------------------------------------------- inputs (a6)
def test_input_channels():
    ph = synth.photons(5000, 4, 12)
    g = O.build_grid(ph, LO, HI, 3, 0, 300)
    act, _ = O.active_leaves(g)
    h = O.hist_for_active(O.splat(ph, g, 2500, 16, 16), act)
    x = O.assemble_inputs(h)
    HW = 256
    for a in range(len(act)):
        s0 = x[a, ..., 0].sum()
        assert abs(s0 - HW) < 1e-9 * HW  # mean-one density
        if h["pow_prev"][a].sum() > 0:
            assert abs(x[a, ..., 1].sum() - HW) < 1e-9 * HW
        c = h["cnt_cur"][a].reshape(16, 16)
        assert np.array_equal(x[a, ..., 4], (c > 0).astype(np.float64))
        assert np.allclose(x[a, ..., 2], np.log1p(c), rtol=0, atol=1e-15)
        k = int(np.argmax(h["pow_cur"][a]))
        assert math.isclose(x[a].reshape(HW, 5)[k, 0],
                            int(h["pow_cur"][a][k]) * HW / int(h["pow_cur"][a].sum()), rel_tol=1e-14)


# ---------------------------------------------------------------- CNN (a7)
@pytest.mark.parametrize("A,H,W,Cin,Cout,k,stride", [
    (2, 8, 8, 5, 7, 3, 1), (3, 16, 8, 6, 4, 3, 2), (1, 8, 16, 3, 2, 1, 1), (2, 4, 4, 9, 3, 3, 1)])
def test_conv2d_matches_torch(A, H, W, Cin, Cout, k, stride):
    rng = np.random.default_rng(13)
    x = rng.standard_normal((A, H, W, Cin))
    w = rng.standard_normal((Cout, k, k, Cin)).astype(np.float32)
    b = rng.standard_normal(Cout).astype(np.float32)
    got = O.conv2d(x, w, b, stride)
    ref = Fnn.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2), torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                     torch.from_numpy(b.astype(np.float64)), stride=stride, padding=k // 2)
    assert np.allclose(got, ref.permute(0, 2, 3, 1).numpy(), rtol=1e-12, atol=1e-12)


def test_oracle_results_do_not_depend_on_thread_count():
    """The parallel loops compute every output by the same sequential sum:
    one host thread and all of them give identical bits."""
    rng = np.random.default_rng(16)
    x = rng.standard_normal((3, 16, 16, 8))
    w = rng.standard_normal((8, 3, 3, 8)).astype(np.float32)
    b = rng.standard_normal(8).astype(np.float32)
    ph = synth.photons(20_000, 4, 16)
    g = O.build_grid(ph, LO, HI, 4, 0, 500)
    act, slot = O.active_leaves(g)
    h = O.hist_for_active(O.splat(ph, g, 10_000, 8, 16), act)
    t = O.tables_from_map(np.exp(O.assemble_inputs(h)[..., 2]))
    pos = synth.query_positions(5000, 16)
    d = synth.query_directions(5000, 16)
    out = []
    try:
        for n in (1, 0):
            O.set_threads(n)
            s = O.sample(g, slot, t, pos, 7)
            out.append((O.conv2d(x, w, b, 1), O.conv2d(x, w, b, 2, 2), s["dir"], s["pdf"], s["bin"],
                        O.eval_pdf(g, slot, t, pos, d)))
    finally:
        O.set_threads(0)
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_conv2d_delta_kernel_is_identity():
    rng = np.random.default_rng(14)
    x = rng.standard_normal((2, 8, 8, 3))
    w = np.zeros((3, 3, 3, 3), np.float32)
    for c in range(3):
        w[c, 1, 1, c] = 1.0
    assert np.array_equal(O.conv2d(x, w, np.zeros(3, np.float32), 1), x)


def test_activations_closed_forms():
    assert O.elu(np.array([2.0]))[0] == 2.0
    assert math.isclose(O.elu(np.array([-1.0]))[0], math.exp(-1) - 1, rel_tol=1e-15)
    assert math.isclose(O.softplus(np.array([0.0]))[0], math.log(2.0), rel_tol=1e-15)
    assert math.isclose(O.softplus(np.array([-40.0]))[0], math.exp(-40.0), rel_tol=1e-12)
    assert O.softplus(np.array([800.0]))[0] == 800.0


def _torch_unet(x, net):
    """The same U-Net wired with torch.nn.functional in float64 (library pin)."""
    t = torch.from_numpy(x).permute(0, 3, 1, 2)
    Ls = net["layers"]

    def run(h, i):
        cout, cin, k, stride, act, w, b = Ls[i]
        h = Fnn.conv2d(h, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                       torch.from_numpy(b.astype(np.float64)), stride=stride, padding=k // 2)
        return Fnn.elu(h) if act == O.ACT_ELU else (Fnn.softplus(h) if act == O.ACT_SOFTPLUS else h)

    up = lambda h: Fnn.interpolate(h, scale_factor=2, mode="nearest")
    e0 = run(run(t, 0), 1)
    e1 = run(run(e0, 2), 3)
    e2 = run(run(e1, 4), 5)
    e3 = run(run(e2, 6), 7)
    d2 = run(run(torch.cat([up(e3), e2], 1), 8), 9)
    d1 = run(run(torch.cat([up(d2), e1], 1), 10), 11)
    d0 = run(run(torch.cat([up(d1), e0], 1), 12), 13)
    return run(d0, 14)[:, 0].numpy()


def test_unet_matches_torch_wiring():
    net = O.parse_net(synth.net_blob(synth.ARCH_UNET4, (8, 8, 16, 16), 15))
    rng = np.random.default_rng(15)
    x = rng.standard_normal((2, 16, 16, 5))
    assert np.allclose(O.cnn_forward(x, net), _torch_unet(x, net), rtol=1e-10, atol=1e-300)


def test_tiny_net_zero_input_interior_closed_form():
    """All-zero input: layer 1 is elu(b1) everywhere; at pixels two away from
    the border every tap sees interior values, so the output is
    softplus(b3 + sum w3 elu(b2 + sum w2 elu(b1)))."""
    net = O.parse_net(synth.net_blob(synth.ARCH_TINY3, (16,), 16))
    (c1, _, _, _, _, w1, b1), (c2, _, _, _, _, w2, b2), (c3, _, _, _, _, w3, b3) = net["layers"]
    y = O.cnn_forward(np.zeros((1, 8, 8, 5)), net)
    h1 = O.elu(b1.astype(np.float64))
    h2 = O.elu(b2 + np.einsum("oyxi,i->o", w2.astype(np.float64), h1))
    ref = O.softplus(b3 + np.einsum("oyxi,i->o", w3.astype(np.float64), h2))[0]
    assert np.allclose(y[0, 2:6, 2:6], ref, rtol=1e-13)


# ---------------------------------------------------------------- normalise / CDF (a8-a9)
def _random_maps(A, H, W, seed, zero_rows=True):
    rng = np.random.default_rng(seed)
    y = rng.lognormal(0, 2, (A, H, W))
    if zero_rows:
        y[0, 3, :] = 0.0
        y[1, :, 5] = 0.0
    return y


def test_pdf_integrates_to_one_and_cdfs_end_at_one():
    y = _random_maps(4, 16, 32, 17)
    t = O.tables_from_map(y)
    H, W = 16, 32
    dOmega = 4 * np.pi / (H * W)
    for a in range(4):
        pdf = t["P"][a] * H * W / (4 * np.pi)
        assert abs((pdf * dOmega).sum() - 1.0) < 1e-12
        assert t["Fz"][a, -1] == pytest.approx(1.0, abs=1e-14)
        assert np.all(np.abs(t["Fphi"][a, :, -1] - 1.0) < 1e-14)
        assert np.all(np.diff(t["Fz"][a]) >= 0) and np.all(np.diff(t["Fphi"][a], axis=1) >= 0)
        # Differences of the CDFs reproduce the map.
        m = np.diff(np.concatenate([[0.0], t["Fz"][a]]))
        assert np.allclose(m, t["P"][a].sum(axis=1), atol=1e-15)
        rows_ok = m > 0
        cond = np.diff(np.concatenate([np.zeros((H, 1)), t["Fphi"][a]], axis=1))
        assert np.allclose((cond * m[:, None])[rows_ok], t["P"][a][rows_ok], atol=1e-15)
    assert np.array_equal(t["Fphi"][0, 3], (np.arange(W) + 1.0) / W)  # empty row -> uniform
    assert t["fz"][0, -1] == 1.0 and np.all(t["fphi"][:, :, -1] == 1.0)


def test_invalid_map_flagged():
    y = np.zeros((2, 4, 4))
    y[1, 0, 0] = 1.0
    t = O.tables_from_map(y)
    assert list(t["valid"]) == [0, 1]
    assert t["P"][1, 0, 0] == 1.0


# ---------------------------------------------------------------- sampling / eval (a10-a12)
def _one_leaf_grid():
    ph = np.zeros((1, 8), np.float32)
    ph[0, :3] = 0.5
    return O.build_grid(ph, LO, HI, 0, 0, 10)


def test_sampling_chi_square_and_bins_and_pdf():
    from scipy.stats import chisquare
    H, W = 8, 16
    g = _one_leaf_grid()
    y = _random_maps(1, H, W, 18, zero_rows=False)
    y[0, 2, :] = 0.0
    y[0, 5, 7] = 0.0
    t = O.tables_from_map(y)
    q = 200000
    pos = np.full((q, 3), 0.25, np.float32)
    s = O.sample(g, np.zeros(1, np.int32), t, pos, seed=99, stream=3)
    assert np.all(s["leaf"] == 0)
    counts = np.bincount(s["bin"].astype(np.int64), minlength=H * W)
    P = t["P"][0].ravel()
    assert counts[P == 0].sum() == 0  # zero-mass bins never drawn
    exp = P * q
    keep = exp >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    assert chisquare(obs, e * obs.sum() / e.sum()).pvalue > 1e-3
    # Sampled directions are unit and land in their bin; returned pdf = eval pdf.
    d32 = s["dir"].astype(np.float32)
    assert np.allclose(np.linalg.norm(s["dir"], axis=1), 1.0, atol=1e-12)
    rows, cols, _ = O.dir_bins(d32, H, W)
    same = (rows * W + cols) == s["bin"]
    assert same.mean() > 1 - 1e-4
    ev = O.eval_pdf(g, np.zeros(1, np.int32), t, pos, d32)
    assert np.allclose(ev[same], s["pdf"][same], rtol=1e-14)
    assert np.allclose(s["pdf"], P[s["bin"]] * H * W / (4 * np.pi), rtol=1e-14)


def test_one_leaf_grids_of_both_forms_sample_alike():
    """A one-voxel grid of the paper's form (R = 1, no split) and a one-cell
    octree are the same single leaf: sampling and evaluation through the
    tree-walk path give what the code-search path gives, value for value."""
    H, W = 8, 16
    ph = synth.photons(500, 2, 21)
    g_oct = _one_leaf_grid()
    g_kd = O.build_kd_grid(ph, None, LO, HI, 1, 8, 10 ** 6, 0.5)
    assert g_kd["L"] == 1 and g_kd["kd"]
    y = _random_maps(1, H, W, 22, zero_rows=False)
    y[0, 3, :] = 0.0  # an empty row
    t = O.tables_from_map(y)
    pos = synth.query_positions(20000, 21)
    one = np.zeros(1, np.int32)
    a = O.sample(g_oct, one, t, pos, seed=31, stream=4)
    b = O.sample(g_kd, one, t, pos, seed=31, stream=4)
    for k in ("leaf", "bin", "dir", "pdf"):
        assert np.array_equal(a[k], b[k]), k
    d = synth.query_directions(20000, 21)
    assert np.array_equal(O.eval_pdf(g_oct, one, t, pos, d), O.eval_pdf(g_kd, one, t, pos, d))


def test_pdf_monte_carlo_mean_is_one():
    """E over uniform directions of p(w) * 4pi equals the integral of p: 1."""
    H, W = 16, 16
    g = _one_leaf_grid()
    t = O.tables_from_map(_random_maps(1, H, W, 19, zero_rows=False))
    rng = np.random.default_rng(19)
    d = synth.uniform_sphere(rng, 400000).astype(np.float32)
    p = O.eval_pdf(g, np.zeros(1, np.int32), t, np.full((d.shape[0], 3), 0.5, np.float32), d) * 4 * np.pi
    assert abs(p.mean() - 1.0) < 5 * p.std() / math.sqrt(p.size)


def test_uniform_fallback_for_leaves_without_map():
    ph = synth.photons(2000, 2, 20)
    g = O.build_grid(ph, LO, HI, 3, 0, 50)
    act, slot = O.active_leaves(g)
    H, W = 8, 8
    t = O.tables_from_map(np.ones((act.size, H, W)))
    pos = synth.query_positions(5000, 20)
    s = O.sample(g, slot, t, pos, seed=5)
    leaf = s["leaf"] & 0x7FFFFFFF
    codes, _ = O.morton_codes(pos, LO, HI, 3)
    assert np.array_equal(leaf, np.searchsorted(g["leaf_code"], codes, side="right") - 1)
    empty = slot[leaf] < 0
    assert empty.any() and (~empty).any()
    assert np.all((s["leaf"] >> 31) == empty)
    assert np.allclose(s["pdf"][empty], 1 / (4 * np.pi))
    assert np.allclose(s["pdf"][~empty], 1 / (4 * np.pi))  # a constant map is the uniform pdf
    assert np.all(s["bin"][empty] == 0xFFFFFFFF)


def test_expert_ranges_follow_the_papers_count_table():
    # Sec. 8: [0,100), [100,500), [500,1000), [1000,5000), [5000,inf).
    counts = [0, 1, 99, 100, 499, 500, 999, 1000, 4999, 5000, 10 ** 7]
    assert O.expert_of(counts).tolist() == [0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4]
    assert O.expert_of([5, 6], bounds=()).tolist() == [0, 0]


def test_experts_forward_routes_each_leaf_to_its_net():
    # With two experts the mixture equals each net on its own leaves.
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 8, 8, 5))
    nets = [O.parse_net(synth.net_blob(synth.ARCH_TINY3, (4,), s)) for s in (1, 2)]
    counts = np.array([10, 700, 3, 100])
    y = O.cnn_forward_experts(x, counts, nets, bounds=(100,))
    for k, e in enumerate(O.expert_of(counts, (100,))):
        assert np.array_equal(y[k], O.cnn_forward(x[k:k + 1], nets[e])[0])


# ---------------------------------------------------------------- one-sample MIS (Sec. 7.3)
def test_mis_alpha_rule_hand_values():
    # Eq. mis_alpha: alpha = avg_B / (avg_B + avg_G), clamped to [0.2, 0.8],
    # changed only where both strategies have at least 50 samples.
    st = dict(nu_b=np.array([50.0, 150.0, 450.0, 0.0, 50.0, 0.0, 7.0]),
              nu_g=np.array([150.0, 50.0, 50.0, 50.0, 150.0, 0.0, 7.0]),
              q_b=np.array([50, 50, 50, 50, 49, 60, 100]),
              q_g=np.array([50, 50, 50, 50, 50, 60, 100]))
    a = O.mis_alpha(st, np.full(7, 0.5))
    assert a.tolist() == [0.25, 0.75, 0.8, 0.2, 0.5, 0.5, 0.5]
    a = O.mis_alpha(st, np.full(7, 0.3), min_count=10, lo=0.0, hi=1.0)
    assert a.tolist()[:4] == [0.25, 0.75, 0.9, 0.0] and a.tolist()[5:] == [0.3, 0.5]
    assert a[4] == pytest.approx((50 / 49) / (50 / 49 + 3), rel=1e-15)


def test_mis_accumulate_matches_loops():
    rng = np.random.default_rng(4)
    L, q = 7, 500
    leaf = rng.integers(0, L, q)
    strat = rng.integers(0, 2, q).astype(np.uint8)
    c = rng.random(q)
    st = O.mis_accumulate(L, leaf, strat, c)
    for j in range(L):
        b = [c[k] for k in range(q) if leaf[k] == j and strat[k] == 0]
        g = [c[k] for k in range(q) if leaf[k] == j and strat[k] == 1]
        assert st["q_b"][j] == len(b) and st["q_g"][j] == len(g)
        assert st["nu_b"][j] == pytest.approx(math.fsum(b), rel=1e-13)
        assert st["nu_g"][j] == pytest.approx(math.fsum(g), rel=1e-13)


def test_tangent_frame_is_orthonormal_and_right_handed():
    rng = np.random.default_rng(5)
    n = synth.uniform_sphere(rng, 1000)
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1e-4, -1 + 5e-9]]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    b1, b2 = O.tangent_frame(n)
    for u, v in ((b1, b1), (b2, b2)):
        assert np.allclose(np.sum(u * v, axis=1), 1.0, atol=1e-9)
    for u, v in ((b1, b2), (b1, n), (b2, n)):
        assert np.allclose(np.sum(u * v, axis=1), 0.0, atol=1e-9)
    assert np.allclose(np.cross(b1, b2), n, atol=1e-9)


def test_cosine_lobe_distribution():
    # Lambertian sampling: (n.w)^2 is uniform on [0, 1] and the azimuth in the
    # tangent plane is uniform; E[n.w] = 2/3.
    from scipy.stats import kstest
    rng = np.random.default_rng(6)
    q = 100000
    n = synth.uniform_sphere(rng, q)
    d = O.cosine_sample(n, rng.random(q), rng.random(q))
    c = np.sum(n * d, axis=1)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12) and np.all(c >= 0)
    assert kstest(c ** 2, "uniform").pvalue > 1e-3
    assert abs(c.mean() - 2 / 3) < 5 * c.std() / math.sqrt(q)
    b1, b2 = O.tangent_frame(n)
    az = np.arctan2(np.sum(b2 * d, axis=1), np.sum(b1 * d, axis=1))
    assert kstest((az + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


def _mis_setup(H=8, W=16, seed=21):
    g = _one_leaf_grid()
    t = O.tables_from_map(_random_maps(1, H, W, seed, zero_rows=False))
    return g, np.zeros(1, np.int32), t


def test_mis_pdf_integrates_to_one():
    g, slot, t = _mis_setup()
    rng = np.random.default_rng(22)
    q = 400000
    d = synth.uniform_sphere(rng, q)
    n = np.tile(np.array([[0.3, -0.4, np.sqrt(0.75)]]), (q, 1))
    p = O.mis_eval(g, slot, t, np.array([0.35]), np.full((q, 3), 0.5, np.float32), n, d) * 4 * np.pi
    assert abs(p.mean() - 1.0) < 5 * p.std() / math.sqrt(q)


def test_mis_sample_is_unbiased_and_selects_with_alpha():
    # One-sample MIS estimator of a known integral: E[f(w) / p_MIS(w)] with
    # f = (1 + z)^2 over the sphere is 16 pi / 3 (the guide map is positive
    # everywhere, so the mixture covers the sphere).
    g, slot, t = _mis_setup()
    q, alpha = 200000, 0.35
    pos = np.full((q, 3), 0.5, np.float32)
    rng = np.random.default_rng(23)
    n = synth.uniform_sphere(rng, q)
    s = O.mis_sample(g, slot, t, np.array([alpha]), pos, n, seed=77, stream=2)
    f = (1.0 + s["dir"][:, 2]) ** 2 / s["pdf"]
    assert abs(f.mean() - 16 * np.pi / 3) < 5 * f.std() / math.sqrt(q)
    k = int((s["strategy"] == 0).sum())
    assert abs(k - alpha * q) < 5 * math.sqrt(q * alpha * (1 - alpha))
    # The guided branch draws exactly the guide's sample for the same query.
    gd = O.sample(g, slot, t, pos, seed=77, stream=2)["dir"]
    sel = s["strategy"] == 1
    assert np.array_equal(s["dir"][sel], gd[sel])
    bs = ~sel
    assert np.all(np.sum(n[bs] * s["dir"][bs], axis=1) >= -1e-12)
    assert np.allclose(s["pdf"], O.mis_eval(g, slot, t, np.array([alpha]), pos, n, s["dir"]), rtol=1e-14)


def test_mis_leaves_without_map_use_bsdf_only():
    ph = synth.photons(2000, 2, 20)
    g = O.build_grid(ph, LO, HI, 3, 0, 50)
    act, slot = O.active_leaves(g)
    t = O.tables_from_map(np.ones((act.size, 8, 8)))
    pos = synth.query_positions(4000, 20)
    rng = np.random.default_rng(24)
    n = synth.uniform_sphere(rng, pos.shape[0])
    s = O.mis_sample(g, slot, t, np.full(g["L"], 0.2), pos, n, seed=3)
    leaf, _ = O.leaf_of_positions(g, pos)
    empty = slot[leaf] < 0
    assert empty.any() and (~empty).any()
    assert np.all(s["strategy"][empty] == 0) and np.all(s["alpha"][empty] == 1.0)
    c = np.sum(n * s["dir"], axis=1)
    assert np.allclose(s["pdf"][empty], c[empty] / np.pi, rtol=1e-12)


# ---------------------------------------------------------------- progressive iterations (Sec. 7.1, 7.2)
def test_split_threshold_schedule_hand_values():
    # Sec. 8: M_thr = c sqrt(2^t) with c = 500.
    assert [O.split_threshold(t) for t in range(5)] == [500, 707, 1000, 1414, 2000]
    assert [O.split_threshold(t, 400.0) for t in range(3)] == [400, 565, 800]


def _leaf_by_range(g, codes):
    """Leaf of each code by direct range membership: leaf l holds the codes
    [start_l, start_l + 8^(D - depth_l))."""
    D = g["D"]
    out = np.full(len(codes), -1)
    for l in range(g["L"]):
        a = int(g["leaf_code"][l])
        b = a + 8 ** (D - int(g["leaf_depth"][l]))
        for i, c in enumerate(codes):
            if a <= int(c) < b:
                assert out[i] == -1
                out[i] = l
    assert np.all(out >= 0)
    return out


def _batches(sizes, seed):
    ph = synth.photons(sum(sizes), 3, seed)
    ends = np.cumsum(sizes)
    return [ph[e - n:e] for n, e in zip(sizes, ends)]


def test_progressive_refinement_rebuilds_from_all_photons():
    # Two refining iterations (c = 20: thresholds 20 then 28) on 150 + 300 photons.
    b = _batches([150, 300], 31)
    pr = O.Progressive(LO, HI, 3, 0, 4, 8, 450, split_c=20.0, refine_iterations=2)
    pr.add_photons(b[0])
    pr.add_photons(b[1])
    allp = np.concatenate(b)
    g = pr.grid
    q = [_deinterleave(c, 3) for c in O.morton_codes(allp, LO, HI, 3)[0]]
    leaves = _brute_grid(q, 3, 0, 28)
    assert g["L"] == len(leaves) and pr.t == 2
    for l, (c, d, idx) in enumerate(leaves):
        assert g["leaf_depth"][l] == d
    # Current planes: every photon; previous planes: the first iteration's.
    pc, cc, pp, cp, _ = _brute_splat(allp, g, 150, 4, 8, 32)
    assert pr.pow_cur.tolist() == pc and pr.cnt_cur.tolist() == cc
    assert pr.pow_prev.tolist() == pp and pr.cnt_prev.tolist() == cp
    assert pr.updated.tolist() == [l for l in range(g["L"]) if sum(cc[l]) > 0]
    assert pr.stored.shape[0] == 0 and pr.status == 0  # the grid is fixed from here on


def test_progressive_accumulation_matches_recount():
    # One refining iteration, then three batches binned into the fixed leaves.
    H, W, F = 4, 8, 32
    b = _batches([400, 200, 400, 800], 32)
    pr = O.Progressive(LO, HI, 4, 1, H, W, 1800, split_c=30.0, refine_iterations=1)
    seen = []
    for t, ph in enumerate(b):
        before = (pr.pow_cur.copy(), pr.cnt_cur.copy()) if t else None
        pr.add_photons(ph)
        seen.append(ph)
        g = pr.grid
        allp = np.concatenate(seen)
        it = np.concatenate([np.full(len(x), k) for k, x in enumerate(seen)])
        leaf = _leaf_by_range(g, O.morton_codes(allp, LO, HI, 4)[0])
        rows, cols, _ = O.dir_bins(allp[:, 3:6], H, W)
        pfx = [int(v) for v in np.rint(allp[:, 6].astype(np.float64) * 2.0 ** F)]
        L = g["L"]
        cur = [[0] * (H * W) for _ in range(L)]
        cnt = [[0] * (H * W) for _ in range(L)]
        prev = [[0] * (H * W) for _ in range(L)]
        cprev = [[0] * (H * W) for _ in range(L)]
        last = [max([int(it[i]) for i in range(len(allp)) if leaf[i] == l], default=-1) for l in range(L)]
        for i in range(len(allp)):
            l, k = int(leaf[i]), int(rows[i] * W + cols[i])
            cur[l][k] += pfx[i]
            cnt[l][k] += 1
            if t == 0 or it[i] < last[l]:  # before the leaf's last update (all earlier for the refine)
                if t > 0 or it[i] < 0:
                    prev[l][k] += pfx[i]
                    cprev[l][k] += 1
        assert pr.status == 0
        assert pr.pow_cur.tolist() == cur and pr.cnt_cur.tolist() == cnt
        if t > 0:
            assert pr.pow_prev.tolist() == prev and pr.cnt_prev.tolist() == cprev
            assert pr.updated.tolist() == sorted({int(leaf[i]) for i in range(len(allp)) if it[i] == t})
            untouched = np.setdiff1d(np.arange(L), pr.updated)
            assert np.array_equal(pr.pow_cur[untouched], before[0][untouched])
        # Eq. (photon): the maps hold every photon's power, exactly.
        assert sum(int(v) for v in pr.pow_cur.ravel()) == sum(pfx)


def test_progressive_maps_change_only_where_photons_arrive():
    H, W = 8, 8
    net = O.parse_net(synth.net_blob(synth.ARCH_TINY3, (4,), 5))
    b = _batches([500, 100, 1000], 33)
    pr = O.Progressive(LO, HI, 3, 1, H, W, 1600, split_c=40.0, refine_iterations=1)
    pr.add_photons(b[0])
    t0 = pr.reconstruct(net)
    m0 = pr.maps.copy()
    assert np.all(t0["valid"][pr.updated] == 1)
    pr.add_photons(b[1])
    pr.reconstruct(net)
    other = np.setdiff1d(np.arange(pr.grid["L"]), pr.updated)
    assert other.size and pr.updated.size
    assert np.array_equal(pr.maps[other], m0[other])
    assert not np.array_equal(pr.maps[pr.updated], m0[pr.updated])


def test_progressive_without_refinement_uses_the_regular_grid():
    pr = O.Progressive(LO, HI, 5, 2, 4, 4, 900, refine_iterations=0)
    assert pr.grid["L"] == 64 and np.all(pr.grid["leaf_depth"] == 2)
    for ph in _batches([300, 600], 34):
        pr.add_photons(ph)
    assert int(pr.cnt_cur.sum()) == 900 and pr.grid["L"] == 64


# ---------------------------------------------------------------- the paper's grid rule (Sec. 7.1)
def _kd_photons(xyz):
    ph = np.zeros((len(xyz), 8), np.float32)
    ph[:, :3] = xyz
    ph[:, 5] = 1.0
    ph[:, 6] = 1.0
    return ph


def test_kd_median_splits_hand_example():
    ph = _kd_photons([[0.4, 0.5, 0.5], [0.1, 0.5, 0.5], [0.3, 0.5, 0.5], [0.2, 0.5, 0.5]])
    g = O.build_kd_grid(ph, None, LO, HI, 1, 2, 1, 1.0)
    # Root splits at the 2nd smallest x (0.3), each child at its 1st (0.2 and 0.4).
    assert g["node_link"].tolist() == [1, 3, 5, ~0, ~1, ~2, ~3]
    assert g["node_tau"][:3].tolist() == [np.float32(0.3), np.float32(0.2), np.float32(0.4)]
    assert g["node_axis"][:3].tolist() == [0, 0, 0]
    assert g["L"] == 4 and g["leaf_depth"].tolist() == [2, 2, 2, 2]
    assert g["perm"].tolist() == [1, 3, 2, 0]  # leaves in x order
    assert g["leaf_of"].tolist() == [3, 0, 2, 1]


def test_kd_ties_go_left_and_flat_nodes_stay_leaves():
    ph = _kd_photons([[0.2, 0.5, 0.5], [0.7, 0.5, 0.5], [0.2, 0.5, 0.5], [0.2, 0.5, 0.5]])
    g = O.build_kd_grid(ph, None, LO, HI, 1, 8, 1, 1.0)
    # The median (0.2) is the minimum: tau is the next float, so x <= 0.2 goes left.
    assert g["node_tau"][0] == np.nextafter(np.float32(0.2), np.float32(1.0))
    assert g["L"] == 2 and (g["leaf_end"] - g["leaf_begin"]).tolist() == [3, 1]


def test_kd_normal_variance_hand_values():
    u = 2 ** O.KD_NORMAL_BITS
    assert O.kd_normal_variance([u, u, 0], 2) == 0.5
    assert O.kd_normal_variance([u, u, u], 3) == pytest.approx(2 / 3, rel=1e-15)
    assert O.kd_normal_variance([5 * u, 0, 0], 5) == 0.0
    # Two photons on perpendicular walls: V = 0.5, not above V_thr = 0.5.
    ph = _kd_photons([[0.2, 0.3, 0.5], [0.6, 0.7, 0.5]])
    nrm = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    assert O.build_kd_grid(ph, nrm, LO, HI, 1, 8, 100, 0.5)["L"] == 1
    # Three photons on three perpendicular walls: V = 2/3 > 0.5 splits.
    ph = _kd_photons([[0.2, 0.3, 0.5], [0.6, 0.7, 0.5], [0.9, 0.1, 0.5]])
    nrm = np.eye(3, dtype=np.float32)
    g = O.build_kd_grid(ph, nrm, LO, HI, 1, 8, 100, 0.5)
    assert g["L"] > 1 and g["node_link"][0] >= 0


def test_kd_without_splits_is_the_regular_grid():
    R = 5
    ph = synth.photons(3000, 4, 41)
    g = O.build_kd_grid(ph, None, LO, HI, R, 8, 10 ** 9, 2.0)
    assert g["L"] == R ** 3 and g["leaf_cell"].tolist() == list(range(R ** 3))
    t = ph[:, :3].astype(np.float64) * R
    far = np.all(np.abs(t - np.round(t)) > 1e-4, axis=1)
    q = np.floor(t).astype(np.int64)
    cell = q[:, 0] + R * (q[:, 1] + R * q[:, 2])
    assert np.array_equal(g["leaf_of"][far], cell[far])


def _kd_node_range(g, v):
    link = int(g["node_link"][v])
    if link < 0:
        return int(g["leaf_begin"][~link]), int(g["leaf_end"][~link])
    return _kd_node_range(g, link)[0], _kd_node_range(g, link + 1)[1]


@pytest.mark.parametrize("n,R,depth,thr,normals,seed", [(4000, 3, 8, 40, False, 42), (3000, 2, 5, 60, True, 43),
                                                         (2000, 4, 3, 10, True, 44)])
def test_kd_grid_brute_properties(n, R, depth, thr, normals, seed):
    ph = synth.photons(n, 6, seed)
    nrm = None
    if normals:  # a unit normal per photon, from a few directions
        rng = np.random.default_rng(seed)
        nrm = synth.uniform_sphere(rng, 5)[rng.integers(0, 5, n)].astype(np.float32)
    g = O.build_kd_grid(ph, nrm, LO, HI, R, depth, thr, 0.5)
    L = g["L"]
    # Leaves partition the photons, in ascending ranges.
    assert g["leaf_begin"][0] == 0 and g["leaf_end"][-1] == n
    assert np.array_equal(g["leaf_begin"][1:], g["leaf_end"][:-1])
    assert sorted(g["perm"].tolist()) == list(range(n))
    # Locating a photon by descent finds the leaf that holds it.
    loc, _ = O.kd_locate(g, ph[:, :3])
    assert np.array_equal(loc, g["leaf_of"].astype(np.int64))
    for l in range(L):
        assert np.all(g["leaf_of"][g["perm"][g["leaf_begin"][l]:g["leaf_end"][l]]] == l)
    # Every node against its photons: the split rule, the axis, the median.
    u = 2 ** O.KD_NORMAL_BITS
    nfx = np.rint(nrm.astype(np.float64) * u).astype(np.int64) if normals else None
    stack = [(c, 0) for c in range(R ** 3)]
    while stack:
        v, d = stack.pop()
        b, e = _kd_node_range(g, v)
        idx = g["perm"][b:e]
        P = ph[idx, :3]
        m = e - b
        spread = (P.max(axis=0) - P.min(axis=0)) if m else np.zeros(3, np.float32)
        V = O.kd_normal_variance(nfx[idx].sum(axis=0).tolist(), m) if (normals and m) else 0.0
        want = d < depth and m >= 2 and spread.max() > 0 and (m > thr or V > 0.5)
        link = int(g["node_link"][v])
        assert (link >= 0) == want, (v, d, m)
        if link < 0:
            continue
        a = int(g["node_axis"][v])
        assert spread[a] == spread.max() and np.all(spread[:a] < spread[a])
        x = np.sort(P[:, a])
        s = x[m // 2]
        tau = g["node_tau"][v]
        assert tau == (s if x[0] < s else np.nextafter(s, np.float32(np.inf)))
        nl = int((P[:, a] < tau).sum())
        assert 0 < nl < m and _kd_node_range(g, link) == (b, b + nl)
        # The left part keeps the photons' order (a stable partition).
        assert np.all(np.diff(np.nonzero(np.isin(g["perm"][b:e], idx[P[:, a] < tau]))[0]) == 1)
        stack += [(link, d + 1), (link + 1, d + 1)]


# ---------------------------------------------------------------- the paper-style network (Sec. 5.1)
@pytest.mark.parametrize("dil,stride", [(2, 1), (4, 1), (2, 2)])
def test_dilated_conv_matches_torch(dil, stride):
    rng = np.random.default_rng(50 + dil)
    x = rng.standard_normal((2, 12, 16, 5))
    w = rng.standard_normal((4, 3, 3, 5)).astype(np.float32)
    b = rng.standard_normal(4).astype(np.float32)
    y = O.conv2d(x, w, b, stride, dil)
    ref = Fnn.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2), torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                     torch.from_numpy(b.astype(np.float64)), stride=stride, padding=dil, dilation=dil)
    assert np.allclose(y, ref.permute(0, 2, 3, 1).numpy(), rtol=1e-12, atol=1e-12)


def test_partial_conv_mask_hand_values():
    m = np.zeros((1, 5, 5))
    m[0, 2, 2] = 1.0
    scale, mo = O.pconv_mask(m, 3, 1, 1)
    want = np.zeros((5, 5))
    want[1:4, 1:4] = 9.0  # one valid pixel under each of these windows
    assert np.array_equal(scale[0], want) and np.array_equal(mo[0], (want > 0).astype(float))
    scale, _ = O.pconv_mask(m, 3, 1, 2)
    want = np.zeros((5, 5))
    for y in (0, 2, 4):
        for x in (0, 2, 4):
            want[y, x] = 9.0
    assert np.array_equal(scale[0], want)
    full, _ = O.pconv_mask(np.ones((1, 4, 4)), 3, 1, 1)
    assert full[0, 1, 1] == 1.0 and full[0, 0, 0] == 9 / 4 and full[0, 0, 1] == 9 / 6


def test_partial_conv_matches_the_definition():
    """W^T (X * M) * sum(1) / sum(M) + b over each window (Liu et al. 2018),
    written as plain loops."""
    rng = np.random.default_rng(53)
    A, H, W, C, O_ = 2, 6, 7, 3, 2
    m = (rng.random((A, H, W)) < 0.4).astype(float)
    x = rng.standard_normal((A, H, W, C)) * m[..., None]
    w = rng.standard_normal((O_, 3, 3, C)).astype(np.float32)
    b = rng.standard_normal(O_).astype(np.float32)
    y, mo = O.pconv(x, m, w, b, 1, 2, 0)
    for a in range(A):
        for i in range(H):
            for j in range(W):
                acc, cnt = np.zeros(O_), 0.0
                for ky in range(3):
                    for kx in range(3):
                        yy, xx = i + 2 * (ky - 1), j + 2 * (kx - 1)
                        if 0 <= yy < H and 0 <= xx < W and m[a, yy, xx]:
                            cnt += 1
                            acc += w[:, ky, kx, :].astype(np.float64) @ x[a, yy, xx]
                want = acc * 9.0 / cnt + b if cnt else np.zeros(O_)
                assert np.allclose(y[a, i, j], want, rtol=1e-12, atol=1e-12)
                assert mo[a, i, j] == (cnt > 0)


def test_residual_link_and_masked_zeros():
    rng = np.random.default_rng(54)
    m = (rng.random((1, 8, 8)) < 0.3).astype(float)
    r = rng.standard_normal((1, 8, 8, 4)) * m[..., None]
    y, _ = O.pconv(r, m, np.zeros((4, 3, 3, 4), np.float32), np.zeros(4, np.float32), 1, 1, O.ACT_ELU, r)
    assert np.array_equal(y, r)  # ELU(0) + r
    # Through the whole network: every layer's output vanishes outside its mask;
    # with every bin valid the first layer is an ordinary conv away from the border.
    net = O.parse_net(synth.net_blob(synth.ARCH_PAPER, (8, 16), 55))
    x = rng.random((2, 16, 16, 5))
    x[..., 4] = 1.0
    cout, cin, k, stride, act, w, b = net["layers"][0]
    y0, _ = O.pconv(x, x[..., 4], w, b, 1, 1, act)
    plain = O.elu(O.conv2d(x, w, b, 1))
    assert np.allclose(y0[:, 1:-1, 1:-1], plain[:, 1:-1, 1:-1], rtol=1e-12, atol=1e-12)
    x[..., 4] = (rng.random((2, 16, 16)) < 0.05)
    x[..., :4] *= x[..., 4:5]
    out = O.cnn_forward(x, net)
    assert out.shape == (2, 16, 16) and np.all(np.isfinite(out)) and np.all(out >= 0)


def _torch_paper_net(x, net):
    """The paper-style masked U-Net wired from its layer table with
    torch.nn.functional in float64 (library pin of the wiring).

    Partial convolution (Liu et al. 2018): conv2d of the masked input, scaled
    by 9 / (valid pixels under the window) counted by conv2d of the mask with
    a ones kernel, plus the bias where that count is positive, else 0.  The
    output mask is a 3x3 max-pool of the input mask (same stride, spacing and
    padding as the layer).  Residual links are explicit adds after the ELU;
    decoder levels concatenate [nearest x2 upsample, skip] along channels, and
    their mask is the elementwise max (union) of the two parts' masks."""
    Ls, dil = net["layers"], net["dil"]
    t = torch.from_numpy(x).permute(0, 3, 1, 2).contiguous()

    def pconv(h, m, i, res=None):
        cout, cin, k, stride, act, w, b = Ls[i]
        d = dil[i]
        wt = torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2)
        y = Fnn.conv2d(h * m, wt, None, stride=stride, padding=d * (k // 2), dilation=d)
        cnt = Fnn.conv2d(m, torch.ones(1, 1, k, k, dtype=torch.float64), None, stride=stride,
                         padding=d * (k // 2), dilation=d)
        bias = torch.from_numpy(b.astype(np.float64)).view(1, -1, 1, 1)
        y = torch.where(cnt > 0, y * (k * k) / cnt.clamp(min=1.0) + bias, torch.zeros_like(y))
        y = Fnn.elu(y)
        if res is not None:
            y = y + res
        pad = d * (k // 2)  # masks are >= 0, so zero padding leaves the max unchanged
        m_out = Fnn.max_pool2d(Fnn.pad(m, (pad, pad, pad, pad)), k, stride=stride, dilation=d)
        return y, m_out

    up = lambda h: Fnn.interpolate(h, scale_factor=2, mode="nearest")
    m = t[:, 4:5]
    a0, m = pconv(t, m, 0)
    e0, me0 = pconv(a0, m, 1, a0)
    a1, m = pconv(e0, me0, 2)
    e1, me1 = pconv(a1, m, 3, a1)
    b0, m = pconv(e1, me1, 4)
    b1, m = pconv(b0, m, 5, b0)
    b2, m = pconv(b1, m, 6, b1)
    d1, m = pconv(torch.cat([up(b2), e1], 1), torch.maximum(up(m), me1), 7)
    d1, m = pconv(d1, m, 8, d1)
    d0, m = pconv(torch.cat([up(d1), e0], 1), torch.maximum(up(m), me0), 9)
    d0, _ = pconv(d0, m, 10, d0)
    cout, cin, k, stride, act, w, b = Ls[11]
    y = Fnn.conv2d(d0, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2),
                   torch.from_numpy(b.astype(np.float64)))
    return Fnn.softplus(y)[:, 0].numpy()


@pytest.mark.parametrize("H,W,density", [(16, 16, 0.15), (32, 16, 0.05), (32, 32, 0.6)])
def test_paper_net_matches_torch_wiring(H, W, density):
    """The whole paper-style network as wired, on sparse masks: a slip in the
    oracle's skip order, mask union, mask pyramid or residual positions moves
    bins that this independent torch build does not."""
    net = O.parse_net(synth.net_blob(synth.ARCH_PAPER, (8, 16), 56))
    rng = np.random.default_rng(57 + H + W)
    A = 3
    mask = (rng.random((A, H, W)) < density).astype(np.float64)
    x = rng.random((A, H, W, 5)) * 2.0
    x[..., 4] = mask
    x[..., :4] *= mask[..., None]
    got = O.cnn_forward(x, net)
    ref = _torch_paper_net(x, net)
    assert got.shape == ref.shape == (A, H, W) and np.all(ref > 0)
    # Compared in log space: for a logit v << 0 softplus(v) ~ e^v, so an FP64
    # rounding of v from another summation order becomes a relative error of
    # |v| * 2^-52 on the map (about 1e-10 at v = -73 in the dense case).
    assert np.allclose(np.log(got), np.log(ref), rtol=0, atol=1e-9)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-300)


def test_paper_net_torch_pin_detects_wiring_slips():
    """The torch build above tells the oracle's wiring from plausible slips:
    the skip halves swapped, the concatenation's mask taken from the skip
    alone, or a residual dropped, each changes the map."""
    net = O.parse_net(synth.net_blob(synth.ARCH_PAPER, (8, 16), 58))
    rng = np.random.default_rng(59)
    mask = np.zeros((2, 32, 32))
    mask[0, 3, 5] = mask[0, 20, 25] = mask[1, 10, 10] = mask[1, 11, 12] = 1.0  # masks stay sparse down the levels
    x = rng.random((2, 32, 32, 5))
    x[..., 4] = mask
    x[..., :4] *= mask[..., None]
    ref = _torch_paper_net(x, net)
    L = net["layers"]

    def variant(swap_skip=False, skip_mask_only=False, drop_res=False):
        def run(h, m, i, res=None):
            cout, cin, k, stride, act, w, b = L[i]
            return O.pconv(h, m, w, b, stride, net["dil"][i], act, None if drop_res and i == 8 else res)
        m0 = x[..., 4]
        a0, m1 = run(x[..., :5], m0, 0)
        e0, me0 = run(a0, m1, 1, a0)
        a1, m3 = run(e0, me0, 2)
        e1, me1 = run(a1, m3, 3, a1)
        b0, m5 = run(e1, me1, 4)
        b1, m6 = run(b0, m5, 5, b0)
        b2, m7 = run(b1, m6, 6, b1)
        parts = [e1, O.upsample2(b2)] if swap_skip else [O.upsample2(b2), e1]
        mk = me1 if skip_mask_only else np.maximum(O.upsample2(m7[..., None])[..., 0], me1)
        d1, md1 = run(np.concatenate(parts, axis=3), mk, 7)  # both halves are c1 wide here
        d1b, md1b = run(d1, md1, 8, d1)
        c0 = np.concatenate([O.upsample2(d1b), e0], axis=3)
        d0, md0 = run(c0, np.maximum(O.upsample2(md1b[..., None])[..., 0], me0), 9)
        d0b, _ = run(d0, md0, 10, d0)
        cout, cin, k, stride, act, w, b = L[11]
        return O._act(O.conv2d(d0b, w, b, stride), act)[..., 0]

    assert np.allclose(variant(), ref, rtol=1e-9, atol=1e-300)
    for kw in ({"swap_skip": True}, {"skip_mask_only": True}, {"drop_res": True}):
        assert not np.allclose(variant(**kw), ref, rtol=1e-6, atol=0), kw


def test_progressive_with_the_papers_grid_rule_and_slots():
    """Refinement by the paper's rule (two iterations, normals), then batches
    binned by walking the voxels' trees; map slots: refined leaves in leaf
    order, later newcomers appended in leaf order."""
    H, W = 4, 8
    b = _batches([300, 600, 900, 900], 35)
    nrm = [synth.wall_normals(x) for x in b]
    pr = O.Progressive(LO, HI, 6, 0, H, W, 2700, split_c=40.0, refine_iterations=2, grid_rule="kd", R=4, vthr=0.5)
    pr.add_photons(b[0], nrm[0])
    pr.add_photons(b[1], nrm[1])
    ref = O.build_kd_grid(np.concatenate(b[:2]), np.concatenate(nrm[:2]), LO, HI, 4, 6, O.split_threshold(1, 40.0),
                          0.5)
    for k in ("leaf_cell", "leaf_depth", "node_link", "node_tau"):
        assert np.array_equal(pr.grid[k], ref[k]), k
    act, _ = O.active_leaves(ref)
    assert pr.slot_leaf == list(act) and np.array_equal(pr.updated_slots, np.arange(act.size))
    total = O.bin_batch(ref, np.concatenate(b[:2]), H, W, 32, n_bound=2700)
    assert np.array_equal(pr.pow_cur, total["pow_cur"]) and np.array_equal(pr.cnt_cur, total["cnt_cur"])
    A = len(pr.slot_leaf)
    seen = list(b[:2])
    for t in (2, 3):
        pr.add_photons(b[t], nrm[t])
        seen.append(b[t])
        total = O.bin_batch(ref, np.concatenate(seen), H, W, 32, n_bound=2700)
        assert np.array_equal(pr.pow_cur, total["pow_cur"]) and np.array_equal(pr.cnt_cur, total["cnt_cur"])
        leaf, _ = O.leaf_of_positions(ref, b[t][:, :3])
        assert pr.updated.tolist() == sorted(set(leaf.tolist()))
        new = [l for l in pr.updated if l not in pr.slot_leaf[:A]]
        assert pr.slot_leaf[A:] == new and list(pr.updated_slots) == [pr.slot_leaf.index(l) for l in pr.updated]
        A = len(pr.slot_leaf)
