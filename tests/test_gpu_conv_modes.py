"""Operand staging modes of the tensor-core convolutions.

Modes 1 (three x-shifted haloed boxes) and 2 (one box of zero-padded rows,
outputs in the padded row space, every tap a descriptor starting at another
row of the same box) issue the same MMAs in the same K order (channel chunk,
tap, K step) for every output pixel.  Mode 4 reads a stride-2 layer's input
as pixel pairs (kernel row by kernel row: tap 0 from the second pixel of the
pairs at x - 1, taps 1 and 2 from the pairs at x) and issues mode 0's MMAs
in mode 0's order.  With the 3-layer net, whose one 3x3
layer is eligible for both, the maps must be bit-identical.  In the U-Net
the modes' eligibility differs per layer, and a layer that falls back to
mode 0 sums its taps in another order, so there the maps agree to the
accumulation order.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

N = 300_000


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = pg.Context()
    ph = torch.from_numpy(synth.photons(N, 16, 901)).cuda()
    g = pg.pg_build_grid(c, ph, N, [0, 0, 0], [1, 1, 1], 8, 0, 4000)
    yield c, ph, g
    c.destroy()


def _maps(ctx, net, h, prec, mode):
    os.environ["PG_TC_FORCE"] = str(mode)
    try:
        m = pg.pg_reconstruct(ctx, h, net, prec)
        ctx.sync()
        return pg.export_map(m)
    finally:
        del os.environ["PG_TC_FORCE"]


@pytest.mark.parametrize("size,prec", [(32, pg.PG_BF16), (64, pg.PG_BF16), (128, pg.PG_BF16),
                                       (32, pg.PG_FP8_E4M3), (64, pg.PG_FP8_E4M3)])
def test_padded_rows_equal_shifted_boxes_bit_for_bit(setup, size, prec):
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, size, size)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_TINY3, (32,), 902))
    y1 = _maps(ctx, net, h, prec, 1)
    y2 = _maps(ctx, net, h, prec, 2)
    assert np.isfinite(y2).all() and (y2 >= 0).all()
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("size,prec", [(64, pg.PG_BF16), (128, pg.PG_BF16), (64, pg.PG_FP8_E4M3)])
def test_unet_modes_agree(setup, size, prec):
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, size, size)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 903))
    y0 = _maps(ctx, net, h, prec, 0)
    y1 = _maps(ctx, net, h, prec, 1)
    y2 = _maps(ctx, net, h, prec, 2)
    for y in (y1, y2):
        assert np.abs(y - y0).sum() / np.abs(y0).sum() < 1e-3
    # Mode 4 (pixel pairs) serves the stride-2 layer over 32 BF16 channels
    # (the other layers run mode 0); it issues mode 0's MMAs in mode 0's K
    # order, so the maps are the same bit for bit.
    y4 = _maps(ctx, net, h, prec, 4)
    assert np.array_equal(y4, y0)


def test_staged_and_direct_output_stores_agree(setup):
    # The epilogue's store paths write the same bytes: staged through shared
    # memory (coalesced), each lane straight to its pixel, or bulk copies.
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, 64, 64)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 905))
    for prec in (pg.PG_BF16, pg.PG_FP8_E4M3):
        for mode, mt in ((0, 2), (2, 2), (2, 1), (2, 4)):
            # One CTA per SM and two stages: every store path fits in shared
            # memory.  Path 2 (bulk async copies of whole pixel runs) serves
            # the padded-row layers with dense 32-channel BF16 outputs.
            paths = (0, 1, 2) if mode == 2 and prec == pg.PG_BF16 else (0, 1)
            ys = [_maps(ctx, net, h, prec, f"{mode},0,{mt},1,2,{so}") for so in paths]
            for y in ys[1:]:
                assert np.array_equal(ys[0], y), (prec, mode, mt)


def test_tuning_round_trip(setup):
    # Launch shapes chosen by the autotuner load into a fresh copy of the net
    # and reproduce its maps bit for bit.
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, 64, 64)
    blob = synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 904)
    a = pg.pg_net_load(ctx, blob)
    pg.pg_autotune(ctx, h, a, pg.PG_BF16)
    tun = pg.pg_net_get_tuning(a)
    assert tun.size == 15 * 3 * 7 and (tun.reshape(15, 3, 7)[:14, 1, 5] == 64 * 64).all()
    b = pg.pg_net_load(ctx, blob)
    pg.pg_net_set_tuning(b, tun)
    assert np.array_equal(pg.pg_net_get_tuning(b), tun)
    ya = pg.export_map(pg.pg_reconstruct(ctx, h, a, pg.PG_BF16))
    yb = pg.export_map(pg.pg_reconstruct(ctx, h, b, pg.PG_BF16))
    assert np.array_equal(ya, yb)
    bad = tun.copy()
    bad[3] = 7  # no such staging mode
    with pytest.raises(pg.PgError):
        pg.pg_net_set_tuning(b, bad)


def _unset(name):
    os.environ.pop(name, None)


@pytest.mark.parametrize("size", [64, 128])
def test_phase_form_matches_the_concatenation(setup, size):
    """A decoder layer over [upsample2(U), S] runs in the phase form: four 2x2
    convolutions of the half-resolution U (one per output phase, each tap the
    sum of the 3x3 taps that land on the same upsampled pixel) plus the 3x3
    taps of S read as four parity sub-grids.  Its maps equal those of the
    explicit x2 upsample into the concatenation up to the BF16 rounding of
    the summed weights and the accumulation order."""
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, size, size)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 906))
    y_ph = pg.export_map(pg.pg_reconstruct(ctx, h, net, pg.PG_BF16))
    os.environ["PG_TC_NO_PHASE"] = "1"
    try:
        y_cat = pg.export_map(pg.pg_reconstruct(ctx, h, net, pg.PG_BF16))
    finally:
        _unset("PG_TC_NO_PHASE")
    assert np.isfinite(y_ph).all() and (y_ph >= 0).all()
    assert not np.array_equal(y_ph, y_cat)  # the phase form did run
    assert np.abs(y_ph - y_cat).sum() / np.abs(y_cat).sum() < 5e-3
    p = y_ph.reshape(len(y_ph), -1) / y_ph.reshape(len(y_ph), -1).sum(axis=1, keepdims=True)
    q = y_cat.reshape(len(y_cat), -1) / y_cat.reshape(len(y_cat), -1).sum(axis=1, keepdims=True)
    kl = (q * np.log(np.maximum(q, 1e-30) / np.maximum(p, 1e-30))).sum(axis=1)
    assert kl.max() < 1e-4, kl.max()


@pytest.mark.parametrize("size", [64, 128])
def test_phase_tiles_of_one_two_or_four_phases_agree_bit_for_bit(setup, size):
    # Every output phase gets the same MMAs in the same K order (skip chunks,
    # taps, then upsampled chunks, 2x2 taps) whether a tile holds one, two or
    # four phases, so the maps are bit-identical.
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, size, size)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 907))
    ys = [_maps(ctx, net, h, pg.PG_BF16, f"3,32,{mt},0,0,0") for mt in (1, 2, 4)]
    assert np.isfinite(ys[0]).all()
    for y in ys[1:]:
        assert np.array_equal(ys[0], y)


@pytest.mark.parametrize("size,prec,mode", [(64, pg.PG_BF16, None), (64, pg.PG_BF16, 0), (64, pg.PG_BF16, 1),
                                            (128, pg.PG_BF16, None), (64, pg.PG_FP8_E4M3, None),
                                            (64, pg.PG_FP8_E4M3, 1)])
def test_weight_images_equal_per_block_loads_bit_for_bit(setup, size, prec, mode):
    # A stage's weights arrive by one bulk copy of the layer's weight image
    # (the blocks as a tensor load lays them out in shared memory) or by one
    # tensor load per block: the same bytes, so the same maps.
    ctx, ph, g = setup
    h = pg.pg_splat_photons(ctx, g, ph, N, N // 2, size, size)
    net = pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), 908))
    if mode is not None:
        os.environ["PG_TC_FORCE"] = str(mode)
    try:
        y_img = pg.export_map(pg.pg_reconstruct(ctx, h, net, prec))
        os.environ["PG_TC_NO_IMAGE"] = "1"
        y_blk = pg.export_map(pg.pg_reconstruct(ctx, h, net, prec))
    finally:
        _unset("PG_TC_NO_IMAGE")
        _unset("PG_TC_FORCE")
    assert np.isfinite(y_img).all()
    assert np.array_equal(y_img, y_blk)
