"""Mixture of experts (Sec. 8: one network per range of voxel photon counts).

Every leaf's map from pg_reconstruct_experts must be, bit for bit, the map
pg_reconstruct gives that leaf with the net of its count range alone; the
range of each leaf is taken here from the exported count planes and the
oracle's reading of the paper's count table.  The FP64 oracle's mixture is
also compared on a few leaves of each range (FP32 form).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

N, D, THR, S = 600_000, 4, 2500, 32


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ctx = pg.Context()
    ph = synth.photons(N, 24, 921)
    d = torch.from_numpy(ph).cuda()
    g = pg.pg_build_grid(ctx, d, N, [0, 0, 0], [1, 1, 1], D, 0, THR)
    h = pg.pg_splat_photons(ctx, g, d, N, N // 2, S, S)
    blobs = [synth.net_blob(synth.ARCH_TINY3, (32,), 930 + e) for e in range(5)]
    nets = [pg.pg_net_load(ctx, b) for b in blobs]
    hist = pg.export_hist(h)
    counts = hist["cnt_cur"].sum(axis=1)
    yield ctx, ph, g, h, nets, blobs, hist, counts
    ctx.destroy()


def test_counts_cover_every_range(setup):
    counts = setup[7]
    assert set(O.expert_of(counts).tolist()) == {0, 1, 2, 3, 4}


@pytest.mark.parametrize("prec", [pg.PG_FP32, pg.PG_BF16])
def test_each_leaf_gets_its_experts_map(setup, prec):
    ctx, _, _, h, nets, _, _, counts = setup
    y = pg.export_map(pg.pg_reconstruct_experts(ctx, h, nets, precision=prec))
    e = O.expert_of(counts)
    for k in range(5):
        ref = pg.export_map(pg.pg_reconstruct(ctx, h, nets[k], prec))
        sel = e == k
        assert np.array_equal(y[sel], ref[sel]), k


def test_mixture_matches_fp64_oracle(setup):
    ctx, ph, g, h, nets, blobs, hist, counts = setup
    y = pg.export_map(pg.pg_reconstruct_experts(ctx, h, nets, precision=pg.PG_FP32))
    e = O.expert_of(counts)
    pick = np.concatenate([np.nonzero(e == k)[0][:2] for k in range(5)])
    sub = {key: hist[key][pick] for key in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev")}
    sub["H"], sub["W"] = S, S
    x = O.assemble_inputs(sub)
    yo = O.cnn_forward_experts(x, counts[pick], [O.parse_net(b) for b in blobs])
    P = y[pick].reshape(len(pick), -1).astype(np.float64)
    Po = yo.reshape(len(pick), -1)
    P /= P.sum(axis=1, keepdims=True)
    Po /= Po.sum(axis=1, keepdims=True)
    # The FP32 CNN gate of tests/test_gpu_parity.py.
    assert np.all(np.abs(P - Po) <= 1e-5 * Po + 1e-7 * Po.max(axis=1, keepdims=True))


def test_single_expert_and_bad_bounds(setup):
    ctx, _, _, h, nets, _, _, _ = setup
    y1 = pg.export_map(pg.pg_reconstruct_experts(ctx, h, nets[:1], count_bounds=(), precision=pg.PG_FP32))
    y0 = pg.export_map(pg.pg_reconstruct(ctx, h, nets[0], pg.PG_FP32))
    assert np.array_equal(y1, y0)
    with pytest.raises(pg.PgError) as ei:
        pg.pg_reconstruct_experts(ctx, h, nets[:3], count_bounds=(500, 100))
    assert ei.value.status == 1


@pytest.mark.parametrize("size,widths,tuned", [(32, (16, 32, 64, 128), False), (64, (16, 32, 64, 128), False),
                                               (64, (32, 64, 128, 256), True)])
def test_grouped_unet_experts_one_launch_per_layer(setup, size, widths, tuned):
    """BF16 U-Net experts run as one tensor-core launch per layer over every
    expert's tiles (leaves grouped by expert on the device, no host
    read-back): every leaf's map equals, bit for bit, its expert's network run
    alone, and the call launches one kernel per layer, not one per expert.
    The tuned case gives every expert the first net's autotuned launch shapes,
    which were chosen without the other experts' bias and head tables in
    shared memory."""
    ctx, ph, g, _, _, _, _, _ = setup
    d = torch.from_numpy(ph).cuda()
    h = pg.pg_splat_photons(ctx, g, d, N, N // 2, size, size)
    counts = pg.export_hist(h)["cnt_cur"].sum(axis=1)
    nets = [pg.pg_net_load(ctx, synth.net_blob(synth.ARCH_UNET4, widths, 940 + e)) for e in range(5)]
    if tuned:
        pg.pg_autotune(ctx, h, nets[0], pg.PG_BF16)
        for n in nets[1:]:
            pg.pg_net_set_tuning(n, pg.pg_net_get_tuning(nets[0]))
    for n in nets:  # weight copies made up front, outside the counted call
        pg.export_map(pg.pg_reconstruct(ctx, h, n, pg.PG_BF16))
    ctx.sync()
    l0 = ctx.launch_count()
    y = pg.export_map(pg.pg_reconstruct_experts(ctx, h, nets, precision=pg.PG_BF16))
    launches = ctx.launch_count() - l0
    assert launches <= 20, launches  # counts, grouping, assembly, 14 layers, scatter
    e = O.expert_of(counts)
    assert len(set(e.tolist())) >= 4
    for k in range(5):
        ref = pg.export_map(pg.pg_reconstruct(ctx, h, nets[k], pg.PG_BF16))
        sel = e == k
        assert np.array_equal(y[sel], ref[sel]), k
