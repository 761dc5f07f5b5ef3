"""Parity at the full size of the scale workload, in the launch configuration
the bench times (4,194,304 photons, depth 10, split 2000, 64x64 maps, the
32-64-128-256 U-Net in BF16 with autotuned launch shapes, 8,388,608 queries
in one call).

Everything the oracle can afford at this size is compared in full: the grid
(codes, permutation, leaf table, leaf of every photon, active list) and all
four histogram planes, bit for bit.  The CNN is checked on leaves stratified
by photon count against the FP64 oracle at the KL gate; sampling on the
first queries of the full call (the Philox counter is the query index) and
evaluation on a strided sample of all of them, given the GPU's own map.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LO = [0.0, 0.0, 0.0]
HI = [1.0, 1.0, 1.0]
SEED = 20101775
N_CNN_LEAVES = 16
N_SAMPLE = 65_536


@pytest.fixture(scope="module")
def run():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    wl = synth.SCALE
    ph, pos, dirs, blob = synth.workload_inputs(wl)
    n, q = wl.n_photons, wl.n_queries
    ctx = pg.Context()
    d_ph = torch.from_numpy(ph).cuda()
    d_pos = torch.from_numpy(pos).cuda()
    d_dir = torch.from_numpy(dirs).cuda()
    g = pg.pg_build_grid(ctx, d_ph, n, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
    h = pg.pg_splat_photons(ctx, g, d_ph, n, wl.n_prev, wl.H, wl.W, wl.frac_bits)
    net = pg.pg_net_load(ctx, blob)
    pg.pg_autotune(ctx, h, net, pg.PG_BF16)
    m = pg.pg_reconstruct(ctx, h, net, pg.PG_BF16)
    t = pg.pg_build_cdf(ctx, m)
    o_d, o_p = torch.empty(q, 3, device="cuda"), torch.empty(q, device="cuda")
    o_l, o_b = torch.empty(q, dtype=torch.int32, device="cuda"), torch.empty(q, dtype=torch.int32, device="cuda")
    o_e = torch.empty(q, device="cuda")
    pg.pg_sample_dirs(ctx, g, t, d_pos, q, SEED, 0, o_d, o_p, o_l, o_b)
    pg.pg_eval_pdf(ctx, g, t, d_pos, d_dir, q, o_e)
    ctx.sync()
    out = dict(wl=wl, ph=ph, pos=pos, dirs=dirs, blob=blob, grid=pg.export_grid(g), hist=pg.export_hist(h),
               y=pg.export_map(m), dir=o_d.cpu().numpy(), pdf=o_p.cpu().numpy(),
               leaf=o_l.cpu().numpy().view(np.uint32), bin=o_b.cpu().numpy().view(np.uint32),
               ev=o_e.cpu().numpy())
    O.set_threads(0)
    out["ref"] = O.build_grid(ph, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
    yield out
    ctx.destroy()


def test_grid_full_size_bit_exact(run):
    got, ref = run["grid"], run["ref"]
    assert got["L"] == ref["L"]
    for k in ("codes", "perm", "leaf_of", "leaf_code", "leaf_begin", "leaf_end", "leaf_depth"):
        assert np.array_equal(got[k], ref[k]), k
    act, slot = O.active_leaves(ref)
    assert np.array_equal(got["active"], act)
    assert np.array_equal(got["slot_of_leaf"], slot)


def _oracle_hist(run):
    # The oracle's histograms of every active leaf (about 1 GB of planes for
    # all leaves), computed once per module.
    if "hr" not in run:
        wl, ref = run["wl"], run["ref"]
        act, _ = O.active_leaves(ref)
        run["hr"] = O.hist_for_active(O.splat(run["ph"], ref, wl.n_prev, wl.H, wl.W, wl.frac_bits), act)
    return run["hr"]


def test_splat_full_size_bit_exact(run):
    hr = _oracle_hist(run)
    got = run["hist"]
    for k in ("pow_cur", "cnt_cur", "pow_prev", "cnt_prev"):
        assert np.array_equal(got[k], hr[k]), k


def test_cnn_full_size_meets_the_kl_gate(run):
    wl, ref = run["wl"], run["ref"]
    act, _ = O.active_leaves(ref)
    counts = (ref["leaf_end"].astype(np.int64) - ref["leaf_begin"])[act]
    order = np.argsort(counts, kind="stable")
    pick = order[np.linspace(0, order.size - 1, N_CNN_LEAVES).astype(np.int64)]
    hr = O.hist_for_active(_oracle_hist(run), pick)
    yr = O.cnn_forward(O.assemble_inputs(hr), O.parse_net(run["blob"]))
    Pr, _ = O.normalise(yr)
    Pg, _ = O.normalise(run["y"][pick].astype(np.float64))
    Pr, Pg = Pr.reshape(len(pick), -1), Pg.reshape(len(pick), -1)
    kl = (Pr * (np.log(np.maximum(Pr, 1e-300)) - np.log(np.maximum(Pg, 1e-300)))).sum(axis=1)
    assert counts[pick].min() <= 2 and counts[pick].max() >= 1000  # the strata span the counts
    assert kl.mean() <= 1e-3, kl
    assert kl.max() <= 5e-3, kl


def test_sample_and_eval_full_size(run):
    ref = run["ref"]
    act, slot = O.active_leaves(ref)
    tabs = O.tables_from_map(run["y"].astype(np.float64))
    s = O.sample(ref, slot, tabs, run["pos"][:N_SAMPLE], SEED, 0)
    assert np.array_equal(run["leaf"][:N_SAMPLE], s["leaf"])
    same = run["bin"][:N_SAMPLE] == s["bin"]
    assert same.mean() >= 1 - 1e-4
    err = np.abs(run["dir"][:N_SAMPLE].astype(np.float64) - s["dir"])
    assert np.all(err[same, 2] <= 2.4e-7)
    assert np.all(err[same, :2] <= 1e-6)
    # FP32 pdfs within 1e-5 relative; the random net drives some bins below
    # FP32's normal range, hence the absolute floor.
    pdf = run["pdf"][:N_SAMPLE].astype(np.float64)
    assert np.all(np.abs(pdf[same] - s["pdf"][same]) <= 1e-5 * s["pdf"][same] + 1e-35)
    # Evaluation: every 128th query of the full call, and the last one.
    idx = np.unique(np.append(np.arange(0, run["pos"].shape[0], 128), run["pos"].shape[0] - 1))
    er = O.eval_pdf(ref, slot, tabs, run["pos"][idx], run["dirs"][idx])
    e = run["ev"][idx].astype(np.float64)
    assert np.all(np.abs(e - er) <= 1e-5 * er + 1e-35)
