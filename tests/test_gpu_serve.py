"""Serving loop on the GPU: every request's results are the same served in a
mix (several workers, scene batches, BF16 and FP8 interleaved) as computed
alone through the single-scene calls; a served BF16 request's maps meet the
reduced-precision gate against the FP64 oracle; a malformed request fails
alone; a request over the HBM budget fails with PG_ERR_OOM while the rest
are served; a waiting request can be cancelled; the shared budget gets a
freed block's bytes back only once the stream has run the free.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2010_01775_gb300 import pg, serve, synth  # noqa: E402

pytestmark = pytest.mark.gpu

NET = synth.net_blob(synth.ARCH_TINY3, (32,), 811)  # 32 channels: 32-byte FP8 rows
POOL_N, POOL_Q = 60_000, 40_000


@pytest.fixture(scope="module")
def pools():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ph = torch.from_numpy(synth.photons(POOL_N, 8, 812)).pin_memory()
    pos = torch.from_numpy(synth.query_positions(POOL_Q, 813)).pin_memory()
    dirs = torch.from_numpy(synth.query_directions(POOL_Q, 813)).pin_memory()
    return ph, pos, dirs


def _requests(pools, k0, count, seed):
    ph, pos, dirs = pools
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(POOL_N))))
        q = int(np.exp(rng.uniform(np.log(1e3), np.log(2e4))))
        o = int(rng.integers(0, POOL_Q - q))
        s = int(rng.choice([16, 32]))
        prec = (pg.PG_BF16, pg.PG_FP8_E4M3)[k % 2]
        out.append(serve.Request(ph[:n], pos[o:o + q], dirs[o:o + q], s, s, prec, max_depth=6, split_threshold=500,
                                 stream_id=k0 + k))
    return out


def _warm(pools):
    ph, pos, dirs = pools
    return [serve.Request(ph[:40_000], pos[:1000], dirs[:1000], s, s, p, max_depth=6, split_threshold=500,
                          stream_id=10_000 + i)
            for i, (s, p) in enumerate([(16, pg.PG_BF16), (32, pg.PG_BF16), (16, pg.PG_FP8_E4M3),
                                        (32, pg.PG_FP8_E4M3)])]


def _alone(ctx, net, seed, r):
    """The request through the single-scene calls on a context of its own."""
    ph = r.photons.cuda()
    pos, din = r.positions.cuda(), r.directions.cuda()
    g = pg.pg_build_grid(ctx, ph, r.n, r.lo, r.hi, r.max_depth, r.min_depth, r.split_threshold)
    h = pg.pg_splat_photons(ctx, g, ph, r.n, r.n // 2, r.H, r.W, r.frac_bits)
    m = pg.pg_reconstruct(ctx, h, net, r.precision)
    t = pg.pg_build_cdf(ctx, m)
    q = r.q
    d = torch.empty(q, 3, device="cuda")
    p = torch.empty(q, device="cuda")
    lf = torch.empty(q, dtype=torch.int32, device="cuda")
    bn = torch.empty(q, dtype=torch.int32, device="cuda")
    e = torch.empty(q, device="cuda")
    pg.pg_sample_dirs(ctx, g, t, pos, q, seed, r.stream_id, d, p, lf, bn)
    pg.pg_eval_pdf(ctx, g, t, pos, din, q, e)
    ctx.sync()
    for x in (t, m, h, g):
        x.free()
    return dict(dirs=d.cpu().numpy(), pdf=p.cpu().numpy(), leaf=lf.cpu().numpy().view(np.uint32),
                bin=bn.cpu().numpy().view(np.uint32), eval_pdf=e.cpu().numpy())


def test_results_same_alone_and_in_the_mix(pools):
    srv = serve.Server(NET, workers=3, hbm_budget=8 << 30, keep_results=True)
    try:
        srv.warmup(_warm(pools))
        rs = [srv.submit(r) for r in _requests(pools, 0, 24, 5)]
        for r in rs:
            assert r.wait(120)
        assert all(r.status == "done" for r in rs), [r.error for r in rs]
        assert max(r.batch_size for r in rs) > 1  # some requests were batched
        ctx = pg.Context()
        for r in rs:
            ref = _alone(ctx, srv.net, srv.seed, r)
            for k in ("dirs", "pdf", "leaf", "bin", "eval_pdf"):
                assert np.array_equal(r.result[k], ref[k]), (r.rid, r.batch_size, k)
        ctx.destroy()
        s = serve.latency_summary(rs)
        assert s["done"] == 24 and s["p99_ms"] >= s["p50_ms"] > 0
    finally:
        srv.close()


def test_malformed_request_fails_alone(pools):
    srv = serve.Server(NET, workers=1, hbm_budget=8 << 30, keep_results=True)
    try:
        srv.warmup(_warm(pools)[:1])
        good = _requests(pools, 100, 6, 6)
        for r in good:
            r.H = r.W = 16
            r.precision = pg.PG_BF16
        bad_ph = good[2].photons.clone()
        bad_ph[5, 4] = float("nan")  # a non-finite direction
        bad = serve.Request(bad_ph, good[2].positions, good[2].directions, 16, 16, pg.PG_BF16, max_depth=6,
                            split_threshold=500, stream_id=999)
        neg = serve.Request(good[3].photons.clone(), good[3].positions, good[3].directions, 16, 16, pg.PG_BF16,
                            max_depth=6, split_threshold=500, stream_id=998)
        neg.photons[7, 6] = -1.0  # negative power
        rs = [srv.submit(r) for r in good[:3] + [bad] + good[3:] + [neg]]
        for r in rs:
            assert r.wait(120)
        assert all(r.status == "done" for r in good), [r.error for r in good]
        assert bad.status == "failed" and bad.error_status == 8, bad.error
        assert neg.status == "failed" and neg.error_status == 8, neg.error
    finally:
        srv.close()


def test_over_budget_request_fails_with_oom_others_served(pools):
    srv = serve.Server(NET, workers=2, hbm_budget=192 << 20, keep_results=False)
    try:
        small = _requests(pools, 200, 6, 7)
        for r in small:
            r.precision = pg.PG_BF16
        ph, pos, dirs = pools
        # 4.8M photons: 154 MB of input fit, the grid's working memory does not.
        big_ph = ph.repeat(80, 1)
        big = serve.Request(big_ph, pos[:1000], dirs[:1000], 16, 16, pg.PG_BF16, max_depth=6, split_threshold=500,
                            stream_id=300)
        rs = [srv.submit(r) for r in small[:3] + [big] + small[3:]]
        for r in rs:
            assert r.wait(120)
        assert all(r.status == "done" for r in small), [r.error for r in small]
        assert big.status == "failed" and big.error_status == 3
        # Everything a request held went back to the budget: only the net remains.
        assert srv.budget.query()[0] == srv._owner.bytes_in_use()
    finally:
        srv.close()


def test_cancel_waiting_request(pools):
    srv = serve.Server(NET, workers=1, hbm_budget=8 << 30)
    try:
        rs = _requests(pools, 400, 8, 8)
        for r in rs:
            r.precision = pg.PG_BF16
        rs = [srv.submit(r) for r in rs]
        last = rs[-1]
        cancelled = srv.cancel(last)
        for r in rs[:-1]:
            assert r.wait(120)
        assert last.wait(120)
        assert last.status == ("cancelled" if cancelled else "done")
        assert all(r.status == "done" for r in rs[:-1])
    finally:
        srv.close()


def test_served_bf16_request_meets_the_gate_against_the_oracle(pools):
    """A BF16 request served in a mix: its results equal the request alone
    (whose tables decide every sample), and the maps of the request alone
    meet the reduced-precision gate, mean KL(P_oracle || P) <= 1e-3 over its
    leaves, against the FP64 oracle's path on the same photons."""
    srv = serve.Server(NET, workers=2, hbm_budget=8 << 30, keep_results=True)
    try:
        srv.warmup(_warm(pools)[:2])
        rs = _requests(pools, 500, 6, 9)
        for r in rs:
            r.precision = pg.PG_BF16
        rs = [srv.submit(r) for r in rs]
        for r in rs:
            assert r.wait(120)
        assert all(r.status == "done" for r in rs), [r.error for r in rs]
        r = max(rs, key=lambda x: x.n)
        ctx = pg.Context()
        ref = _alone(ctx, srv.net, srv.seed, r)
        for k in ("dirs", "pdf", "leaf", "bin", "eval_pdf"):
            assert np.array_equal(r.result[k], ref[k]), k
        ph = r.photons.numpy()
        g = pg.pg_build_grid(ctx, r.photons.cuda(), r.n, r.lo, r.hi, r.max_depth, r.min_depth, r.split_threshold)
        h = pg.pg_splat_photons(ctx, g, r.photons.cuda(), r.n, r.n // 2, r.H, r.W, r.frac_bits)
        m = pg.pg_reconstruct(ctx, h, srv.net, pg.PG_BF16)
        t = pg.pg_build_cdf(ctx, m)
        ctx.sync()
        P = pg.export_tables(t)["P"].reshape(-1, r.H * r.W).astype(np.float64)
        for x in (t, m, h, g):
            x.free()
        ctx.destroy()
        og = O.build_grid(ph, r.lo, r.hi, r.max_depth, r.min_depth, r.split_threshold)
        act, _ = O.active_leaves(og)
        oh = O.hist_for_active(O.splat(ph, og, r.n // 2, r.H, r.W, r.frac_bits), act)
        Po = O.tables_from_map(O.cnn_forward(O.assemble_inputs(oh), O.parse_net(NET)))["P"].reshape(-1, r.H * r.W)
        assert Po.shape == P.shape and act.size > 3
        kl = [float(np.sum(p[p > 0] * np.log(p[p > 0] / np.maximum(q[p > 0], 1e-300)))) for p, q in zip(Po, P)]
        assert np.mean(kl) <= 1e-3, (np.mean(kl), np.max(kl))
    finally:
        srv.close()


def test_shared_budget_released_after_the_free_runs():
    """A handle freed behind queued GPU work stays charged to the shared
    budget until the stream has run its free; synchronising the context
    returns the bytes."""
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    ctx = pg.Context(st.cuda_stream)
    b = pg.Budget(1 << 34)
    b.attach(ctx)
    try:
        ph = synth.photons(200_000, 8, 830)
        d = torch.from_numpy(ph).cuda()
        torch.cuda.synchronize()
        g = pg.pg_build_grid(ctx, d, 200_000, [0, 0, 0], [1, 1, 1], 8, 0, 500)
        ctx.sync()
        charged = b.query()[0]
        gbytes = g.info(pg.PG_INFO_BYTES)
        assert charged >= gbytes > 0 and charged == ctx.bytes_in_use()
        with torch.cuda.stream(st):
            torch.cuda._sleep(400_000_000)  # about 0.2 s of GPU time ahead of the free
        g.free()
        assert b.query()[0] == charged  # the free has not run yet
        ctx.sync()
        assert b.query()[0] <= charged - gbytes
        assert b.query()[0] == ctx.bytes_in_use()
    finally:
        b.detach(ctx)
        ctx.destroy()
        b.destroy()
