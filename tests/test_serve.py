"""Serving loop host logic on the CPU: batching, cancellation, argument
checks, the shared HBM budget (the real native pg_budget) and what the
workers do on an allocation refusal or a device-side input error.  The GPU
executor is replaced by a fake that charges the budget like the library
does; failures are made on the host (a refused allocation, an error status
from a fake library call), never on a GPU.
"""
import threading
import time

import numpy as np
import pytest

from paper_2010_01775_gb300 import pg, serve


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    pg.load()


def _req(n=10, q=4, H=16, W=16, prec=pg.PG_BF16, **kw):
    return serve.Request(np.zeros((n, 8), np.float32), np.zeros((q, 3), np.float32), np.zeros((q, 3), np.float32),
                         H, W, prec, **kw)


def test_scheduler_batches_compatible_requests_in_fifo_order():
    s = serve.Scheduler(max_scenes=3, max_photons=100, max_queries=1000)
    rs = [_req(), _req(H=32, W=32), _req(), _req(n=95), _req(), _req(), _req()]
    for r in rs:
        s.submit(r)
    b = s.take()
    # Head + compatible followers, skipping the 32x32 one and the one that
    # would pass the photon limit; at most 3 scenes.
    assert b == [rs[0], rs[2], rs[4]]
    assert s.take() == [rs[1]]
    assert s.take() == [rs[3]]  # 95 photons: 95 + 10 > 100, runs alone
    assert s.take() == [rs[5], rs[6]]
    assert s.take(timeout=0.01) is None


def test_scheduler_solo_and_no_batching():
    s = serve.Scheduler(batching=False)
    a, b = _req(), _req()
    s.submit(a)
    s.submit(b)
    assert s.take() == [a] and s.take() == [b]
    s = serve.Scheduler()
    a, b, c = _req(), _req(), _req()
    b.solo = True
    for r in (a, b, c):
        s.submit(r)
    assert s.take() == [a, c]
    assert s.take() == [b]


def test_cancel_waiting_request():
    s = serve.Scheduler()
    a, b = _req(), _req()
    s.submit(a)
    s.submit(b)
    assert s.cancel(b)
    assert b.status == "cancelled" and b.wait(0)
    assert s.take() == [a]
    assert not s.cancel(a)  # already taken


def test_validate_rejects_malformed_requests():
    assert serve.validate(_req()) == ""
    assert "powers of two" in serve.validate(_req(H=24))
    assert "powers of two" in serve.validate(_req(H=256, W=256))
    r = _req()
    r.positions = np.zeros((4, 2), np.float32)
    assert "positions" in serve.validate(r)
    assert "empty domain" in serve.validate(_req(lo=(0, 0, 0), hi=(1, 0, 1)))
    assert "n_prev" in serve.validate(_req(n_prev=11))


def test_budget_threads_never_pass_capacity():
    b = pg.Budget(1000)
    peak, lock, stop = [0], threading.Lock(), time.time() + 0.5

    def worker(k):
        rng = np.random.default_rng(k)
        while time.time() < stop:
            x = int(rng.integers(1, 400))
            if b.charge(x):
                used = b.query()[0]
                with lock:
                    peak[0] = max(peak[0], used)
                b.release(x)

    ts = [threading.Thread(target=worker, args=(k,)) for k in range(6)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert b.query()[0] == 0
    assert 0 < peak[0] <= 1000
    b.destroy()


def test_budget_wait_wakes_on_release_and_times_out():
    b = pg.Budget(100)
    assert b.charge(80)
    gen = b.query()[2]
    ok, gen2 = b.wait(50, gen, 20)
    assert not ok and gen2 == gen
    threading.Timer(0.05, lambda: b.release(80)).start()
    t = time.time()
    ok, gen3 = b.wait(50, gen, 5000)
    assert ok and gen3 == gen + 1 and time.time() - t < 2
    b.destroy()


class FakeExecutor(serve.Executor):
    """Charges r.n bytes for inputs and, through a fake library call that
    refuses like the library (PG_ERR_OOM, nothing charged), r.q bytes of
    working memory; a request with stream_id 666 posts a device input error."""

    def __init__(self, server):
        self.server = server

    def _fake_call(self, b, nbytes):
        # Like a library call that allocates its output, then its scratch,
        # and on refusal gives the output back before returning PG_ERR_OOM.
        half = nbytes // 2
        if not self.server.budget.charge(half):
            raise pg.PgError(3, "fake")
        if not self.server.budget.charge(nbytes - half):
            self.server.budget.release(half)
            raise pg.PgError(3, "fake")
        b.charged += nbytes

    def run(self, batch):
        b = serve._Batch()
        self._t0 = batch[0].t_start
        try:
            self._charge(b, sum(r.n for r in batch))
            time.sleep(0.002)
            self._retry(b, self._fake_call, b, sum(r.q for r in batch))
            time.sleep(0.005)
            if any(r.stream_id == 666 for r in batch):
                raise pg.PgError(8, "fake device input error")
            for r in batch:
                r.batch_size = len(batch)
                r._finish("done")
        finally:
            if b.charged:
                self.server.budget.release(b.charged)


def _server(**kw):
    return serve.Server(b"", executor=FakeExecutor, stall_ms=10, **kw)


def test_server_waits_for_memory_and_fails_what_cannot_fit():
    srv = _server(workers=4, hbm_budget=1000)
    rs = [srv.submit(_req(n=300, q=200, H=16 << (k % 2), W=16 << (k % 2))) for k in range(12)]
    big = srv.submit(_req(n=600, q=600))  # 1200 bytes: never fits 1000
    for r in rs + [big]:
        assert r.wait(30), "serving loop stalled"
    srv.close()
    assert all(r.status == "done" for r in rs)
    assert big.status == "failed" and big.error_status == 3
    assert srv.budget.ptr is None


def test_server_isolates_malformed_request_in_batch():
    srv = _server(workers=1, hbm_budget=10 ** 6)
    gate = threading.Event()
    # Hold the only worker so that the next requests queue up and batch.
    blocker = _req()
    orig = FakeExecutor.run

    def slow_run(self, batch):
        if batch[0] is blocker:
            gate.wait(5)
        return orig(self, batch)

    FakeExecutor.run = slow_run
    try:
        srv.submit(blocker)
        time.sleep(0.05)
        rs = [srv.submit(_req(stream_id=k)) for k in range(3)]
        bad = srv.submit(_req(stream_id=666))
        rs += [srv.submit(_req(stream_id=k)) for k in range(3, 5)]
        cancelled = srv.submit(_req(stream_id=7))
        assert srv.cancel(cancelled)
        gate.set()
        for r in rs + [bad, blocker]:
            assert r.wait(10)
    finally:
        FakeExecutor.run = orig
        srv.close()
    assert all(r.status == "done" for r in rs)
    assert bad.status == "failed" and bad.error_status == 8
    assert cancelled.status == "cancelled"
    # The five good ones first ran batched with the bad one, then alone.
    assert all(r.batch_size == 1 for r in rs)


def test_server_rejects_invalid_request_at_submit():
    srv = _server(workers=1, hbm_budget=10 ** 6)
    r = srv.submit(_req(H=12))
    assert r.wait(1) and r.status == "failed" and r.error_status == 1
    srv.close()


def test_latency_summary():
    rs = [_req() for _ in range(4)]
    for k, r in enumerate(rs):
        r.arrival, r.t_done, r.status, r.batch_size = 0.0, 0.1 * (k + 1), "done", 2
    s = serve.latency_summary(rs)
    assert s["done"] == 4 and abs(s["p50_ms"] - 250) < 1e-6 and abs(s["makespan_s"] - 0.4) < 1e-12
    assert abs(s["requests_per_s"] - 10) < 1e-9 and s["mean_batch"] == 2


def test_big_request_does_not_livelock_small_ones():
    # A request that never fits (its working memory is over the budget once
    # its inputs are charged) must not keep the memory it gives back away
    # from the requests queued behind it.
    for _ in range(5):
        srv = _server(workers=2, hbm_budget=1000)
        big = srv.submit(_req(n=600, q=600))
        small = [srv.submit(_req(n=300, q=200)) for _ in range(6)]
        for r in [big] + small:
            assert r.wait(30), "serving loop stalled"
        srv.close()
        assert all(r.status == "done" for r in small)
        assert big.status == "failed" and big.error_status == 3
