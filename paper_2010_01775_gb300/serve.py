"""Multi-request serving of the guiding path on one GPU.

A request is one scene's photons plus a set of path vertices that want
guided directions (Algorithm 1: locate the voxel, sample the guide, evaluate
its pdf for MIS).  The paper renders one scene at a time and has no server;
this module is the layer a renderer farm would put in front of the library:

* Workers: a fixed pool of threads, each with its own CUDA stream and
  library context; every step of a request runs in the library's kernels on
  that stream (the library calls release the GIL, so the workers' streams
  overlap on the GPU).
* Admission: one shared HBM byte budget (pg_budget) charged by every worker
  context and by the request buffers the workers allocate.  A library call
  that would pass the budget fails with PG_ERR_OOM having allocated nothing;
  the worker then waits for another worker to release memory and retries
  the same call, and no new batch is admitted while a running one waits.
  When every busy worker is waiting, the youngest batch that holds memory
  gives it back: a batch of several requests returns to the front of the
  queue as single requests, a single request to the back.  A batch that
  holds the only memory held and still does not fit fails with PG_ERR_OOM.
* Continuous batching: a worker that becomes free takes the oldest waiting
  request and, behind it, every waiting request with the same map size,
  precision, grid rule and fixed-point scale (up to per-batch limits) and
  runs them as one scene batch (the library's batched calls).  A scene's
  results do not depend on the batch it ran in: the batched grid, splat,
  reconstruction, tables and samples are the ones it gets alone.
* Isolation: a device-side input error (non-finite photon, overflow) in a
  batch re-runs its requests one by one, so only the malformed request
  fails.  Requests can be cancelled while they wait.

Latency of a request = completion (its results are in host memory) minus
arrival (its submit call).
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from . import pg

PG_ERR_OOM = 3
_DEVICE_INPUT_ERRORS = (4, 8)  # PG_ERR_OVERFLOW, PG_ERR_INVALID_INPUT


@dataclasses.dataclass(eq=False)
class Request:
    """One scene's photons (n x 8 float32, pg_photon records) and q query
    positions (q x 3) with q directions (q x 3) whose guide pdf is wanted.
    Tensors may live on the host (pinned for asynchronous copies) or on the
    device.  Results (when the server keeps them) are host arrays: dirs
    (q x 3), pdf (q), leaf (q, uint32), bin (q, uint32), eval_pdf (q)."""

    photons: object
    positions: object
    directions: object
    H: int
    W: int
    precision: int = pg.PG_BF16
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    max_depth: int = 10
    min_depth: int = 0
    split_threshold: int = 2000
    frac_bits: int = 32
    n_prev: int | None = None  # default n // 2
    stream_id: int = 0
    rid: int = -1
    # filled in by the server
    status: str = "new"  # queued, running, done, failed, cancelled
    error: str = ""
    error_status: int = 0
    arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    batch_size: int = 0
    evictions: int = 0
    solo: bool = False
    result: dict | None = None
    _done: threading.Event = dataclasses.field(default_factory=threading.Event, repr=False)

    @property
    def n(self) -> int:
        return int(self.photons.shape[0])

    @property
    def q(self) -> int:
        return int(self.positions.shape[0])

    @property
    def key(self):
        """Requests with equal keys can share one scene batch."""
        return (self.H, self.W, self.precision, self.max_depth, self.min_depth, self.split_threshold,
                self.frac_bits)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    def wait(self, timeout=None) -> bool:
        return self._done.wait(timeout)

    def _finish(self, status, error="", error_status=0):
        self.status, self.error, self.error_status = status, error, error_status
        self.t_done = time.perf_counter()
        self._done.set()


def validate(r: Request) -> str:
    """Host-side shape/argument checks done at submit (no data scan)."""
    if len(getattr(r.photons, "shape", ())) != 2 or r.photons.shape[1] != 8:
        return "photons must be (n, 8) float32 records"
    for name in ("positions", "directions"):
        a = getattr(r, name)
        if len(getattr(a, "shape", ())) != 2 or a.shape[1] != 3 or a.shape[0] != r.q:
            return f"{name} must be (q, 3)"
    if r.H not in (4, 8, 16, 32, 64, 128, 256) or r.W not in (4, 8, 16, 32, 64, 128, 256) or r.H * r.W > 16384:
        return "H and W must be powers of two in [4, 256] with H*W <= 16384"
    if r.precision not in (pg.PG_FP32, pg.PG_BF16, pg.PG_FP8_E4M3):
        return "unknown precision"
    if not (0 <= r.min_depth <= r.max_depth <= 16) or not (0 <= r.frac_bits <= 62):
        return "bad grid depth or fixed-point bits"
    if any(not (h > l) for l, h in zip(r.lo, r.hi)):
        return "empty domain"
    if r.n_prev is not None and not (0 <= r.n_prev <= r.n):
        return "n_prev outside [0, n]"
    if r.n >= 1 << 31 or r.q >= 1 << 32:
        return "too many photons or queries"
    return ""


class Scheduler:
    """FIFO of waiting requests with greedy batching of compatible ones."""

    def __init__(self, batching=True, max_scenes=64, max_photons=8 << 20, max_queries=32 << 20):
        self.batching, self.max_scenes = batching, max_scenes
        self.max_photons, self.max_queries = max_photons, max_queries
        self._q = collections.deque()
        self._cv = threading.Condition()
        self._closed = False

    def submit(self, r: Request):
        with self._cv:
            if self._closed:
                raise RuntimeError("scheduler closed")
            r.status = "queued"
            self._q.append(r)
            self._cv.notify()

    def requeue_front(self, reqs):
        with self._cv:
            for r in reversed(reqs):
                r.status = "queued"
                self._q.appendleft(r)
            self._cv.notify_all()

    def requeue_back(self, r: Request):
        with self._cv:
            r.status = "queued"
            self._q.append(r)
            self._cv.notify_all()

    def cancel(self, r: Request) -> bool:
        with self._cv:
            try:
                self._q.remove(r)
            except ValueError:
                return False
        r._finish("cancelled")
        return True

    def pending(self) -> int:
        with self._cv:
            return len(self._q)

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()

    def take(self, timeout=None):
        """Oldest waiting request plus compatible followers; None once the
        scheduler is closed and empty (or on timeout)."""
        with self._cv:
            end = None if timeout is None else time.monotonic() + timeout
            while not self._q:
                if self._closed:
                    return None
                left = None if end is None else end - time.monotonic()
                if left is not None and left <= 0:
                    return None
                self._cv.wait(left)
            head = self._q.popleft()
            batch = [head]
            if self.batching and not head.solo and head.n <= self.max_photons and head.q <= self.max_queries:
                n, q, keep = head.n, head.q, collections.deque()
                while self._q:
                    r = self._q.popleft()
                    if (len(batch) < self.max_scenes and not r.solo and r.key == head.key
                            and n + r.n <= self.max_photons and q + r.q <= self.max_queries):
                        batch.append(r)
                        n, q = n + r.n, q + r.q
                    else:
                        keep.append(r)
                self._q = keep
            for r in batch:
                r.status = "running"
            return batch


class Evicted(Exception):
    """The batch gave its memory back; its requests go back to the queue,
    or fail when `final` (the batch cannot fit the budget)."""

    def __init__(self, final=False):
        super().__init__("evicted")
        self.final = final


class _Batch:
    """Device buffers and library handles of one running batch."""

    def __init__(self):
        self.handles, self.charged, self.tensors = [], 0, {}


class Executor:
    """Memory protocol shared by executors: budget charges and library calls
    that wait for released memory on PG_ERR_OOM."""

    server = None
    _t0 = 0.0

    def held(self, b: _Batch) -> int:
        """Bytes this worker holds for its running batch."""
        return b.charged

    def _retry(self, b: _Batch, fn, *args):
        """Runs a library call, waiting for released memory on PG_ERR_OOM.
        Before giving its memory back the batch tries once more (memory may
        have been released while it looked)."""
        confirm = False
        while True:
            try:
                return fn(*args)
            except pg.PgError as e:
                if e.status != PG_ERR_OOM:
                    raise
            v = self.server._wait_for_release(self._t0, self.held(b))
            if v == "retry" or not confirm:
                confirm = v != "retry"
                continue
            raise Evicted(final=v == "fail")

    def _charge(self, b: _Batch, nbytes):
        """Charges a new batch's buffers.  No new batch is admitted while a
        running one waits for memory (it has priority on what is released)."""
        confirm = False
        while True:
            if not self.server._holder_waiting() and self.server.budget.charge(nbytes):
                b.charged += nbytes
                return
            v = self.server._wait_for_release(self._t0, self.held(b))
            if v == "retry" or not confirm:
                confirm = v != "retry"
                continue
            raise Evicted(final=v == "fail")

    def close(self):
        pass


class GpuExecutor(Executor):
    """One worker's stream, context and staging buffer."""

    def __init__(self, server, device):
        import torch

        self.torch, self.server = torch, server
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = pg.Context(self.stream.cuda_stream)
        server.budget.attach(self.ctx)
        self.stage = None  # pinned host staging for results

    def close(self):
        try:
            self.ctx.sync()
        finally:
            self.ctx.destroy()

    def held(self, b: _Batch) -> int:
        return b.charged + self.ctx.bytes_in_use()

    def _release(self, b: _Batch):
        for h in reversed(b.handles):
            h.free()
        b.handles.clear()
        # The library returns a freed block's bytes to the shared budget once
        # the stream has run the free; synchronising the context does that now.
        try:
            self.ctx.sync()
        except pg.PgError:
            pass  # a device-side error of the failed batch, already reported
        if b.tensors:
            self.stream.synchronize()
            b.tensors.clear()
        if b.charged:
            self.server.budget.release(b.charged)
            b.charged = 0

    # ---------------------------------------------------------------- run
    def run(self, batch):
        torch = self.torch
        b = _Batch()
        S = len(batch)
        ns = [r.n for r in batch]
        qs = [r.q for r in batch]
        n, Q = sum(ns), sum(qs)
        pbeg = np.concatenate([[0], np.cumsum(ns)]).astype(np.uint32)
        qbeg = np.concatenate([[0], np.cumsum(qs)]).astype(np.uint32)
        r0 = batch[0]
        self._t0 = r0.t_start
        try:
            self._charge(b, 32 * n + 52 * Q + 4096)
            dev = torch.device("cuda", self.device)
            with torch.cuda.stream(self.stream):
                t = b.tensors
                t["ph"] = ph = torch.empty((n, 8), dtype=torch.float32, device=dev)
                t["pos"] = pos = torch.empty((Q, 3), dtype=torch.float32, device=dev)
                t["din"] = din = torch.empty((Q, 3), dtype=torch.float32, device=dev)
                # Outputs in one block: dirs (3Q floats), pdf, leaf, bin, eval pdf (Q each).
                t["out"] = out = torch.empty(7 * Q, dtype=torch.float32, device=dev)
                for i, r in enumerate(batch):
                    if ns[i]:
                        ph[pbeg[i]:pbeg[i + 1]].copy_(r.photons, non_blocking=True)
                    if qs[i]:
                        pos[qbeg[i]:qbeg[i + 1]].copy_(r.positions, non_blocking=True)
                        din[qbeg[i]:qbeg[i + 1]].copy_(r.directions, non_blocking=True)
                o_dir, o_pdf = out[:3 * Q], out[3 * Q:4 * Q]
                o_leaf, o_bin, o_ev = out[4 * Q:5 * Q], out[5 * Q:6 * Q], out[6 * Q:]
                net = self.server.net
                if S == 1:
                    g = self._retry(b, pg.pg_build_grid, self.ctx, ph if n else 0, n, r0.lo, r0.hi, r0.max_depth,
                                    r0.min_depth, r0.split_threshold)
                else:
                    g = self._retry(b, pg.pg_build_grid_batched, self.ctx, ph, n, pbeg, [r.lo for r in batch],
                                    [r.hi for r in batch], r0.max_depth, r0.min_depth, r0.split_threshold)
                b.handles.append(g)
                # First leaf of every scene, to return scene-local leaf ids.
                lb = (g.export(pg.PG_GRID_SCENE_LEAF_BEGIN, np.uint32, S + 1) if S > 1 and self.server.keep_results
                      else np.zeros(S + 1, np.uint32))
                nprev = [r.n // 2 if r.n_prev is None else r.n_prev for r in batch]
                if S == 1:
                    h = self._retry(b, pg.pg_splat_photons, self.ctx, g, ph if n else 0, n, nprev[0], r0.H, r0.W,
                                    r0.frac_bits)
                else:
                    h = self._retry(b, pg.pg_splat_photons_batched, self.ctx, g, ph, n, np.array(nprev, np.uint32),
                                    r0.H, r0.W, r0.frac_bits)
                b.handles.append(h)
                m = self._retry(b, pg.pg_reconstruct, self.ctx, h, net, r0.precision)
                b.handles.append(m)
                h.free()
                tab = self._retry(b, pg.pg_build_cdf, self.ctx, m)
                b.handles.append(tab)
                m.free()
                if Q:
                    if S == 1:
                        self._retry(b, pg.pg_sample_dirs, self.ctx, g, tab, pos, Q, self.server.seed, r0.stream_id,
                                    o_dir, o_pdf, o_leaf, o_bin)
                        self._retry(b, pg.pg_eval_pdf, self.ctx, g, tab, pos, din, Q, o_ev)
                    else:
                        sid = np.array([r.stream_id for r in batch], np.uint32)
                        self._retry(b, pg.pg_sample_dirs_batched, self.ctx, g, tab, pos, qbeg, Q, self.server.seed,
                                    sid, o_dir, o_pdf, o_leaf, o_bin)
                        self._retry(b, pg.pg_eval_pdf_batched, self.ctx, g, tab, pos, din, qbeg, Q, o_ev)
                tab.free()
                g.free()
                b.handles.clear()
                # Results to host memory (pinned staging, grown on demand).
                if self.stage is None or self.stage.numel() < 7 * Q:
                    self.stage = torch.empty(max(7 * Q, 1 << 20) * 5 // 4, dtype=torch.float32, pin_memory=True)
                host = self.stage[:7 * Q]
                if Q:
                    host.copy_(out, non_blocking=True)
            self.ctx.sync()  # waits for the stream; raises a device-side input error
            t_done = time.perf_counter()
            for i, r in enumerate(batch):
                if self.server.keep_results:
                    a, e = int(qbeg[i]), int(qbeg[i + 1])
                    hv = host.numpy()
                    leaf = hv[4 * Q + a:4 * Q + e].view(np.uint32)
                    leaf = (leaf & np.uint32(0x80000000)) | ((leaf & np.uint32(0x7FFFFFFF)) - lb[i])
                    r.result = dict(dirs=hv[3 * a:3 * e].reshape(-1, 3).copy(), pdf=hv[3 * Q + a:3 * Q + e].copy(),
                                    leaf=leaf,
                                    bin=hv[5 * Q + a:5 * Q + e].view(np.uint32).copy(),
                                    eval_pdf=hv[6 * Q + a:6 * Q + e].copy())
                r.batch_size = S
                r._finish("done")
                r.t_done = t_done
        finally:
            self._release(b)


class Server:
    """Worker pool + scheduler + shared budget around one network."""

    def __init__(self, net_blob: bytes, workers=4, hbm_budget=120 << 30, batching=True, seed=20101775,
                 keep_results=False, device=0, stall_ms=50, executor=None, **sched_kw):
        self.budget = pg.Budget(hbm_budget)
        self.seed, self.keep_results, self.stall_ms = seed, keep_results, stall_ms
        self.sched = Scheduler(batching=batching, **sched_kw)
        self._lock = threading.Lock()
        self._busy = 0
        self._stalled = {}  # waiting worker -> start time of its batch
        self._next_id = 0
        self.completed = []
        if executor is None:
            import torch

            torch.cuda.set_device(device)
            self._owner = pg.Context(torch.cuda.current_stream(device).cuda_stream)
            self.budget.attach(self._owner)
            self.net = pg.pg_net_load(self._owner, net_blob)
            make = lambda: GpuExecutor(self, device)  # noqa: E731
        else:
            self._owner, self.net = None, None
            make = lambda: executor(self)  # noqa: E731
        self.executors = [make() for _ in range(workers)]
        self._threads = [threading.Thread(target=self._worker, args=(ex, device), daemon=True)
                         for ex in self.executors]
        for th in self._threads:
            th.start()

    # -------------------------------------------------------------- client API
    def warmup(self, requests, autotune=True):
        """Runs requests one by one on worker 0's context before serving:
        tunes the tensor-core layers for each map size and calibrates the FP8
        activation scales (the net's state is fixed from then on, so results
        do not depend on which worker or batch serves a request)."""
        ex = self.executors[0]
        for r in requests:
            if autotune and r.precision != pg.PG_FP32:
                with self._lock:
                    self._busy += 1
                try:
                    self._tune(ex, r)
                finally:
                    with self._lock:
                        self._busy -= 1
            self.submit(r)
            r.wait()
            if r.status != "done":
                raise RuntimeError(f"warm-up request failed: {r.error}")

    def _tune(self, ex, r):
        import torch

        with torch.cuda.stream(ex.stream):
            ph = torch.as_tensor(r.photons).to(f"cuda:{ex.device}")
            g = pg.pg_build_grid(ex.ctx, ph, r.n, r.lo, r.hi, r.max_depth, r.min_depth, r.split_threshold)
            h = pg.pg_splat_photons(ex.ctx, g, ph, r.n, r.n // 2, r.H, r.W, r.frac_bits)
            pg.pg_autotune(ex.ctx, h, self.net, r.precision)
            ex.ctx.sync()
            h.free()
            g.free()

    def submit(self, r: Request) -> Request:
        r.arrival = time.perf_counter()
        with self._lock:
            r.rid = self._next_id
            self._next_id += 1
        err = validate(r)
        if err:
            r._finish("failed", err, 1)
            return r
        self.sched.submit(r)
        return r

    def cancel(self, r: Request) -> bool:
        return self.sched.cancel(r)

    def close(self):
        self.sched.close()
        for th in self._threads:
            th.join()
        for ex in self.executors:
            ex.close()
        if self._owner is not None:
            self._owner.destroy()
        self.budget.destroy()

    # -------------------------------------------------------------- internals
    def _holder_waiting(self) -> bool:
        """True while another worker holding memory waits for more."""
        me = threading.get_ident()
        with self._lock:
            return any(h > 0 for k, (_, h) in self._stalled.items() if k != me)

    def _wait_for_release(self, t0, held) -> str:
        """After an allocation refusal: 'retry' once the bytes in use dropped
        below what they were after the refusal (a failed call's own rollback
        does not count, so two waiting workers cannot wake each other up
        forever).  When every busy worker is waiting, nothing will be
        released unless a worker gives memory back: the youngest batch holding
        memory gets 'evict'; a worker that holds the only memory held (or none
        while no one holds any) cannot fit its batch at all and gets 'fail'."""
        me = threading.get_ident()
        used0, cap, gen = self.budget.query()
        need = max(1, min(cap - used0 + 1, 1 << 63))  # fits iff in_use < used0
        with self._lock:
            self._stalled[me] = (t0, held)
        try:
            while True:
                end = time.monotonic() + self.stall_ms / 1000.0
                while True:
                    left = end - time.monotonic()
                    if left <= 0:
                        break
                    _, gen = self.budget.wait(need, gen, max(1, int(left * 1000)))
                    if self.budget.query()[0] < used0:
                        return "retry"
                with self._lock:
                    if self._busy - len(self._stalled) > 0:
                        continue
                    holders = [t for t, h in self._stalled.values() if h > 0]
                    if (held > 0 and len(holders) == 1) or not holders:
                        return "fail"
                    if held > 0 and t0 >= max(holders):
                        return "evict"
        finally:
            with self._lock:
                del self._stalled[me]

    def _worker(self, ex, device):
        if self.net is not None:
            import torch

            torch.cuda.set_device(device)
        while True:
            batch = self.sched.take()
            if batch is None:
                return
            with self._lock:
                self._busy += 1
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                ex.run(batch)
            except Evicted as ev:
                if len(batch) > 1:
                    for r in batch:
                        r.solo = True
                    self.sched.requeue_front(batch)
                else:
                    # A request that gave its memory back waits behind the
                    # queue (at the front it would take the memory it just
                    # released again before the requests it made room for);
                    # one that does not fit while running alone fails.
                    r = batch[0]
                    r.evictions += 1
                    if ev.final:
                        r._finish("failed", "does not fit the HBM budget", PG_ERR_OOM)
                    else:
                        r.solo = True
                        self.sched.requeue_back(r)
            except pg.PgError as e:
                if len(batch) > 1 and e.status in _DEVICE_INPUT_ERRORS:
                    # Find the malformed request: run the batch's requests alone.
                    for r in batch:
                        r.solo = True
                    self.sched.requeue_front(batch)
                else:
                    for r in batch:
                        r._finish("failed", str(e), e.status)
            except Exception as e:  # noqa: BLE001 - a worker must not die
                for r in batch:
                    r._finish("failed", repr(e), -1)
            finally:
                with self._lock:
                    self._busy -= 1
                    self.completed.extend(r for r in batch if r._done.is_set())


def latency_summary(reqs) -> dict:
    done = [r for r in reqs if r.status == "done"]
    lat = np.array([r.latency for r in done]) * 1e3
    if not len(lat):
        return dict(done=0)
    t0 = min(r.arrival for r in reqs)
    t1 = max(r.t_done for r in done)
    errors = sorted({f"{r.error_status}: {r.error}" for r in reqs if r.status == "failed"})[:4]
    return dict(done=len(done), failed=sum(r.status == "failed" for r in reqs), errors=errors,
                cancelled=sum(r.status == "cancelled" for r in reqs), p50_ms=float(np.percentile(lat, 50)),
                p90_ms=float(np.percentile(lat, 90)), p99_ms=float(np.percentile(lat, 99)), max_ms=float(lat.max()),
                makespan_s=t1 - t0, requests_per_s=len(done) / (t1 - t0),
                samples_per_s=sum(r.q for r in done) / (t1 - t0),
                mean_batch=float(np.mean([r.batch_size for r in done])))
