// C-ABI entry points of libpg: argument checks, host/device staging, handle
// lifetime and the HBM budget.  Every compute step is a kernel launched by
// the per-step files (grid.cu, splat.cu, cnn.cu, cdf.cu, sample.cu).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <new>
#include <vector>

#include "pg_internal.cuh"

// Shared byte budget: charges are a compare-and-swap on in_use; releases
// bump a generation counter and wake waiters.
struct pg_budget {
  uint64_t capacity;
  std::atomic<uint64_t> in_use{0};
  std::atomic<uint64_t> generation{0};
  std::atomic<int> attached{0};
  std::mutex mu;
  std::condition_variable cv;
};

namespace pgi {

bool budget_try_charge(pg_budget *b, size_t bytes) {
  uint64_t cur = b->in_use.load(std::memory_order_relaxed);
  do {
    if (bytes > b->capacity || cur > b->capacity - bytes) return false;
  } while (!b->in_use.compare_exchange_weak(cur, cur + bytes, std::memory_order_acq_rel));
  return true;
}

void budget_release(pg_budget *b, size_t bytes) {
  uint64_t cur = b->in_use.load(std::memory_order_relaxed);
  while (!b->in_use.compare_exchange_weak(cur, cur >= bytes ? cur - bytes : 0, std::memory_order_acq_rel)) {
  }
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->generation.fetch_add(1, std::memory_order_acq_rel);
  }
  b->cv.notify_all();
}

cudaError_t &last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

// Frees are stream-ordered: cudaFreeAsync returns at once, and the block
// stays live until the stream reaches it.  The shared budget gets the bytes
// back only then: each free records an event, and the bytes of completed
// events are released when the context next allocates, synchronises or is
// destroyed (in stream order, so the queue is reaped from its head).
struct PendingFrees {
  std::mutex mu;
  std::vector<cudaEvent_t> spare;                          // reusable events
  std::vector<std::pair<cudaEvent_t, size_t>> queue;       // in stream order
  size_t head = 0;
};

void ctx_reap_frees(pg_ctx *ctx, bool all) {
  PendingFrees *pf = ctx->pending;
  if (!pf) return;
  if (all) cudaStreamSynchronize(ctx->stream);
  std::lock_guard<std::mutex> lk(pf->mu);
  size_t released = 0;
  while (pf->head < pf->queue.size()) {
    auto &e = pf->queue[pf->head];
    const cudaError_t q = all ? cudaEventSynchronize(e.first) : cudaEventQuery(e.first);
    if (q == cudaErrorNotReady) break;
    released += e.second;
    pf->spare.push_back(e.first);
    ++pf->head;
  }
  cudaGetLastError();
  if (pf->head == pf->queue.size()) {
    pf->queue.clear();
    pf->head = 0;
  }
  if (released && ctx->shared) budget_release(ctx->shared, released);
}

// Bytes still charged to the shared budget for frees that have not run.
static size_t pending_bytes(pg_ctx *ctx) {
  PendingFrees *pf = ctx->pending;
  if (!pf) return 0;
  std::lock_guard<std::mutex> lk(pf->mu);
  size_t b = 0;
  for (size_t i = pf->head; i < pf->queue.size(); ++i) b += pf->queue[i].second;
  return b;
}

pg_status ctx_alloc(pg_ctx *ctx, size_t bytes, void **ptr) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  if (ctx->shared) ctx_reap_frees(ctx, false);
  if (ctx->budget && ctx->in_use + bytes > ctx->budget) return PG_ERR_OOM;
  if (ctx->shared && !budget_try_charge(ctx->shared, bytes)) return PG_ERR_OOM;
  cudaError_t e = cudaMallocAsync(ptr, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    if (ctx->shared) budget_release(ctx->shared, bytes);
    return PG_ERR_OOM;
  }
  ctx->in_use += bytes;
  return PG_OK;
}

// Long-lived device memory outside the stream-ordered pool (charged to the
// same budget): a block taken from the pool in the middle of a call that
// holds large scratch can split the pool's free space so that the next
// call's scratch no longer fits and the pool maps new memory every call.
pg_status ctx_alloc_static(pg_ctx *ctx, size_t bytes, void **ptr) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  if (ctx->shared) ctx_reap_frees(ctx, false);
  if (ctx->budget && ctx->in_use + bytes > ctx->budget) return PG_ERR_OOM;
  if (ctx->shared && !budget_try_charge(ctx->shared, bytes)) return PG_ERR_OOM;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    if (ctx->shared) budget_release(ctx->shared, bytes);
    return PG_ERR_OOM;
  }
  ctx->in_use += bytes;
  return PG_OK;
}

void ctx_free_static(pg_ctx *ctx, void *ptr, size_t bytes) {
  if (!ptr) return;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  cudaFree(ptr);  // waits for the device
  ctx->in_use = ctx->in_use >= bytes ? ctx->in_use - bytes : 0;
  if (ctx->shared) budget_release(ctx->shared, bytes);
}

void ctx_free(pg_ctx *ctx, void *ptr, size_t bytes) {
  if (!ptr) return;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  cudaFreeAsync(ptr, ctx->stream);
  ctx->in_use = ctx->in_use >= bytes ? ctx->in_use - bytes : 0;
  if (!ctx->shared) return;
  // A free captured into a CUDA graph is a graph node, not work on the
  // stream: its bytes go back at once, as the capture's allocations were
  // charged at capture time.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (!ctx->pending || cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    budget_release(ctx->shared, bytes);
    return;
  }
  PendingFrees *pf = ctx->pending;
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(pf->mu);
    if (!pf->spare.empty()) {
      ev = pf->spare.back();
      pf->spare.pop_back();
    }
  }
  if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) ev = nullptr;
  if (!ev || cudaEventRecord(ev, ctx->stream) != cudaSuccess) {
    // No event: wait for the stream, after which the free has run.
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(ctx->stream);
    budget_release(ctx->shared, bytes);
    return;
  }
  std::lock_guard<std::mutex> lk(pf->mu);
  pf->queue.emplace_back(ev, bytes);
}

// Boundary rays of the W phi sectors: (float cos, float sin) of 2 pi j / W,
// exactly (1,0), (0,1), (-1,0), (0,-1) on the quarter turns.
namespace {
__global__ void k_read_words(const uint32_t *a, const uint32_t *b, uint32_t *out) {
  if (threadIdx.x == 0) {
    volatile uint32_t *o = out;
    o[0] = *a;
    if (b) o[1] = *b;
    __threadfence_system();
  }
}
}  // namespace

pg_status read_words(pg_ctx *ctx, cudaStream_t st, const uint32_t *a, uint32_t *ha, const uint32_t *b,
                     uint32_t *hb) {
  k_read_words<<<1, 32, 0, st>>>(a, b, ctx->d_words + 8), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaStreamSynchronize(st));
  *ha = ctx->h_words[8];
  if (b) *hb = ctx->h_words[9];
  return PG_OK;
}

pg_status phi_table(pg_ctx *ctx, int W, const float **d_table) {
  int lg = 0;
  while ((1 << lg) < W) ++lg;
  if ((1 << lg) != W || lg > 8) return PG_ERR_NOT_POW2;
  if (!ctx->d_phi[lg]) {
    float host[512];
    for (int j = 0; j < W; ++j) {
      float c, s;
      if ((4 * j) % W == 0) {
        static const float cq[4] = {1.0f, 0.0f, -1.0f, 0.0f}, sq[4] = {0.0f, 1.0f, 0.0f, -1.0f};
        c = cq[(4 * j) / W];
        s = sq[(4 * j) / W];
      } else {
        double th = 2.0 * M_PI * (double)j / (double)W;
        c = (float)cos(th);
        s = (float)sin(th);
      }
      host[j] = c;
      host[W + j] = s;
    }
    float *d = nullptr;
    PG_CUDA(cudaMalloc(&d, sizeof(float) * 2 * W));
    PG_CUDA(cudaMemcpy(d, host, sizeof(float) * 2 * W, cudaMemcpyHostToDevice));
    ctx->d_phi[lg] = d;
  }
  *d_table = ctx->d_phi[lg];
  return PG_OK;
}

// A caller array that may live on the host: device arrays are used in place,
// host arrays are copied through a device buffer on the context stream.
struct Staged {
  pg_ctx *ctx = nullptr;
  void *dev = nullptr;
  void *host = nullptr;
  size_t bytes = 0;
  bool owned = false, out = false;
  ~Staged() {
    if (owned) ctx_free(ctx, dev, bytes);
  }
};

static pg_status classify(const void *p, bool *on_device) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PG_ERR_NOT_DEVICE_PTR;
  }
  *on_device = (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  return PG_OK;
}

static pg_status stage_in(pg_ctx *ctx, const void *p, size_t bytes, Staged &s) {
  bool dev;
  PG_TRY(classify(p, &dev));
  s.ctx = ctx;
  s.bytes = bytes;
  if (dev) {
    s.dev = const_cast<void *>(p);
    return PG_OK;
  }
  PG_TRY(ctx_alloc(ctx, bytes, &s.dev));
  s.owned = true;
  PG_CUDA(cudaMemcpyAsync(s.dev, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return PG_OK;
}

static pg_status stage_out(pg_ctx *ctx, void *p, size_t bytes, Staged &s) {
  if (!p) return PG_OK;
  bool dev;
  PG_TRY(classify(p, &dev));
  s.ctx = ctx;
  s.bytes = bytes;
  if (dev) {
    s.dev = p;
    return PG_OK;
  }
  PG_TRY(ctx_alloc(ctx, bytes, &s.dev));
  s.owned = true;
  s.out = true;
  s.host = p;
  return PG_OK;
}

static pg_status finish_out(Staged &s) {
  if (s.owned && s.out) PG_CUDA(cudaMemcpyAsync(s.host, s.dev, s.bytes, cudaMemcpyDeviceToHost, s.ctx->stream));
  return PG_OK;
}

static bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

template <class T>
static T *as(const void *h, uint32_t kind) {
  if (!h) return nullptr;
  const Handle *b = static_cast<const Handle *>(h);
  return b->kind == kind ? (T *)h : nullptr;
}

// ---------------------------------------------------------------- progressive iterations
// Frees a handle that a progress state owns (and lends out).
static void release_owned(void *h) {
  if (!h) return;
  ((Handle *)h)->borrowed = 0;
  pg_free(h);
}

static void free_progress(Progress *s) {
  pg_ctx *c = s->h.ctx;
  release_owned(s->grid);
  release_owned(s->cum);
  release_owned(s->map);
  release_owned(s->tab);
  ctx_free(c, s->stored, s->cap_stored * sizeof(pg_photon));
  ctx_free(c, s->stored_n, s->cap_stored * 3 * sizeof(float));
  ctx_free(c, s->updated, 4ull * s->cap_updated);
  s->h.kind = 0;
  delete s;
}

static pg_status progress_reserve_updated(pg_ctx *c, Progress *s, uint32_t A) {
  if (A > s->cap_updated) {
    void *b;
    PG_TRY(ctx_alloc(c, 4ull * A, &b));
    ctx_free(c, s->updated, 4ull * s->cap_updated);
    s->updated = (uint32_t *)b;
    s->cap_updated = A;
  }
  return PG_OK;
}

// A refining iteration: the grid is rebuilt from every photon kept so far
// (split threshold thr), and all its leaves' planes are recomputed; photons
// with index < n_prev are the earlier iterations'.  The leaves with photons
// take slots 0.. in leaf order (the grid's own active list).
static pg_status progress_regrid(pg_ctx *c, Progress *s, uint64_t n_prev, uint32_t thr) {
  const pg_progress_params &p = s->p;
  Grid *g = new (std::nothrow) Grid();
  Hist *cum = new (std::nothrow) Hist();
  Map *m = new (std::nothrow) Map();
  if (!g || !cum || !m) {
    delete g;
    delete cum;
    delete m;
    return PG_ERR_OOM;
  }
  memset(g, 0, sizeof(*g));
  memset(cum, 0, sizeof(*cum));
  memset(m, 0, sizeof(*m));
  g->h.kind = KIND_GRID;
  cum->h.kind = KIND_HIST;
  m->h.kind = KIND_MAP;
  g->h.ctx = cum->h.ctx = m->h.ctx = c;
  g->h.borrowed = cum->h.borrowed = m->h.borrowed = 1;
  pg_status st;
  if (p.grid_rule == 1) {
    pg_kd_params kp;
    for (int a = 0; a < 3; ++a) {
      kp.lo[a] = p.lo[a];
      kp.hi[a] = p.hi[a];
    }
    kp.resolution = p.resolution;
    kp.max_depth = p.max_depth;
    kp.split_threshold = thr;
    kp.normal_variance_threshold = p.normal_variance_threshold;
    st = build_grid_kd(c, s->stored, s->normals == 1 ? s->stored_n : nullptr, s->n_stored, &kp, g);
  } else {
    pg_grid_params gp;
    for (int a = 0; a < 3; ++a) {
      gp.lo[a] = p.lo[a];
      gp.hi[a] = p.hi[a];
    }
    gp.max_depth = p.max_depth;
    gp.min_depth = p.min_depth;
    gp.split_threshold = thr;
    st = build_grid(c, s->stored, s->n_stored, &gp, g);
  }
  if (st == PG_OK) {
    cum->H = p.H;
    cum->W = p.W;
    cum->A = g->A;
    st = splat(c, g, s->stored, p.max_photons, n_prev, p.frac_bits, cum);  // slot-indexed by the active list
  }
  if (st == PG_OK) st = progress_reserve_updated(c, s, g->A);
  if (st == PG_OK) st = iota_slots(c, g->A, s->updated);
  if (st == PG_OK) {
    m->A = g->A;
    m->H = p.H;
    m->W = p.W;
    m->h.bytes = (size_t)std::max<uint32_t>(g->A, 1) * p.H * p.W * sizeof(float);
    st = ctx_alloc(c, m->h.bytes, &m->block);
    if (st == PG_OK) {
      m->y = (float *)m->block;
      st = cudaMemsetAsync(m->block, 0, m->h.bytes, c->stream) == cudaSuccess ? PG_OK : PG_ERR_CUDA;
    }
  }
  if (st != PG_OK) {
    release_owned(g);
    release_owned(cum);
    release_owned(m);
    return st;
  }
  release_owned(s->grid);
  release_owned(s->cum);
  release_owned(s->map);
  release_owned(s->tab);
  s->tab = nullptr;
  s->grid = g;
  s->cum = cum;
  s->map = m;
  s->cap_slots = g->A;  // rows of cum (the map holds at least as many)
  s->n_updated = g->A;
  return PG_OK;
}

}  // namespace pgi

using namespace pgi;

extern "C" {

const char *pg_status_string(pg_status s) {
  switch (s) {
    case PG_OK: return "ok";
    case PG_ERR_INVALID_ARG: return "invalid argument";
    case PG_ERR_NOT_DEVICE_PTR: return "pointer not classifiable by the CUDA runtime";
    case PG_ERR_OOM: return "out of device memory or over the HBM budget";
    case PG_ERR_OVERFLOW: return "fixed-point photon power overflow";
    case PG_ERR_NOT_POW2: return "histogram size not a supported power of two";
    case PG_ERR_TIMEOUT: return "bounded device wait timed out";
    case PG_ERR_CUDA: return cudaGetErrorString(last_cuda_error());
    case PG_ERR_INVALID_INPUT: return "non-finite position/direction or negative photon power";
    case PG_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

pg_status pg_create(pg_ctx **out, void *stream, size_t budget) {
  if (!out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  pg_ctx *c = new (std::nothrow) pg_ctx();
  if (!c) return PG_ERR_OOM;
  memset(c, 0, sizeof(*c));
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return PG_ERR_CUDA;
  }
  c->stream = (cudaStream_t)stream;
  c->budget = budget;
  // Handles and call scratch come from the device's default stream-ordered
  // pool; keep freed blocks mapped so that repeated calls reuse them instead
  // of returning memory to the driver at every synchronisation.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
    delete c;
    return PG_ERR_CUDA;
  }
  void *hw = nullptr;
  if (cudaHostAlloc(&hw, 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&c->d_words, hw, 0) != cudaSuccess) {
    cudaGetLastError();
    if (hw) cudaFreeHost(hw);
    cudaFree(c->d_status);
    delete c;
    return PG_ERR_CUDA;
  }
  c->h_words = (volatile uint32_t *)hw;
  c->pending = new (std::nothrow) PendingFrees();
  if (!c->pending) {
    cudaFreeHost(hw);
    cudaFree(c->d_status);
    delete c;
    return PG_ERR_OOM;
  }
  *out = c;
  return PG_OK;
}

pg_status pg_destroy(pg_ctx *c) {
  if (!c) return PG_OK;
  cudaStreamSynchronize(c->stream);
  ctx_reap_frees(c, true);
  if (c->shared) pg_ctx_attach_budget(c, nullptr);
  for (int i = 0; i < 9; ++i)
    if (c->d_phi[i]) cudaFree(c->d_phi[i]);
  cudaFree(c->d_status);
  cudaFreeHost((void *)c->h_words);
  for (cudaEvent_t e : c->pending->spare) cudaEventDestroy(e);
  delete c->pending;
  delete c;
  return PG_OK;
}

pg_status pg_set_stream(pg_ctx *c, void *stream) {
  if (!c) return PG_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return PG_OK;
}

pg_status pg_sync(pg_ctx *c) {
  if (!c) return PG_ERR_INVALID_ARG;
  uint32_t st = 0;
  PG_TRY(read_words(c, c->stream, c->d_status, &st));
  PG_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream));
  ctx_reap_frees(c, false);  // every free enqueued so far has run
  if (st & ST_INVALID_INPUT) return PG_ERR_INVALID_INPUT;
  if (st & ST_OVERFLOW) return PG_ERR_OVERFLOW;
  if (st & ST_TIMEOUT) return PG_ERR_TIMEOUT;
  if (st & ST_CAPACITY) return PG_ERR_UNSUPPORTED;
  return PG_OK;
}

pg_status pg_net_get_tuning(const pg_net *netp, int32_t *out, size_t n, size_t *needed) {
  const Net *net = as<Net>(netp, KIND_NET);
  if (!net) return PG_ERR_INVALID_ARG;
  const size_t need = (size_t)net->n_layers * 3 * 7;
  if (needed) *needed = need;
  if (!out) return PG_OK;
  if (n < need) return PG_ERR_INVALID_ARG;
  for (int l = 0; l < net->n_layers; ++l)
    for (int p = 0; p < 3; ++p) {
      const Layer &L = net->layers[l];
      int32_t *o = out + ((size_t)l * 3 + p) * 7;
      o[0] = L.tc_ctas[p]; o[1] = L.tc_stages[p]; o[2] = L.tc_mt[p];
      o[3] = L.tc_halo[p]; o[4] = L.tc_cb[p]; o[5] = L.tuned_hw[p]; o[6] = L.tc_so[p];
    }
  return PG_OK;
}

pg_status pg_net_set_tuning(pg_net *netp, const int32_t *in, size_t n) {
  Net *net = as<Net>(netp, KIND_NET);
  if (!net || !in || n != (size_t)net->n_layers * 3 * 7) return PG_ERR_INVALID_ARG;
  for (size_t i = 0; i < n; i += 7)
    if (in[i] < 0 || in[i] > 4 || in[i + 1] < 0 || in[i + 1] > 24 || in[i + 2] < 0 || in[i + 2] > 4 ||
        in[i + 3] < 0 || in[i + 3] > 4 || (in[i + 4] != 0 && in[i + 4] != 32 && in[i + 4] != 64 && in[i + 4] != 128) ||
        in[i + 5] < 0 || in[i + 6] < 0 || in[i + 6] > 2)
      return PG_ERR_INVALID_ARG;
  for (int l = 0; l < net->n_layers; ++l)
    for (int p = 0; p < 3; ++p) {
      Layer &L = net->layers[l];
      const int32_t *v = in + ((size_t)l * 3 + p) * 7;
      L.tc_ctas[p] = v[0]; L.tc_stages[p] = v[1]; L.tc_mt[p] = v[2];
      L.tc_halo[p] = v[3]; L.tc_cb[p] = v[4]; L.tuned_hw[p] = v[5]; L.tc_so[p] = v[6];
    }
  return PG_OK;
}

pg_status pg_launch_count(const pg_ctx *c, uint64_t *launches) {
  if (!c || !launches) return PG_ERR_INVALID_ARG;
  *launches = c->launches;
  return PG_OK;
}

pg_status pg_bytes_in_use(const pg_ctx *c, uint64_t *bytes) {
  if (!c || !bytes) return PG_ERR_INVALID_ARG;
  *bytes = c->in_use;
  return PG_OK;
}

pg_status pg_budget_create(uint64_t capacity, pg_budget **out) {
  if (!out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  pg_budget *b = new (std::nothrow) pg_budget();
  if (!b) return PG_ERR_OOM;
  b->capacity = capacity;
  *out = b;
  return PG_OK;
}

pg_status pg_budget_destroy(pg_budget *b) {
  if (!b) return PG_OK;
  if (b->attached.load() != 0) return PG_ERR_INVALID_ARG;
  delete b;
  return PG_OK;
}

pg_status pg_ctx_attach_budget(pg_ctx *c, pg_budget *b) {
  if (!c) return PG_ERR_INVALID_ARG;
  if (b == c->shared) return PG_OK;
  if (c->shared && pending_bytes(c)) ctx_reap_frees(c, true);  // the old budget gets its bytes back first
  if (b && !budget_try_charge(b, c->in_use)) return PG_ERR_OOM;
  if (c->shared) {
    budget_release(c->shared, c->in_use);
    c->shared->attached.fetch_sub(1);
  }
  if (b) b->attached.fetch_add(1);
  c->shared = b;
  return PG_OK;
}

pg_status pg_budget_charge(pg_budget *b, uint64_t bytes) {
  if (!b) return PG_ERR_INVALID_ARG;
  return budget_try_charge(b, bytes) ? PG_OK : PG_ERR_OOM;
}

pg_status pg_budget_release(pg_budget *b, uint64_t bytes) {
  if (!b) return PG_ERR_INVALID_ARG;
  budget_release(b, bytes);
  return PG_OK;
}

pg_status pg_budget_wait(pg_budget *b, uint64_t bytes, uint64_t *generation, uint32_t timeout_ms) {
  if (!b || !generation) return PG_ERR_INVALID_ARG;
  const uint64_t seen = *generation;
  std::unique_lock<std::mutex> lk(b->mu);
  bool ok = b->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    return b->generation.load() != seen || b->in_use.load() + bytes <= b->capacity;
  });
  *generation = b->generation.load();
  return ok ? PG_OK : PG_ERR_TIMEOUT;
}

pg_status pg_budget_query(const pg_budget *b, uint64_t *in_use, uint64_t *capacity, uint64_t *generation) {
  if (!b) return PG_ERR_INVALID_ARG;
  if (in_use) *in_use = b->in_use.load();
  if (capacity) *capacity = b->capacity;
  if (generation) *generation = b->generation.load();
  return PG_OK;
}

pg_status pg_build_grid(pg_ctx *c, const pg_photon *d_ph, uint64_t n, const pg_grid_params *p, pg_grid **out) {
  if (!c || !p || !out || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
  if (p->max_depth < 0 || p->max_depth > 16 || p->min_depth < 0 || p->min_depth > 6 ||
      p->min_depth > p->max_depth)
    return PG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->lo[a]) || !isfinite(p->hi[a]) || !(p->hi[a] > p->lo[a])) return PG_ERR_INVALID_ARG;
  Staged ph;
  if (n) PG_TRY(stage_in(c, d_ph, n * sizeof(pg_photon), ph));
  Grid *g = new (std::nothrow) Grid();
  if (!g) return PG_ERR_OOM;
  memset(g, 0, sizeof(*g));
  g->h.kind = KIND_GRID;
  g->h.ctx = c;
  pg_status s = build_grid(c, (const pg_photon *)ph.dev, n, p, g);
  if (s != PG_OK) {
    if (g->block) ctx_free(c, g->block, g->h.bytes);
    delete g;
    return s;
  }
  *out = (pg_grid *)g;
  return PG_OK;
}

pg_status pg_build_grid_kd(pg_ctx *c, const pg_photon *d_ph, const float *d_normals, uint64_t n,
                           const pg_kd_params *p, pg_grid **out) {
  if (!c || !p || !out || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
  if (p->resolution < 1 || (uint64_t)p->resolution * p->resolution * p->resolution > (1ull << 27) ||
      p->max_depth < 0 || p->max_depth > 16 || !(p->normal_variance_threshold == p->normal_variance_threshold))
    return PG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->lo[a]) || !isfinite(p->hi[a]) || !(p->hi[a] > p->lo[a])) return PG_ERR_INVALID_ARG;
  Staged ph, nr;
  if (n) PG_TRY(stage_in(c, d_ph, n * sizeof(pg_photon), ph));
  if (n && d_normals) PG_TRY(stage_in(c, d_normals, n * 3 * sizeof(float), nr));
  Grid *g = new (std::nothrow) Grid();
  if (!g) return PG_ERR_OOM;
  memset(g, 0, sizeof(*g));
  g->h.kind = KIND_GRID;
  g->h.ctx = c;
  pg_status s = build_grid_kd(c, (const pg_photon *)ph.dev, d_normals ? (const float *)nr.dev : nullptr, n, p, g);
  if (s != PG_OK) {
    if (g->block) ctx_free(c, g->block, g->h.bytes);
    delete g;
    return s;
  }
  *out = (pg_grid *)g;
  return PG_OK;
}

pg_status pg_build_grid_batched(pg_ctx *c, const pg_photon *d_ph, uint64_t n, const uint32_t *d_scene_begin,
                                uint32_t S, const pg_grid_params *p, pg_grid **out) {
  if (!c || !p || !out || !d_scene_begin || S == 0 || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n >= (1ull << 31) || S > 4096) return PG_ERR_UNSUPPORTED;
  for (uint32_t s = 0; s < S; ++s) {
    if (p[s].max_depth != p[0].max_depth || p[s].min_depth != p[0].min_depth ||
        p[s].split_threshold != p[0].split_threshold)
      return PG_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
      if (!isfinite(p[s].lo[a]) || !isfinite(p[s].hi[a]) || !(p[s].hi[a] > p[s].lo[a])) return PG_ERR_INVALID_ARG;
  }
  if (p[0].max_depth < 0 || p[0].max_depth > 16 || p[0].min_depth < 0 || p[0].min_depth > p[0].max_depth)
    return PG_ERR_INVALID_ARG;
  // Scene offsets: checked on the host (non-decreasing, 0 .. n).
  uint32_t *hb = (uint32_t *)malloc(4ull * (S + 1));
  if (!hb) return PG_ERR_OOM;
  if (cudaMemcpyAsync(hb, d_scene_begin, 4ull * (S + 1), cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    free(hb);
    cudaGetLastError();
    return PG_ERR_NOT_DEVICE_PTR;
  }
  bool okb = hb[0] == 0 && hb[S] == n;
  for (uint32_t s = 0; s < S && okb; ++s) okb = hb[s] <= hb[s + 1];
  float *geom = (float *)malloc(24ull * S);
  if (!okb || !geom) {
    free(hb);
    free(geom);
    return okb ? PG_ERR_OOM : PG_ERR_INVALID_ARG;
  }
  for (uint32_t s = 0; s < S; ++s)
    for (int a = 0; a < 3; ++a) {
      geom[6 * s + a] = p[s].lo[a];
      geom[6 * s + 3 + a] = (float)(ldexp(1.0, p[0].max_depth) / ((double)p[s].hi[a] - (double)p[s].lo[a]));
    }
  Staged ph, sbeg;
  pg_status s0 = PG_OK;
  if (n) s0 = stage_in(c, d_ph, n * sizeof(pg_photon), ph);
  if (s0 == PG_OK) s0 = stage_in(c, hb, 4ull * (S + 1), sbeg);
  Grid *g = s0 == PG_OK ? new (std::nothrow) Grid() : nullptr;
  if (!g) {
    free(hb);
    free(geom);
    return s0 == PG_OK ? PG_ERR_OOM : s0;
  }
  memset(g, 0, sizeof(*g));
  g->h.kind = KIND_GRID;
  g->h.ctx = c;
  SceneBatch sb;
  sb.S = S;
  sb.d_begin = (const uint32_t *)sbeg.dev;
  sb.h_geom = geom;
  pg_status st = build_grid(c, (const pg_photon *)ph.dev, n, &p[0], g, &sb);
  free(hb);
  free(geom);
  if (st != PG_OK) {
    if (g->block) ctx_free(c, g->block, g->h.bytes);
    delete g;
    return st;
  }
  *out = (pg_grid *)g;
  return PG_OK;
}

pg_status pg_splat_photons_batched(pg_ctx *c, const pg_grid *grid, const pg_photon *d_ph, uint64_t n,
                                   const uint32_t *d_n_prev, int H, int W, int F, pg_hist **out) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  if (!c || !g || !out || !d_n_prev || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (g->kd) return PG_ERR_UNSUPPORTED;
  if (n != g->n || F < 0 || F > 62) return PG_ERR_INVALID_ARG;
  if (!pow2_in(H, 4, 256) || !pow2_in(W, 4, 256) || H * W > 16384) return PG_ERR_NOT_POW2;
  Staged ph, np;
  if (n) PG_TRY(stage_in(c, d_ph, n * sizeof(pg_photon), ph));
  PG_TRY(stage_in(c, d_n_prev, 4ull * g->n_scenes, np));
  Hist *h = new (std::nothrow) Hist();
  if (!h) return PG_ERR_OOM;
  memset(h, 0, sizeof(*h));
  h->h.kind = KIND_HIST;
  h->h.ctx = c;
  h->A = g->A;
  h->H = H;
  h->W = W;
  pg_status s = splat(c, g, (const pg_photon *)ph.dev, n, 0, F, h, (const uint32_t *)np.dev);
  if (s != PG_OK) {
    if (h->block) ctx_free(c, h->block, h->h.bytes);
    delete h;
    return s;
  }
  *out = (pg_hist *)h;
  return PG_OK;
}

pg_status pg_splat_photons(pg_ctx *c, const pg_grid *grid, const pg_photon *d_ph, uint64_t n, uint64_t n_prev,
                           int H, int W, int F, pg_hist **out) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  if (!c || !g || !out || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n != g->n || n_prev > n || F < 0 || F > 62) return PG_ERR_INVALID_ARG;
  if (!pow2_in(H, 4, 256) || !pow2_in(W, 4, 256) || H * W > 16384) return PG_ERR_NOT_POW2;
  Staged ph;
  if (n) PG_TRY(stage_in(c, d_ph, n * sizeof(pg_photon), ph));
  Hist *h = new (std::nothrow) Hist();
  if (!h) return PG_ERR_OOM;
  memset(h, 0, sizeof(*h));
  h->h.kind = KIND_HIST;
  h->h.ctx = c;
  h->A = g->A;
  h->H = H;
  h->W = W;
  pg_status s = splat(c, g, (const pg_photon *)ph.dev, n, n_prev, F, h);
  if (s != PG_OK) {
    if (h->block) ctx_free(c, h->block, h->h.bytes);
    delete h;
    return s;
  }
  *out = (pg_hist *)h;
  return PG_OK;
}

pg_status pg_net_load(pg_ctx *c, const void *blob, size_t bytes, pg_net **out) {
  if (!c || !blob || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  const uint8_t *b = (const uint8_t *)blob;
  if (bytes < 40) return PG_ERR_INVALID_ARG;
  uint32_t hdr[8];
  memcpy(hdr, b, 32);
  if (hdr[0] != 0x314E4750u || hdr[2] != 5u) return PG_ERR_INVALID_ARG;
  uint32_t arch = hdr[1], nl = hdr[3];
  static const int expect_layers[3] = {3, 15, 12};
  if (arch > 2 || nl != (uint32_t)expect_layers[arch]) return PG_ERR_UNSUPPORTED;
  Net *net = new (std::nothrow) Net();
  if (!net) return PG_ERR_OOM;
  memset(net, 0, sizeof(*net));
  net->h.kind = KIND_NET;
  net->h.ctx = c;
  net->arch = (int)arch;
  net->n_layers = (int)nl;
  for (int i = 0; i < 4; ++i) net->widths[i] = (int)hdr[4 + i];
  // First pass: parse descriptors and size the device block.
  size_t off = 40, total = 0;
  for (uint32_t l = 0; l < nl; ++l) {
    if (off + 24 > bytes) { delete net; return PG_ERR_INVALID_ARG; }
    uint32_t d[6];
    memcpy(d, b + off, 24);
    off += 24;
    Layer &L = net->layers[l];
    L.cout = (int)d[0]; L.cin = (int)d[1]; L.k = (int)d[2]; L.stride = (int)d[3]; L.act = (int)d[4];
    L.dil = d[5] ? (int)d[5] : 1;
    if (L.cout <= 0 || L.cin <= 0 || (L.k != 1 && L.k != 3) || (L.stride != 1 && L.stride != 2) || L.act > 2 ||
        (L.dil != 1 && L.dil != 2 && L.dil != 4 && L.dil != 8) || (L.dil > 1 && (L.k != 3 || L.stride != 1))) {
      delete net;
      return PG_ERR_INVALID_ARG;
    }
    size_t nw = (size_t)L.cout * L.k * L.k * L.cin;
    if (off + 4 * (nw + L.cout) > bytes) { delete net; return PG_ERR_INVALID_ARG; }
    off += 4 * (nw + L.cout);
    // The 5-channel network input is stored with 8 channels (3 zero), so the
    // first layer's weights are padded to 8 input channels.
    size_t cin_eff = (l == 0 && L.cin == 5) ? 8 : (size_t)L.cin;
    size_t nw_eff = (size_t)L.cout * L.k * L.k * cin_eff;
    total += ((4 * nw_eff + 255) & ~(size_t)255) + ((4 * (size_t)L.cout + 255) & ~(size_t)255);
  }
  void *block = nullptr;
  pg_status s = ctx_alloc(c, total, &block);
  if (s != PG_OK) { delete net; return s; }
  net->block = block;
  net->h.bytes = total;
  // Second pass: transpose [cout][k][k][cin] to the GEMM layout [k*k*cin][cout].
  off = 40;
  uint8_t *dst = (uint8_t *)block;
  for (uint32_t l = 0; l < nl; ++l) {
    Layer &L = net->layers[l];
    off += 24;
    const int cin = L.cin, cin_eff = (l == 0 && L.cin == 5) ? 8 : L.cin;
    const size_t taps = (size_t)L.k * L.k, K = taps * cin, Ke = taps * cin_eff;
    const size_t nw = K * L.cout, nwe = Ke * L.cout;
    float *tw = (float *)calloc(nwe, 4);
    if (!tw) { pg_free(net); return PG_ERR_OOM; }
    const float *src = (const float *)(b + off);
    for (int o = 0; o < L.cout; ++o)
      for (size_t t = 0; t < taps; ++t)
        for (int i = 0; i < cin; ++i) {
          float v;
          memcpy(&v, src + (size_t)o * K + t * cin + i, 4);
          tw[(t * cin_eff + i) * L.cout + o] = v;
        }
    L.cin = cin_eff;
    L.w = (float *)dst;
    cudaError_t e = cudaMemcpyAsync(L.w, tw, 4 * nwe, cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    free(tw);
    if (e != cudaSuccess) { last_cuda_error() = e; pg_free(net); return PG_ERR_CUDA; }
    dst += (4 * nwe + 255) & ~(size_t)255;
    off += 4 * nw;
    L.b = (float *)dst;
    e = cudaMemcpyAsync(L.b, b + off, 4 * (size_t)L.cout, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) { last_cuda_error() = e; pg_free(net); return PG_ERR_CUDA; }
    dst += (4 * (size_t)L.cout + 255) & ~(size_t)255;
    off += 4 * (size_t)L.cout;
  }
  PG_CUDA(cudaStreamSynchronize(c->stream));
  *out = (pg_net *)net;
  return PG_OK;
}

pg_status pg_reconstruct(pg_ctx *c, const pg_hist *hist, const pg_net *netp, pg_precision prec, pg_map **out) {
  const Hist *h = as<Hist>(hist, KIND_HIST);
  Net *net = as<Net>(netp, KIND_NET);
  if (!c || !h || !net || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != PG_FP32 && prec != PG_BF16 && prec != PG_FP8_E4M3 && prec != PG_FP8_MIXED) return PG_ERR_INVALID_ARG;
  if (net->arch >= 1 && (h->H < 8 || h->W < 8)) return PG_ERR_UNSUPPORTED;
  PG_TRY(net_prepare(c, net, prec));
  Map *m = new (std::nothrow) Map();
  if (!m) return PG_ERR_OOM;
  memset(m, 0, sizeof(*m));
  m->h.kind = KIND_MAP;
  m->h.ctx = c;
  m->A = h->A;
  m->H = h->H;
  m->W = h->W;
  m->h.bytes = (size_t)m->A * h->H * h->W * sizeof(float);
  pg_status s = ctx_alloc(c, m->h.bytes, &m->block);
  if (s == PG_OK) {
    m->y = (float *)m->block;
    s = reconstruct(c, h, net, prec, m);
  }
  if (s != PG_OK) {
    if (m->block) ctx_free(c, m->block, m->h.bytes);
    delete m;
    return s;
  }
  *out = (pg_map *)m;
  return PG_OK;
}

pg_status pg_reconstruct_experts(pg_ctx *c, const pg_hist *hist, const pg_net *const *nets, int n_experts,
                                 const uint32_t *count_bounds, pg_precision prec, pg_map **out) {
  const Hist *h = as<Hist>(hist, KIND_HIST);
  if (!c || !h || !nets || !out || n_experts < 1 || n_experts > 16 || (n_experts > 1 && !count_bounds))
    return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != PG_FP32 && prec != PG_BF16 && prec != PG_FP8_E4M3 && prec != PG_FP8_MIXED) return PG_ERR_INVALID_ARG;
  Net *ns[16];
  for (int e = 0; e < n_experts; ++e) {
    ns[e] = as<Net>(nets[e], KIND_NET);
    if (!ns[e]) return PG_ERR_INVALID_ARG;
    if (ns[e]->arch >= 1 && (h->H < 8 || h->W < 8)) return PG_ERR_UNSUPPORTED;
    if (e + 1 < n_experts && e > 0 && count_bounds[e] <= count_bounds[e - 1]) return PG_ERR_INVALID_ARG;
  }
  const uint32_t A = h->A;
  const size_t HW = (size_t)h->H * h->W;
  // BF16 U-Net experts: grouped on the device and run as one launch per
  // layer over every expert's tiles (no host read-back of the counts).
  bool grouped = prec == PG_BF16 && n_experts > 1 && A > 0;
  for (int e = 0; e < n_experts && grouped; ++e) grouped = ns[e]->arch == 1;
  if (grouped) {
    for (int e = 0; e < n_experts; ++e) PG_TRY(net_prepare(c, ns[e], prec));
    Map *m = new (std::nothrow) Map();
    if (!m) return PG_ERR_OOM;
    memset(m, 0, sizeof(*m));
    m->h.kind = KIND_MAP;
    m->h.ctx = c;
    m->A = A;
    m->H = h->H;
    m->W = h->W;
    m->h.bytes = (size_t)A * HW * sizeof(float);
    pg_status s = ctx_alloc(c, m->h.bytes, &m->block);
    if (s == PG_OK) {
      m->y = (float *)m->block;
      s = reconstruct_experts_grouped(c, h, (const Net *const *)ns, n_experts, count_bounds, m->y);
    }
    if (s == PG_OK) {
      *out = (pg_map *)m;
      return PG_OK;
    }
    pg_free(m);
    if (s != PG_ERR_UNSUPPORTED) return s;
  }
  // Photon count of every leaf -> expert (the number of bounds <= count),
  // and the leaves grouped by expert, each group in slot order.
  std::vector<uint32_t> cnt(A), perm(A);
  std::vector<uint32_t> first(n_experts + 1, 0);
  if (A) {
    uint32_t *d_cnt;
    PG_TRY(ctx_alloc(c, 4ull * A, (void **)&d_cnt));
    pg_status s = leaf_counts(c, h, d_cnt);
    if (s == PG_OK && (cudaMemcpyAsync(cnt.data(), d_cnt, 4ull * A, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                       cudaStreamSynchronize(c->stream) != cudaSuccess))
      s = PG_ERR_CUDA;
    ctx_free(c, d_cnt, 4ull * A);
    PG_TRY(s);
    std::vector<int> ex(A);
    for (uint32_t k = 0; k < A; ++k) {
      int e = 0;
      while (e + 1 < n_experts && cnt[k] >= count_bounds[e]) ++e;
      ex[k] = e;
      ++first[e + 1];
    }
    for (int e = 0; e < n_experts; ++e) first[e + 1] += first[e];
    std::vector<uint32_t> at(first.begin(), first.end() - 1);
    for (uint32_t k = 0; k < A; ++k) perm[at[ex[k]]++] = k;
  }
  for (int e = 0; e < n_experts; ++e)
    if (first[e + 1] > first[e]) PG_TRY(net_prepare(c, ns[e], prec));
  Map *m = new (std::nothrow) Map();
  if (!m) return PG_ERR_OOM;
  memset(m, 0, sizeof(*m));
  m->h.kind = KIND_MAP;
  m->h.ctx = c;
  m->A = A;
  m->H = h->H;
  m->W = h->W;
  m->h.bytes = (size_t)A * HW * sizeof(float);
  pg_status s = ctx_alloc(c, m->h.bytes, &m->block);
  if (s == PG_OK) m->y = (float *)m->block;
  int used = 0;
  for (int e = 0; e < n_experts; ++e) used += first[e + 1] > first[e] ? 1 : 0;
  if (s == PG_OK && used <= 1) {
    // One expert (or none) has leaves: it runs over all of them in place.
    int e = 0;
    while (e + 1 < n_experts && first[e + 1] == first[e]) ++e;
    s = reconstruct(c, h, ns[e], prec, m);
  } else if (s == PG_OK) {
    // Each expert runs over its leaves (contiguous positions of `perm`) into
    // a position-ordered map, which one scatter returns to slot order.
    uint32_t *d_perm = nullptr;
    float *yp = nullptr;
    const size_t yb = (size_t)A * HW * sizeof(float);
    s = ctx_alloc(c, 4ull * A, (void **)&d_perm);
    if (s == PG_OK) s = ctx_alloc(c, yb, (void **)&yp);
    if (s == PG_OK && cudaMemcpyAsync(d_perm, perm.data(), 4ull * A, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      s = PG_ERR_CUDA;
    for (int e = 0; e < n_experts && s == PG_OK; ++e)
      if (first[e + 1] > first[e])
        s = reconstruct_range(c, h, ns[e], prec, yp + (size_t)first[e] * HW, d_perm, first[e], first[e + 1] - first[e]);
    if (s == PG_OK) s = scatter_rows(c, yp, d_perm, A, (int)HW, m->y);
    if (s == PG_OK) s = cudaStreamSynchronize(c->stream) == cudaSuccess ? PG_OK : PG_ERR_CUDA;  // perm is host memory
    if (yp) ctx_free(c, yp, yb);
    if (d_perm) ctx_free(c, d_perm, 4ull * A);
  }
  if (s != PG_OK) {
    if (m->block) ctx_free(c, m->block, m->h.bytes);
    delete m;
    return s;
  }
  *out = (pg_map *)m;
  return PG_OK;
}

pg_status pg_mis_create(pg_ctx *c, const pg_grid *grid, pg_mis **out) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  if (!c || !g || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (g->n_scenes != 1) return PG_ERR_UNSUPPORTED;
  Mis *m = new (std::nothrow) Mis();
  if (!m) return PG_ERR_OOM;
  memset(m, 0, sizeof(*m));
  m->h.kind = KIND_MIS;
  m->h.ctx = c;
  m->L = g->L;
  const size_t L = g->L, b8 = (8 * L + 255) & ~(size_t)255, b4 = (4 * L + 255) & ~(size_t)255;
  m->h.bytes = 2 * b8 + 3 * b4;
  pg_status s = ctx_alloc(c, m->h.bytes, &m->block);
  if (s != PG_OK) {
    delete m;
    return s;
  }
  uint8_t *p = (uint8_t *)m->block;
  m->nu_b = (double *)p;
  m->nu_g = (double *)(p + b8);
  m->q_b = (uint32_t *)(p + 2 * b8);
  m->q_g = (uint32_t *)(p + 2 * b8 + b4);
  m->alpha = (float *)(p + 2 * b8 + 2 * b4);
  s = mis_init(c, m);
  if (s != PG_OK) {
    pg_free(m);
    return s;
  }
  *out = (pg_mis *)m;
  return PG_OK;
}

pg_status pg_mis_accumulate(pg_ctx *c, pg_mis *misp, const pg_grid *grid, const float *d_pos,
                            const uint8_t *d_strategy, const float *d_contrib, uint64_t q) {
  Mis *m = as<Mis>(misp, KIND_MIS);
  const Grid *g = as<Grid>(grid, KIND_GRID);
  if (!c || !m || !g || (q && (!d_pos || !d_strategy || !d_contrib))) return PG_ERR_INVALID_ARG;
  if (g->L != m->L || g->n_scenes != 1) return PG_ERR_INVALID_ARG;
  if (q == 0) return PG_OK;
  Staged pos, st, co;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_strategy, q, st));
  PG_TRY(stage_in(c, d_contrib, q * 4, co));
  return mis_accumulate(c, m, g, (const float *)pos.dev, (const uint8_t *)st.dev, (const float *)co.dev, q);
}

pg_status pg_mis_update(pg_ctx *c, pg_mis *misp, uint32_t min_count, float alpha_lo, float alpha_hi) {
  Mis *m = as<Mis>(misp, KIND_MIS);
  if (!c || !m || !(alpha_lo >= 0.0f) || !(alpha_hi <= 1.0f) || !(alpha_lo <= alpha_hi)) return PG_ERR_INVALID_ARG;
  return mis_update(c, m, min_count, alpha_lo, alpha_hi);
}

pg_status pg_mis_sample(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const pg_mis *misp, const float *d_pos,
                        const float *d_normal, uint64_t q, uint64_t seed, uint32_t stream_id, float *d_dir,
                        float *d_pdf, uint8_t *d_strategy) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  const Mis *m = as<Mis>(misp, KIND_MIS);
  if (!c || !g || !t || !m || (q && (!d_pos || !d_normal || !d_dir || !d_pdf || !d_strategy)))
    return PG_ERR_INVALID_ARG;
  if (t->A != g->A || m->L != g->L || g->n_scenes != 1) return PG_ERR_INVALID_ARG;
  if (q == 0) return PG_OK;
  Staged pos, nrm, dir, pdf, st;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_normal, q * 12, nrm));
  PG_TRY(stage_out(c, d_dir, q * 12, dir));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  PG_TRY(stage_out(c, d_strategy, q, st));
  PG_TRY(mis_sample(c, g, t, m, (const float *)pos.dev, (const float *)nrm.dev, q, seed, stream_id, (float *)dir.dev,
                    (float *)pdf.dev, (uint8_t *)st.dev));
  PG_TRY(finish_out(dir));
  PG_TRY(finish_out(pdf));
  PG_TRY(finish_out(st));
  return PG_OK;
}

pg_status pg_mis_eval(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const pg_mis *misp, const float *d_pos,
                      const float *d_normal, const float *d_dir, uint64_t q, float *d_pdf) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  const Mis *m = as<Mis>(misp, KIND_MIS);
  if (!c || !g || !t || !m || (q && (!d_pos || !d_normal || !d_dir || !d_pdf))) return PG_ERR_INVALID_ARG;
  if (t->A != g->A || m->L != g->L || g->n_scenes != 1) return PG_ERR_INVALID_ARG;
  if (q == 0) return PG_OK;
  Staged pos, nrm, dir, pdf;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_normal, q * 12, nrm));
  PG_TRY(stage_in(c, d_dir, q * 12, dir));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  PG_TRY(mis_eval(c, g, t, m, (const float *)pos.dev, (const float *)nrm.dev, (const float *)dir.dev, q,
                  (float *)pdf.dev));
  PG_TRY(finish_out(pdf));
  return PG_OK;
}

pg_status pg_autotune(pg_ctx *c, const pg_hist *hist, pg_net *netp, pg_precision prec) {
  const Hist *h = as<Hist>(hist, KIND_HIST);
  Net *net = as<Net>(netp, KIND_NET);
  if (!c || !h || !net) return PG_ERR_INVALID_ARG;
  if (prec != PG_BF16 && prec != PG_FP8_E4M3 && prec != PG_FP8_MIXED) return PG_OK;  // FP32: nothing to tune
  if (h->A == 0) return PG_OK;
  PG_TRY(net_prepare(c, net, prec));
  Map m;
  memset(&m, 0, sizeof(m));
  m.A = h->A;
  m.H = h->H;
  m.W = h->W;
  size_t bytes = (size_t)h->A * h->H * h->W * sizeof(float);
  void *block = nullptr;
  PG_TRY(ctx_alloc(c, bytes, &block));
  m.y = (float *)block;
  pg_status s = reconstruct(c, h, net, prec, &m, true);
  ctx_free(c, block, bytes);
  return s;
}

pg_status pg_map_import(pg_ctx *c, const float *d_y, uint64_t n_maps, int H, int W, pg_map **out) {
  if (!c || !out || (n_maps && !d_y)) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!pow2_in(H, 4, 256) || !pow2_in(W, 4, 256) || H * W > 16384) return PG_ERR_NOT_POW2;
  if (n_maps >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
  Map *m = new (std::nothrow) Map();
  if (!m) return PG_ERR_OOM;
  memset(m, 0, sizeof(*m));
  m->h.kind = KIND_MAP;
  m->h.ctx = c;
  m->A = (uint32_t)n_maps;
  m->H = H;
  m->W = W;
  m->h.bytes = (size_t)n_maps * H * W * sizeof(float);
  pg_status s = ctx_alloc(c, m->h.bytes, &m->block);
  if (s != PG_OK) { delete m; return s; }
  m->y = (float *)m->block;
  if (n_maps) {
    cudaError_t e = cudaMemcpyAsync(m->y, d_y, m->h.bytes, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) { last_cuda_error() = e; pg_free(m); return PG_ERR_CUDA; }
  }
  *out = (pg_map *)m;
  return PG_OK;
}

pg_status pg_build_cdf(pg_ctx *c, const pg_map *map, pg_tables **out) {
  const Map *m = as<Map>(map, KIND_MAP);
  if (!c || !m || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  Tables *t = new (std::nothrow) Tables();
  if (!t) return PG_ERR_OOM;
  memset(t, 0, sizeof(*t));
  t->h.kind = KIND_TABLES;
  t->h.ctx = c;
  t->A = m->A;
  t->H = m->H;
  t->W = m->W;
  size_t HW = (size_t)m->H * m->W, A = m->A;
  size_t bP = (A * HW * 4 + 255) & ~(size_t)255, bz = (A * m->H * 4 + 255) & ~(size_t)255;
  // Segment summaries (every 8th CDF entry) for rows of 16 or more bins.
  size_t bsp = m->W >= 16 ? (A * HW / 8 * 4 + 255) & ~(size_t)255 : 0;
  size_t bsz = m->H >= 16 ? (A * m->H / 8 * 4 + 255) & ~(size_t)255 : 0;
  size_t bv = (A + 255) & ~(size_t)255;
  t->h.bytes = 2 * bP + bz + bsp + bsz + bv;
  pg_status s = ctx_alloc(c, t->h.bytes, &t->block);
  if (s != PG_OK) { delete t; return s; }
  uint8_t *p = (uint8_t *)t->block;
  t->P = (float *)p;
  t->cdf_phi = (float *)(p + bP);
  t->cdf_z = (float *)(p + 2 * bP);
  t->sum_phi = bsp ? (float *)(p + 2 * bP + bz) : nullptr;
  t->sum_z = bsz ? (float *)(p + 2 * bP + bz + bsp) : nullptr;
  t->valid = p + 2 * bP + bz + bsp + bsz;
  s = build_cdf(c, m, t);
  if (s != PG_OK) { pg_free(t); return s; }
  *out = (pg_tables *)t;
  return PG_OK;
}

pg_status pg_sample_dirs(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const float *d_pos, uint64_t q,
                         uint64_t seed, uint32_t stream_id, float *d_dir, float *d_pdf, uint32_t *d_leaf,
                         uint32_t *d_bin) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  if (!c || !g || !t || (q && (!d_pos || !d_dir || !d_pdf || !d_leaf))) return PG_ERR_INVALID_ARG;
  if (t->A != g->A) return PG_ERR_INVALID_ARG;
  if (q == 0) return PG_OK;
  Staged pos, dir, pdf, leaf, bin;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_out(c, d_dir, q * 12, dir));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  PG_TRY(stage_out(c, d_leaf, q * 4, leaf));
  if (d_bin) PG_TRY(stage_out(c, d_bin, q * 4, bin));
  PG_TRY(sample(c, g, t, (const float *)pos.dev, q, seed, stream_id, (float *)dir.dev, (float *)pdf.dev,
                (uint32_t *)leaf.dev, d_bin ? (uint32_t *)bin.dev : nullptr));
  PG_TRY(finish_out(dir));
  PG_TRY(finish_out(pdf));
  PG_TRY(finish_out(leaf));
  if (d_bin) PG_TRY(finish_out(bin));
  return PG_OK;
}

pg_status pg_sample_dirs_batched(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const float *d_pos,
                                 const uint32_t *d_query_begin, uint64_t q, uint64_t seed, const uint32_t *d_stream_ids,
                                 float *d_dir, float *d_pdf, uint32_t *d_leaf, uint32_t *d_bin) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  if (!c || !g || !t || !d_query_begin || !d_stream_ids || (q && (!d_pos || !d_dir || !d_pdf || !d_leaf)))
    return PG_ERR_INVALID_ARG;
  if (t->A != g->A) return PG_ERR_INVALID_ARG;
  if (g->kd) return PG_ERR_UNSUPPORTED;  // scene batches are octree grids
  if (q == 0) return PG_OK;
  if (q >= (1ull << 32)) return PG_ERR_UNSUPPORTED;
  Staged pos, qb, sid, dir, pdf, leaf, bin;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_query_begin, 4ull * (g->n_scenes + 1), qb));
  PG_TRY(stage_in(c, d_stream_ids, 4ull * g->n_scenes, sid));
  PG_TRY(stage_out(c, d_dir, q * 12, dir));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  PG_TRY(stage_out(c, d_leaf, q * 4, leaf));
  if (d_bin) PG_TRY(stage_out(c, d_bin, q * 4, bin));
  QueryScenes qs;
  qs.d_qbegin = (const uint32_t *)qb.dev;
  qs.d_streams = (const uint32_t *)sid.dev;
  PG_TRY(sample(c, g, t, (const float *)pos.dev, q, seed, 0, (float *)dir.dev, (float *)pdf.dev,
                (uint32_t *)leaf.dev, d_bin ? (uint32_t *)bin.dev : nullptr, qs));
  PG_TRY(finish_out(dir));
  PG_TRY(finish_out(pdf));
  PG_TRY(finish_out(leaf));
  if (d_bin) PG_TRY(finish_out(bin));
  return PG_OK;
}

pg_status pg_eval_pdf_batched(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const float *d_pos,
                              const float *d_dir, const uint32_t *d_query_begin, uint64_t q, float *d_pdf) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  if (!c || !g || !t || !d_query_begin || (q && (!d_pos || !d_dir || !d_pdf))) return PG_ERR_INVALID_ARG;
  if (t->A != g->A) return PG_ERR_INVALID_ARG;
  if (g->kd) return PG_ERR_UNSUPPORTED;  // scene batches are octree grids
  if (q == 0) return PG_OK;
  if (q >= (1ull << 32)) return PG_ERR_UNSUPPORTED;
  Staged pos, dir, qb, pdf;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_dir, q * 12, dir));
  PG_TRY(stage_in(c, d_query_begin, 4ull * (g->n_scenes + 1), qb));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  QueryScenes qs;
  qs.d_qbegin = (const uint32_t *)qb.dev;
  qs.d_streams = nullptr;
  PG_TRY(eval_pdf(c, g, t, (const float *)pos.dev, (const float *)dir.dev, q, (float *)pdf.dev, qs));
  PG_TRY(finish_out(pdf));
  return PG_OK;
}

pg_status pg_eval_pdf(pg_ctx *c, const pg_grid *grid, const pg_tables *tab, const float *d_pos, const float *d_dir,
                      uint64_t q, float *d_pdf) {
  const Grid *g = as<Grid>(grid, KIND_GRID);
  const Tables *t = as<Tables>(tab, KIND_TABLES);
  if (!c || !g || !t || (q && (!d_pos || !d_dir || !d_pdf))) return PG_ERR_INVALID_ARG;
  if (t->A != g->A) return PG_ERR_INVALID_ARG;
  if (q == 0) return PG_OK;
  Staged pos, dir, pdf;
  PG_TRY(stage_in(c, d_pos, q * 12, pos));
  PG_TRY(stage_in(c, d_dir, q * 12, dir));
  PG_TRY(stage_out(c, d_pdf, q * 4, pdf));
  PG_TRY(eval_pdf(c, g, t, (const float *)pos.dev, (const float *)dir.dev, q, (float *)pdf.dev));
  PG_TRY(finish_out(pdf));
  return PG_OK;
}

pg_status pg_progress_create(pg_ctx *c, const pg_progress_params *p, pg_progress **out) {
  if (!c || !p || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->max_depth < 0 || p->max_depth > 16 || p->min_depth < 0 || p->min_depth > 6 ||
      p->min_depth > p->max_depth)
    return PG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->lo[a]) || !isfinite(p->hi[a]) || !(p->hi[a] > p->lo[a])) return PG_ERR_INVALID_ARG;
  if (!isfinite(p->split_c) || !(p->split_c >= 0.0) || p->refine_iterations < 0 || p->refine_iterations > 31 ||
      p->frac_bits < 0 || p->frac_bits > 62 || p->max_photons == 0 || p->max_photons >= (1ull << 31))
    return PG_ERR_INVALID_ARG;
  if (p->grid_rule != 0 && p->grid_rule != 1) return PG_ERR_INVALID_ARG;
  if (p->grid_rule == 1 &&
      (p->resolution < 1 || (uint64_t)p->resolution * p->resolution * p->resolution > (1ull << 27) ||
       !(p->normal_variance_threshold == p->normal_variance_threshold)))
    return PG_ERR_INVALID_ARG;
  if (!pow2_in(p->H, 4, 256) || !pow2_in(p->W, 4, 256) || p->H * p->W > 16384) return PG_ERR_NOT_POW2;
  Progress *s = new (std::nothrow) Progress();
  if (!s) return PG_ERR_OOM;
  memset(s, 0, sizeof(*s));
  s->h.kind = KIND_PROGRESS;
  s->h.ctx = c;
  s->p = *p;
  s->normals = -1;
  if (p->refine_iterations == 0) {  // the unrefined grid, for good
    pg_status st = progress_regrid(c, s, 0, 0xFFFFFFFFu);
    if (st != PG_OK) {
      free_progress(s);
      return st;
    }
  }
  *out = (pg_progress *)s;
  return PG_OK;
}

pg_status pg_progress_add_photons(pg_ctx *c, pg_progress *sp, const pg_photon *d_ph, uint64_t n) {
  return pg_progress_add_photons_normals(c, sp, d_ph, nullptr, n);
}

pg_status pg_progress_add_photons_normals(pg_ctx *c, pg_progress *sp, const pg_photon *d_ph, const float *d_nrm,
                                          uint64_t n) {
  Progress *s = as<Progress>(sp, KIND_PROGRESS);
  if (!c || !s || (n && !d_ph)) return PG_ERR_INVALID_ARG;
  if (n > s->p.max_photons || s->total + n > s->p.max_photons) return PG_ERR_INVALID_ARG;
  const uint32_t t = s->t;
  const bool refining = (int64_t)t < s->p.refine_iterations;
  const int with_n = d_nrm ? 1 : 0;
  if (refining && s->p.grid_rule == 1 && s->normals >= 0 && s->normals != with_n) return PG_ERR_INVALID_ARG;
  Staged ph, nr;
  if (n) PG_TRY(stage_in(c, d_ph, n * sizeof(pg_photon), ph));
  const bool keep_n = refining && s->p.grid_rule == 1 && with_n;
  if (n && keep_n) PG_TRY(stage_in(c, d_nrm, n * 3 * sizeof(float), nr));
  if (refining) {
    if (s->n_stored + n > s->cap_stored) {
      const uint64_t cap = std::max<uint64_t>(2 * s->cap_stored, s->n_stored + n);
      void *b, *bn = nullptr;
      PG_TRY(ctx_alloc(c, cap * sizeof(pg_photon), &b));
      if (keep_n) {
        pg_status sa = ctx_alloc(c, cap * 3 * sizeof(float), &bn);
        if (sa != PG_OK) {
          ctx_free(c, b, cap * sizeof(pg_photon));
          return sa;
        }
      }
      if (s->n_stored) {
        PG_CUDA(cudaMemcpyAsync(b, s->stored, s->n_stored * sizeof(pg_photon), cudaMemcpyDeviceToDevice, c->stream));
        if (keep_n && s->stored_n)
          PG_CUDA(cudaMemcpyAsync(bn, s->stored_n, s->n_stored * 3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                  c->stream));
      }
      ctx_free(c, s->stored, s->cap_stored * sizeof(pg_photon));
      ctx_free(c, s->stored_n, s->cap_stored * 3 * sizeof(float));
      s->stored = (pg_photon *)b;
      s->stored_n = (float *)bn;
      s->cap_stored = cap;
    }
    if (n) {
      PG_CUDA(cudaMemcpyAsync(s->stored + s->n_stored, ph.dev, n * sizeof(pg_photon), cudaMemcpyDeviceToDevice,
                              c->stream));
      if (keep_n)
        PG_CUDA(cudaMemcpyAsync(s->stored_n + 3 * s->n_stored, nr.dev, n * 3 * sizeof(float),
                                cudaMemcpyDeviceToDevice, c->stream));
    }
    if (s->p.grid_rule == 1) s->normals = with_n;
    const uint64_t n_prev = s->n_stored;
    s->n_stored += n;
    // M_thr = c sqrt(2^t); counts are integers, so count > M_thr <=> count > floor(M_thr).
    const double m_thr = floor(s->p.split_c * sqrt(ldexp(1.0, (int)t)));
    const uint32_t thr = m_thr >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)m_thr;
    pg_status st = progress_regrid(c, s, n_prev, thr);
    if (st != PG_OK) {
      s->n_stored = n_prev;
      return st;
    }
    if ((int64_t)t + 1 == s->p.refine_iterations) {  // the grid is fixed from here on
      ctx_free(c, s->stored, s->cap_stored * sizeof(pg_photon));
      ctx_free(c, s->stored_n, s->cap_stored * 3 * sizeof(float));
      s->stored = nullptr;
      s->stored_n = nullptr;
      s->n_stored = s->cap_stored = 0;
    }
  } else {
    Grid view;
    void *scr = nullptr;
    size_t sb = 0;
    Grid *g = s->grid;
    pg_status st = g->kd ? bin_into_grid_kd(c, g, (const pg_photon *)ph.dev, n, &view, &scr, &sb)
                         : bin_into_grid(c, g, (const pg_photon *)ph.dev, n, &view, &scr, &sb);
    // Leaves that receive their first photons take the next slots.
    uint32_t fresh = 0;
    if (st == PG_OK) st = assign_slots(c, view.A, view.active, g, &fresh);
    const uint32_t A0 = g->A, A1 = A0 + fresh;
    if (st == PG_OK && A1 > s->cap_slots) {
      const uint32_t cap = std::max<uint32_t>(2 * s->cap_slots, A1);
      st = hist_grow(c, s->cum, A0, cap);
      if (st == PG_OK) st = map_grow(c, s->map, A0, cap);
      if (st == PG_OK) s->cap_slots = cap;
    }
    if (st == PG_OK) {
      g->A = A1;
      s->cum->A = A1;
      s->map->A = A1;
      st = splat_merge(c, &view, (const pg_photon *)ph.dev, s->p.max_photons, s->p.frac_bits, g->slot_of_leaf,
                       s->cum);
    }
    if (st == PG_OK) st = progress_reserve_updated(c, s, view.A);
    if (st == PG_OK) st = slots_of(c, view.A, view.active, g, s->updated);
    if (st == PG_OK) s->n_updated = view.A;
    ctx_free(c, scr, sb);
    if (st != PG_OK) return st;
  }
  s->t = t + 1;
  s->total += n;
  return PG_OK;
}

pg_status pg_progress_reconstruct(pg_ctx *c, pg_progress *sp, const pg_net *netp, pg_precision prec) {
  Progress *s = as<Progress>(sp, KIND_PROGRESS);
  Net *net = as<Net>(netp, KIND_NET);
  if (!c || !s || !net || !s->grid) return PG_ERR_INVALID_ARG;
  if (prec != PG_FP32 && prec != PG_BF16 && prec != PG_FP8_E4M3 && prec != PG_FP8_MIXED) return PG_ERR_INVALID_ARG;
  if (net->arch >= 1 && (s->p.H < 8 || s->p.W < 8)) return PG_ERR_UNSUPPORTED;
  PG_TRY(net_prepare(c, net, prec));
  const uint32_t A = s->n_updated;
  const int HW = s->p.H * s->p.W;
  if (A) {
    void *yp;
    PG_TRY(ctx_alloc(c, (size_t)A * HW * sizeof(float), &yp));
    pg_status st = reconstruct_range(c, s->cum, net, prec, (float *)yp, s->updated, 0, A);
    if (st == PG_OK) st = scatter_rows(c, (const float *)yp, s->updated, A, HW, s->map->y);
    ctx_free(c, yp, (size_t)A * HW * sizeof(float));
    if (st != PG_OK) return st;
  }
  pg_tables *t = nullptr;
  PG_TRY(pg_build_cdf(c, (const pg_map *)s->map, &t));
  ((Handle *)t)->borrowed = 1;
  release_owned(s->tab);
  s->tab = (Tables *)t;
  return PG_OK;
}

pg_status pg_progress_view(const pg_progress *sp, const pg_grid **grid, const pg_hist **planes, const pg_map **map,
                           const pg_tables **tables) {
  const Progress *s = as<Progress>(sp, KIND_PROGRESS);
  if (!s) return PG_ERR_INVALID_ARG;
  if (grid) *grid = (const pg_grid *)s->grid;
  if (planes) *planes = (const pg_hist *)s->cum;
  if (map) *map = (const pg_map *)s->map;
  if (tables) *tables = (const pg_tables *)s->tab;
  return PG_OK;
}

pg_status pg_info(const void *handle, int what, uint64_t *v) {
  if (!handle || !v) return PG_ERR_INVALID_ARG;
  const Handle *b = (const Handle *)handle;
  switch (b->kind) {
    case KIND_GRID: {
      const Grid *g = (const Grid *)handle;
      if (what == PG_INFO_N_PHOTONS) *v = g->n;
      else if (what == PG_INFO_N_LEAVES) *v = g->L;
      else if (what == PG_INFO_N_ACTIVE) *v = g->A;
      else if (what == PG_INFO_MAX_DEPTH) *v = (uint64_t)g->D;
      else if (what == PG_INFO_N_SCENES) *v = g->n_scenes;
      else if (what == PG_INFO_SCENE_LEVELS) *v = (uint64_t)g->scene_levels;
      else if (what == PG_INFO_KD_NODES && g->kd) *v = g->kd_nodes;
      else if (what == PG_INFO_BYTES) *v = b->bytes;
      else return PG_ERR_INVALID_ARG;
      return PG_OK;
    }
    case KIND_HIST: case KIND_MAP: case KIND_TABLES: {
      uint32_t A; int H, W;
      if (b->kind == KIND_HIST) { const Hist *h = (const Hist *)handle; A = h->A; H = h->H; W = h->W; }
      else if (b->kind == KIND_MAP) { const Map *m = (const Map *)handle; A = m->A; H = m->H; W = m->W; }
      else { const Tables *t = (const Tables *)handle; A = t->A; H = t->H; W = t->W; }
      if (what == PG_INFO_N_ACTIVE) *v = A;
      else if (what == PG_INFO_H) *v = (uint64_t)H;
      else if (what == PG_INFO_W) *v = (uint64_t)W;
      else if (what == PG_INFO_BYTES) *v = b->bytes;
      else return PG_ERR_INVALID_ARG;
      return PG_OK;
    }
    case KIND_NET:
      if (what == PG_INFO_BYTES) { *v = b->bytes; return PG_OK; }
      return PG_ERR_INVALID_ARG;
    case KIND_MIS:
      if (what == PG_INFO_N_LEAVES) { *v = ((const Mis *)handle)->L; return PG_OK; }
      if (what == PG_INFO_BYTES) { *v = b->bytes; return PG_OK; }
      return PG_ERR_INVALID_ARG;
    case KIND_PROGRESS: {
      const Progress *s = (const Progress *)handle;
      if (what == PG_INFO_ITERATION) *v = s->t;
      else if (what == PG_INFO_N_UPDATED) *v = s->n_updated;
      else if (what == PG_INFO_N_PHOTONS) *v = s->total;
      else if (what == PG_INFO_N_LEAVES) *v = s->grid ? s->grid->L : 0;
      else if (what == PG_INFO_H) *v = (uint64_t)s->p.H;
      else if (what == PG_INFO_W) *v = (uint64_t)s->p.W;
      else return PG_ERR_INVALID_ARG;
      return PG_OK;
    }
  }
  return PG_ERR_INVALID_ARG;
}

pg_status pg_export(pg_ctx *c, const void *handle, int what, void *dst, size_t bytes) {
  if (!c || !handle || (bytes && !dst)) return PG_ERR_INVALID_ARG;
  const Handle *b = (const Handle *)handle;
  const void *src = nullptr;
  size_t need = 0;
  if (b->kind == KIND_GRID) {
    const Grid *g = (const Grid *)handle;
    switch (what) {
      case PG_GRID_CODES: src = g->codes; need = g->n * 8; break;
      case PG_GRID_PERM: src = g->perm; need = g->n * 4; break;
      case PG_GRID_LEAF_OF: src = g->leaf_of; need = g->n * 4; break;
      case PG_GRID_LEAF_CODE: src = g->leaf_code; need = (size_t)g->L * 8; break;
      case PG_GRID_LEAF_DEPTH: src = g->leaf_depth; need = (size_t)g->L * 4; break;
      case PG_GRID_LEAF_BEGIN: src = g->leaf_begin; need = (size_t)g->L * 4; break;
      case PG_GRID_LEAF_END: src = g->leaf_end; need = (size_t)g->L * 4; break;
      case PG_GRID_ACTIVE: src = g->active; need = (size_t)g->A * 4; break;
      case PG_GRID_SLOT_OF_LEAF: src = g->slot_of_leaf; need = (size_t)g->L * 4; break;
      case PG_GRID_SCENE_LEAF_BEGIN: src = g->scene_leaf_begin; need = 4ull * (g->n_scenes + 1); break;
      case PG_GRID_KD_AXIS: src = g->kd ? (const void *)g->kd_axis : nullptr; need = g->kd ? g->kd_nodes : 0; break;
      case PG_GRID_KD_TAU: src = g->kd ? (const void *)g->kd_tau : nullptr; need = g->kd ? 4ull * g->kd_nodes : 0; break;
      case PG_GRID_KD_LINK: src = g->kd ? (const void *)g->kd_link : nullptr; need = g->kd ? 4ull * g->kd_nodes : 0; break;
      default: return PG_ERR_INVALID_ARG;
    }
  } else if (b->kind == KIND_HIST) {
    const Hist *h = (const Hist *)handle;
    size_t n = (size_t)h->A * h->H * h->W;
    switch (what) {
      case PG_HIST_POW_CUR: src = h->pow_cur; need = n * 8; break;
      case PG_HIST_CNT_CUR: src = h->cnt_cur; need = n * 4; break;
      case PG_HIST_POW_PREV: src = h->pow_prev; need = n * 8; break;
      case PG_HIST_CNT_PREV: src = h->cnt_prev; need = n * 4; break;
      default: return PG_ERR_INVALID_ARG;
    }
  } else if (b->kind == KIND_MAP) {
    const Map *m = (const Map *)handle;
    if (what != PG_MAP_Y) return PG_ERR_INVALID_ARG;
    src = m->y;
    need = (size_t)m->A * m->H * m->W * 4;
  } else if (b->kind == KIND_TABLES) {
    const Tables *t = (const Tables *)handle;
    size_t n = (size_t)t->A * t->H * t->W;
    switch (what) {
      case PG_TAB_P: src = t->P; need = n * 4; break;
      case PG_TAB_CDF_PHI: src = t->cdf_phi; need = n * 4; break;
      case PG_TAB_CDF_Z: src = t->cdf_z; need = (size_t)t->A * t->H * 4; break;
      case PG_TAB_VALID: src = t->valid; need = t->A; break;
      default: return PG_ERR_INVALID_ARG;
    }
  } else if (b->kind == KIND_MIS) {
    const Mis *m = (const Mis *)handle;
    switch (what) {
      case PG_MIS_NU_B: src = m->nu_b; need = (size_t)m->L * 8; break;
      case PG_MIS_NU_G: src = m->nu_g; need = (size_t)m->L * 8; break;
      case PG_MIS_Q_B: src = m->q_b; need = (size_t)m->L * 4; break;
      case PG_MIS_Q_G: src = m->q_g; need = (size_t)m->L * 4; break;
      case PG_MIS_ALPHA: src = m->alpha; need = (size_t)m->L * 4; break;
      default: return PG_ERR_INVALID_ARG;
    }
  } else if (b->kind == KIND_PROGRESS) {
    const Progress *s = (const Progress *)handle;
    if (what != PG_PROGRESS_UPDATED) return PG_ERR_INVALID_ARG;
    src = s->updated;
    need = 4ull * s->n_updated;
  } else {
    return PG_ERR_INVALID_ARG;
  }
  if (bytes != need) return PG_ERR_INVALID_ARG;
  if (need == 0) return PG_OK;
  PG_CUDA(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return PG_OK;
}

void pg_free(void *handle) {
  if (!handle) return;
  Handle *b = (Handle *)handle;
  if (b->borrowed) return;
  if (b->kind == KIND_PROGRESS) {
    free_progress((Progress *)handle);
    return;
  }
  void *block = nullptr;
  switch (b->kind) {
    case KIND_GRID: block = ((Grid *)handle)->block; break;
    case KIND_HIST: block = ((Hist *)handle)->block; break;
    case KIND_NET: {
      Net *n = (Net *)handle;
      block = n->block;
      for (int i = 0; i < n->n_layers; ++i) {
        if (n->layers[i].w_bf16) ctx_free(b->ctx, n->layers[i].w_bf16, n->layers[i].w_bf16_bytes);
        if (n->layers[i].w_fp8) ctx_free(b->ctx, n->layers[i].w_fp8, n->layers[i].w_fp8_bytes);
        if (n->layers[i].w_ph_bf16) ctx_free(b->ctx, n->layers[i].w_ph_bf16, n->layers[i].w_ph_bytes);
        for (int e = 0; e < 2; ++e)
          for (int o = 0; o < 3; ++o)
            for (int c = 0; c < 3; ++c)
              if (n->layers[i].bimg[e][o][c])
                ctx_free_static(b->ctx, n->layers[i].bimg[e][o][c], n->layers[i].bimg_bytes[e][o][c]);
      }
      break;
    }
    case KIND_MAP: block = ((Map *)handle)->block; break;
    case KIND_TABLES: block = ((Tables *)handle)->block; break;
    case KIND_MIS: block = ((Mis *)handle)->block; break;
    default: return;
  }
  ctx_free(b->ctx, block, b->bytes);
  uint32_t kind = b->kind;
  b->kind = 0;
  switch (kind) {
    case KIND_GRID: delete (Grid *)handle; break;
    case KIND_HIST: delete (Hist *)handle; break;
    case KIND_NET: delete (Net *)handle; break;
    case KIND_MIS: delete (Mis *)handle; break;
    case KIND_MAP: delete (Map *)handle; break;
    default: delete (Tables *)handle; break;
  }
}

}  // extern "C"
