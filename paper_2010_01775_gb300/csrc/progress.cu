// Progressive iterations (Sec. 7.1, 7.2; Algorithm 1): photon batches of
// doubling size arrive one iteration at a time.  Every leaf with photons
// owns a map slot whose planes hold its energy and count maps summed over
// all iterations so far and, for the network's previous-iteration channels,
// the sums as they stood before the last iteration that brought it photons.
// These kernels hand out slots to leaves that first receive photons and grow
// the slot arrays; the merge of a batch is the splat kernel's merge mode and
// the iteration logic is in the C ABI layer.
#include "pg_internal.cuh"

namespace pgi {

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Leaves of a batch (ascending) that have no slot yet take slots A0, A0+1, ...
// in that order; *count gets their number.  One block.
__global__ void __launch_bounds__(1024) k_assign_slots(uint32_t nA, const uint32_t *__restrict__ leaves,
                                                       int32_t *__restrict__ slot_of_leaf,
                                                       uint32_t *__restrict__ slot_leaf, uint32_t A0,
                                                       uint32_t *__restrict__ count) {
  __shared__ uint32_t sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nA; base += blockDim.x) {
    const uint32_t a = base + threadIdx.x;
    const uint32_t l = a < nA ? leaves[a] : 0u;
    const uint32_t f = (a < nA && slot_of_leaf[l] < 0) ? 1u : 0u;
    // Exclusive block scan of f.
    uint32_t x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = lane < nw ? sh[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
      }
      sh[lane] = v;
    }
    __syncthreads();
    const uint32_t p = (warp ? sh[warp - 1] : 0u) + x - f;
    const uint32_t tot = sh[nw - 1];
    __syncthreads();
    if (f) {
      slot_of_leaf[l] = (int32_t)(A0 + carry + p);
      slot_leaf[A0 + carry + p] = l;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void k_slots_of(uint32_t nA, const uint32_t *__restrict__ leaves, const int32_t *__restrict__ slot_of_leaf,
                           uint32_t *__restrict__ out) {
  const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < nA) out[a] = (uint32_t)slot_of_leaf[leaves[a]];
}

__global__ void k_iota_slots(uint32_t n, uint32_t *__restrict__ out) {
  const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) out[a] = a;
}

}  // namespace

pg_status hist_alloc(pg_ctx *ctx, Hist *h, uint32_t A, int H, int W) {
  const size_t HW = (size_t)H * W;
  const size_t b64 = align256(8 * (size_t)A * HW), b32 = align256(4 * (size_t)A * HW), bt = align256(8 * (size_t)A);
  h->A = A;
  h->H = H;
  h->W = W;
  h->h.bytes = 2 * b64 + 2 * b32 + 2 * bt;
  PG_TRY(ctx_alloc(ctx, h->h.bytes, &h->block));
  uint8_t *q = (uint8_t *)h->block;
  h->pow_cur = (uint64_t *)q; q += b64;
  h->pow_prev = (uint64_t *)q; q += b64;
  h->cnt_cur = (uint32_t *)q; q += b32;
  h->cnt_prev = (uint32_t *)q; q += b32;
  h->tot_cur = (uint64_t *)q; q += bt;
  h->tot_prev = (uint64_t *)q;
  PG_CUDA(cudaMemsetAsync(h->block, 0, h->h.bytes, ctx->stream));
  return PG_OK;
}

pg_status hist_grow(pg_ctx *ctx, Hist *h, uint32_t rows, uint32_t cap) {
  Hist n;
  memset(&n, 0, sizeof(n));
  n.h = h->h;
  PG_TRY(hist_alloc(ctx, &n, cap, h->H, h->W));
  const size_t HW = (size_t)h->H * h->W;
  cudaStream_t st = ctx->stream;
  if (rows) {
    PG_CUDA(cudaMemcpyAsync(n.pow_cur, h->pow_cur, 8 * rows * HW, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(n.pow_prev, h->pow_prev, 8 * rows * HW, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(n.cnt_cur, h->cnt_cur, 4 * rows * HW, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(n.cnt_prev, h->cnt_prev, 4 * rows * HW, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(n.tot_cur, h->tot_cur, 8ull * rows, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(n.tot_prev, h->tot_prev, 8ull * rows, cudaMemcpyDeviceToDevice, st));
  }
  ctx_free(ctx, h->block, h->h.bytes);
  const Handle keep = h->h;
  *h = n;
  h->h.kind = keep.kind;
  h->h.borrowed = keep.borrowed;
  h->h.ctx = keep.ctx;
  h->h.bytes = n.h.bytes;
  h->A = rows;
  return PG_OK;
}

pg_status map_grow(pg_ctx *ctx, Map *m, uint32_t rows, uint32_t cap) {
  const size_t HW = (size_t)m->H * m->W, bytes = (size_t)cap * HW * sizeof(float);
  void *b;
  PG_TRY(ctx_alloc(ctx, bytes, &b));
  PG_CUDA(cudaMemsetAsync(b, 0, bytes, ctx->stream));
  if (rows) PG_CUDA(cudaMemcpyAsync(b, m->y, (size_t)rows * HW * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx_free(ctx, m->block, m->h.bytes);
  m->block = b;
  m->y = (float *)b;
  m->h.bytes = bytes;
  m->A = rows;
  return PG_OK;
}

pg_status assign_slots(pg_ctx *ctx, uint32_t nA, const uint32_t *d_leaves, Grid *g, uint32_t *new_slots) {
  *new_slots = 0;
  if (nA == 0) return PG_OK;
  void *d_count;
  PG_TRY(ctx_alloc(ctx, 256, &d_count));
  k_assign_slots<<<1, 1024, 0, ctx->stream>>>(nA, d_leaves, g->slot_of_leaf, g->active, g->A, (uint32_t *)d_count),
      PG_COUNT(ctx);
  const pg_status s = read_words(ctx, ctx->stream, (const uint32_t *)d_count, new_slots);
  ctx_free(ctx, d_count, 256);
  return s;
}

pg_status slots_of(pg_ctx *ctx, uint32_t nA, const uint32_t *d_leaves, const Grid *g, uint32_t *d_out) {
  if (nA == 0) return PG_OK;
  k_slots_of<<<ceil_div(nA, 256), 256, 0, ctx->stream>>>(nA, d_leaves, g->slot_of_leaf, d_out), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status iota_slots(pg_ctx *ctx, uint32_t n, uint32_t *d_out) {
  if (n == 0) return PG_OK;
  k_iota_slots<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(n, d_out), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
