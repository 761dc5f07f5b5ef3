// Progressive iterations (Sec. 7.1, 7.2; Algorithm 1): photon batches of
// doubling size arrive one iteration at a time.  Every leaf keeps its energy
// and count maps summed over all iterations so far and, for the network's
// previous-iteration channels, the sums as they stood before the last
// iteration that brought it photons.  These kernels lay out those
// leaf-indexed planes after a refining iteration (the merge of a later batch
// is the splat kernel's merge mode); the iteration logic is in the C ABI
// layer.
#include "pg_internal.cuh"

namespace pgi {

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// dst[active[a]] = src[a] for the four planes and both totals; dst rows of
// leaves not in the list are left as they are.
__global__ void k_rows_to_leaves(const uint64_t *__restrict__ spc, const uint32_t *__restrict__ scc,
                                 const uint64_t *__restrict__ spp, const uint32_t *__restrict__ scp,
                                 const uint64_t *__restrict__ stc, const uint64_t *__restrict__ stp,
                                 const uint32_t *__restrict__ active, int HW, uint64_t *__restrict__ dpc,
                                 uint32_t *__restrict__ dcc, uint64_t *__restrict__ dpp, uint32_t *__restrict__ dcp,
                                 uint64_t *__restrict__ dtc, uint64_t *__restrict__ dtp) {
  const uint32_t a = blockIdx.x, l = active[a];
  const size_t s0 = (size_t)a * HW, d0 = (size_t)l * HW;
  for (int k = threadIdx.x; k < HW; k += blockDim.x) {
    dpc[d0 + k] = spc[s0 + k];
    dcc[d0 + k] = scc[s0 + k];
    dpp[d0 + k] = spp[s0 + k];
    dcp[d0 + k] = scp[s0 + k];
  }
  if (threadIdx.x == 0) {
    dtc[l] = stc[a];
    dtp[l] = stp[a];
  }
}

__global__ void k_identity_slots(int32_t *__restrict__ slot_of_leaf, uint32_t *__restrict__ active, uint32_t L) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  slot_of_leaf[l] = (int32_t)l;
  active[l] = l;
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

pg_status rows_to_leaves(pg_ctx *ctx, const Hist *src, const uint32_t *d_active, Hist *dst) {
  if (src->A == 0) return PG_OK;
  k_rows_to_leaves<<<src->A, 256, 0, ctx->stream>>>(src->pow_cur, src->cnt_cur, src->pow_prev, src->cnt_prev,
                                                    src->tot_cur, src->tot_prev, d_active, src->H * src->W,
                                                    dst->pow_cur, dst->cnt_cur, dst->pow_prev, dst->cnt_prev,
                                                    dst->tot_cur, dst->tot_prev), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status identity_slots(pg_ctx *ctx, Grid *g) {
  if (g->L) {
    k_identity_slots<<<ceil_div(g->L, 256), 256, 0, ctx->stream>>>(g->slot_of_leaf, g->active, g->L),
        PG_COUNT(ctx);
    PG_CUDA(cudaGetLastError());
  }
  g->A = g->L;
  return PG_OK;
}

}  // namespace pgi
