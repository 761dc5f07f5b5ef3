// a5: photon energy and count maps (Eq. "photon" of Sec. 4; the count maps
// P_{e,t}, P_{e,t-1} and the previous-iteration map of Sec. 5).
//
// One CTA per active leaf.  The leaf's photons are the contiguous range of
// the sorted permutation; each thread gathers a 32-byte photon record, takes
// its direction bin and fixed-point power and adds into a shared-memory
// histogram (64-bit power, 32-bit count); the record loads of up to three
// photons per thread are issued together.  Photons of one warp that land in
// the same bin are combined first (warp match), so a hot bin costs one shared
// atomic per warp instead of one per photon.  The finished histogram is
// written once, coalesced, with the per-leaf power totals.  Histograms up to
// 8192 bins keep all four planes in shared memory (24 B/bin = 192 KB); at
// 16384 bins the current and previous planes run as two launches.
#include "pg_internal.cuh"

namespace pgi {

namespace {

constexpr int kSplatThreads = 512;

// Bulk asynchronous copy shared -> global (16-byte aligned, size a multiple
// of 16 bytes), completion tracked by the issuing thread's bulk group.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
               : "memory");
}

// kMode 0: all four planes; 1: current planes only; 2: previous planes only;
// 3: merge into leaf-indexed running sums (progressive iterations): the
// leaf's previous planes take its current sums, and the current planes add
// this batch.
template <int kMode>
__global__ void __launch_bounds__(kSplatThreads) k_splat(
    const pg_photon *__restrict__ ph, const uint32_t *__restrict__ perm, const uint32_t *__restrict__ active,
    const uint32_t *__restrict__ leaf_begin, const uint32_t *__restrict__ leaf_end, uint32_t n_prev, int H, int W,
    float two_f, uint64_t limit, const float *__restrict__ phi_tab, uint64_t *__restrict__ pow_cur,
    uint32_t *__restrict__ cnt_cur, uint64_t *__restrict__ pow_prev, uint32_t *__restrict__ cnt_prev,
    uint64_t *__restrict__ tot_cur, uint64_t *__restrict__ tot_prev, uint32_t *status,
    const uint64_t *__restrict__ leaf_code, const uint32_t *__restrict__ sc_begin,
    const uint32_t *__restrict__ sc_nprev, int sc_shift, const int32_t *__restrict__ merge_slot) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kPlanes = kMode == 0 ? 2 : 1;
  const int HW = H * W;
  unsigned long long *s_pow = reinterpret_cast<unsigned long long *>(smem);  // [kPlanes][HW]
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_pow + kPlanes * HW);         // [kPlanes][HW]
  float *s_tab = reinterpret_cast<float *>(s_cnt + kPlanes * HW);               // [2W]
  __shared__ unsigned long long s_tot[2][kSplatThreads / 32];

  const uint32_t slot = blockIdx.x;
  const uint32_t leaf = active[slot];
  const uint32_t b = leaf_begin[leaf], e = leaf_end[leaf];
  // "Previous iteration" photons: original index below n_prev, counted
  // within the leaf's scene for a scene batch.
  // A scene of a batch has the overflow bound of the same scene alone,
  // (2^63 - 1) / (its photon count).
  uint32_t prev_base = 0, prev_lim = n_prev;
  if (sc_nprev) {
    const uint32_t sc = (uint32_t)(leaf_code[leaf] >> sc_shift);
    prev_base = sc_begin[sc];
    prev_lim = sc_nprev[sc];
    limit = (uint64_t)INT64_MAX / (uint64_t)(sc_begin[sc + 1] - prev_base);
  }
  const int tid = threadIdx.x, lane = tid & 31;

  // The leaf's photons go in batches of kU x 512: each thread first issues
  // the permutation loads of its kU photons, then their record loads (all
  // independent), so a batch costs two memory round trips instead of two per
  // photon; the first batch's loads are in flight while the shared
  // histogram is zeroed.
  constexpr int kU = 3;
  uint32_t bad = 0;
  bool zeroed = false;
  for (uint64_t base = b; base < e || !zeroed; base += kU * kSplatThreads) {
    uint32_t pidx[kU];
    bool live[kU];
    float4 ra[kU], rb[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint64_t i = base + (uint64_t)(u * kSplatThreads + tid);
      live[u] = i < e;
      pidx[u] = live[u] ? __ldg(perm + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (live[u]) {
        const float4 *r = reinterpret_cast<const float4 *>(ph + pidx[u]);
        ra[u] = __ldg(r);
        rb[u] = __ldg(r + 1);
      } else {
        ra[u] = rb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (!zeroed) {
      uint4 *z = reinterpret_cast<uint4 *>(smem);
      const int n16 = (kPlanes * HW * 12) / 16;
      for (int k = tid; k < n16; k += kSplatThreads) z[k] = make_uint4(0, 0, 0, 0);
      for (int k = tid; k < 2 * W; k += kSplatThreads) s_tab[k] = phi_tab[k];
      __syncthreads();
      zeroed = true;
      if (base >= e) break;  // no photons (not an active leaf): zeroed planes only
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
    if (base + (uint64_t)u * kSplatThreads < e) {  // skip the part of the batch past the leaf (uniform)
    int bin = -1;
    unsigned long long pfx = 0;
    bool prev = false;
    if (live[u]) {
      const uint32_t p = pidx[u];
      float dx = ra[u].w, dy = rb[u].x, dz = rb[u].y, power = rb[u].z;
      int row = 0, col = 0;
      if (isfinite(dx) && isfinite(dy) && isfinite(dz)) {
        row = dir_row(dz, H);
        col = dir_col(dx, dy, W, s_tab);
      } else {
        bad |= ST_INVALID_INPUT;
      }
      bin = row * W + col;
      if (!(power >= 0.0f) || !isfinite(power)) {
        bad |= ST_INVALID_INPUT;
      } else {
        float v = __fmul_rn(power, two_f);  // exact: scaling by a power of two
        if (v >= 9.2233720368547758e18f) {
          bad |= ST_OVERFLOW;
        } else {
          pfx = __float2ull_rn(v);
          if (pfx > limit) {
            bad |= ST_OVERFLOW;
            pfx = 0;
          }
        }
      }
      prev = p - prev_base < prev_lim;
      if (kMode == 2 && !prev) bin = -1;
    }
    // Combine photons of this warp that share a bin.
    unsigned peers = __match_any_sync(0xFFFFFFFFu, bin);
    int leader = __ffs(peers) - 1;
    unsigned long long gsum = pfx;
    uint32_t gcnt = 1, gsum_p_cnt = prev ? 1u : 0u;
    unsigned long long gsum_p = prev ? pfx : 0ull;
    // Sum over the peer group by walking its lanes (all group members loop
    // the same number of times).
    {
      unsigned rest = peers & ~(1u << leader);
      gsum = __shfl_sync(peers, pfx, leader);
      gsum_p = __shfl_sync(peers, prev ? pfx : 0ull, leader);
      gsum_p_cnt = __shfl_sync(peers, prev ? 1u : 0u, leader);
      while (rest) {
        int l = __ffs(rest) - 1;
        rest &= rest - 1;
        gsum += __shfl_sync(peers, pfx, l);
        gsum_p += __shfl_sync(peers, prev ? pfx : 0ull, l);
        gsum_p_cnt += __shfl_sync(peers, prev ? 1u : 0u, l);
      }
      gcnt = __popc(peers);
    }
    if (lane == leader && bin >= 0) {
      if (kMode == 0) {
        atomicAdd(&s_pow[bin], gsum);
        atomicAdd(&s_cnt[bin], gcnt);
        if (gsum_p_cnt) {
          atomicAdd(&s_pow[HW + bin], gsum_p);
          atomicAdd(&s_cnt[HW + bin], gsum_p_cnt);
        }
      } else if (kMode == 1 || kMode == 3) {
        atomicAdd(&s_pow[bin], gsum);
        atomicAdd(&s_cnt[bin], gcnt);
      } else {
        atomicAdd(&s_pow[bin], gsum_p);
        atomicAdd(&s_cnt[bin], gsum_p_cnt);
      }
    }
    }  // a live part of the batch
    }  // kU photons of the batch
  }
  if (bad) atomicOr(status, bad);
  __syncthreads();

  if (kMode == 3) {
    // Read-modify-write of the leaf's slot rows, coalesced; totals likewise.
    const uint32_t row = (uint32_t)merge_slot[leaf];
    const size_t o = (size_t)row * HW;
    unsigned long long t_add = 0;
    for (int k = tid; k < HW; k += kSplatThreads) {
      const unsigned long long add = s_pow[k];
      const unsigned long long p0 = pow_cur[o + k];
      const uint32_t c0 = cnt_cur[o + k];
      pow_prev[o + k] = p0;
      cnt_prev[o + k] = c0;
      pow_cur[o + k] = p0 + add;
      cnt_cur[o + k] = c0 + s_cnt[k];
      t_add += add;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) t_add += __shfl_xor_sync(0xFFFFFFFFu, t_add, off);
    if (lane == 0) s_tot[0][tid >> 5] = t_add;
    __syncthreads();
    if (tid == 0) {
      unsigned long long a = 0;
      for (int w = 0; w < kSplatThreads / 32; ++w) a += s_tot[0][w];
      const unsigned long long t0 = tot_cur[row];
      tot_prev[row] = t0;
      tot_cur[row] = t0 + a;
    }
    return;
  }

  // Flush: the finished planes leave shared memory as bulk asynchronous
  // copies issued by one thread, so the CTA can retire (and the next leaf's
  // CTA start on this SM) while its histogram drains to HBM; the per-leaf
  // totals come from a block reduction over the shared planes.
  const size_t o = (size_t)slot * HW;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // atomics above -> bulk-copy reads below
  unsigned long long t_cur = 0, t_prev = 0;
  const int P = kMode == 0 ? HW : 0;
  for (int k = tid; k < HW; k += kSplatThreads) {
    if (kMode != 2) t_cur += s_pow[k];
    if (kMode != 1) t_prev += s_pow[P + k];
  }
  __syncthreads();
  if (tid == 0) {
    if (kMode != 2) {
      bulk_store(pow_cur + o, s_pow, 8u * HW);
      bulk_store(cnt_cur + o, s_cnt, 4u * HW);
    }
    if (kMode != 1) {
      bulk_store(pow_prev + o, s_pow + P, 8u * HW);
      bulk_store(cnt_prev + o, s_cnt + P, 4u * HW);
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    t_cur += __shfl_xor_sync(0xFFFFFFFFu, t_cur, off);
    t_prev += __shfl_xor_sync(0xFFFFFFFFu, t_prev, off);
  }
  if (lane == 0) {
    s_tot[0][tid >> 5] = t_cur;
    s_tot[1][tid >> 5] = t_prev;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0, c = 0;
    for (int w = 0; w < kSplatThreads / 32; ++w) {
      a += s_tot[0][w];
      c += s_tot[1][w];
    }
    if (kMode != 2) tot_cur[slot] = a;
    if (kMode != 1) tot_prev[slot] = c;
    // Shared memory must outlive the copies' reads of it (not their writes).
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

pg_status splat_merge(pg_ctx *ctx, const Grid *view, const pg_photon *d_ph, uint64_t n_bound, int F,
                      const int32_t *d_slot_of_leaf, Hist *cum) {
  if (view->A == 0) return PG_OK;
  const size_t HW = (size_t)cum->H * cum->W;
  const float *tab;
  PG_TRY(phi_table(ctx, cum->W, &tab));
  const float two_f = ldexpf(1.0f, F);
  const uint64_t limit = n_bound ? (uint64_t)INT64_MAX / n_bound : 0;
  const size_t smem = 12 * HW + 8 * (size_t)cum->W;
  PG_CUDA(cudaFuncSetAttribute(k_splat<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_splat<3><<<(unsigned)view->A, kSplatThreads, smem, ctx->stream>>>(
      d_ph, view->perm, view->active, view->leaf_begin, view->leaf_end, 0u, cum->H, cum->W, two_f, limit, tab,
      cum->pow_cur, cum->cnt_cur, cum->pow_prev, cum->cnt_prev, cum->tot_cur, cum->tot_prev, ctx->d_status,
      view->leaf_code, view->scene_begin, nullptr, 3 * view->D, d_slot_of_leaf), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status splat(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n, uint64_t n_prev, int F, Hist *h,
                const uint32_t *d_scene_nprev) {
  const size_t A = g->A, HW = (size_t)h->H * h->W;
  size_t b64 = align256(8 * A * HW), b32 = align256(4 * A * HW), bt = align256(8 * A);
  h->h.bytes = 2 * b64 + 2 * b32 + 2 * bt;
  PG_TRY(ctx_alloc(ctx, h->h.bytes, &h->block));
  uint8_t *q = (uint8_t *)h->block;
  h->pow_cur = (uint64_t *)q; q += b64;
  h->pow_prev = (uint64_t *)q; q += b64;
  h->cnt_cur = (uint32_t *)q; q += b32;
  h->cnt_prev = (uint32_t *)q; q += b32;
  h->tot_cur = (uint64_t *)q; q += bt;
  h->tot_prev = (uint64_t *)q;
  if (A == 0) return PG_OK;
  const float *tab;
  PG_TRY(phi_table(ctx, h->W, &tab));
  const float two_f = ldexpf(1.0f, F);
  const uint64_t limit = n ? (uint64_t)INT64_MAX / n : 0;
  const bool one_pass = HW <= 8192;
  if (one_pass) {
    size_t smem = 24 * HW + 8 * (size_t)h->W;
    PG_CUDA(cudaFuncSetAttribute(k_splat<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_splat<0><<<(unsigned)A, kSplatThreads, smem, ctx->stream>>>(
        d_ph, g->perm, g->active, g->leaf_begin, g->leaf_end, (uint32_t)n_prev, h->H, h->W, two_f, limit, tab,
        h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev, h->tot_cur, h->tot_prev, ctx->d_status, g->leaf_code,
        g->scene_begin, d_scene_nprev, 3 * g->D, nullptr), PG_COUNT(ctx);
  } else {
    size_t smem = 12 * HW + 8 * (size_t)h->W;
    PG_CUDA(cudaFuncSetAttribute(k_splat<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PG_CUDA(cudaFuncSetAttribute(k_splat<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_splat<1><<<(unsigned)A, kSplatThreads, smem, ctx->stream>>>(
        d_ph, g->perm, g->active, g->leaf_begin, g->leaf_end, (uint32_t)n_prev, h->H, h->W, two_f, limit, tab,
        h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev, h->tot_cur, h->tot_prev, ctx->d_status, g->leaf_code,
        g->scene_begin, d_scene_nprev, 3 * g->D, nullptr), PG_COUNT(ctx);
    k_splat<2><<<(unsigned)A, kSplatThreads, smem, ctx->stream>>>(
        d_ph, g->perm, g->active, g->leaf_begin, g->leaf_end, (uint32_t)n_prev, h->H, h->W, two_f, limit, tab,
        h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev, h->tot_cur, h->tot_prev, ctx->d_status, g->leaf_code,
        g->scene_begin, d_scene_nprev, 3 * g->D, nullptr), PG_COUNT(ctx);
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
