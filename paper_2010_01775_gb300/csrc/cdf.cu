// a8-a9: sampling map and CDFs (Eq. energy_target; Sec. 7.3: the CDF is a
// cumulative sum over the map pixels, as for an environment map).
//
// One CTA per map.  Each row is split over T consecutive lanes, N bins per
// lane: a lane sums its bins in sequence, a T-lane shuffle scan joins the
// segments, and the conditional CDF of the row is prefix / row sum (1 in the
// last bin, uniform for an empty row).  Warp 0 then scans the row sums into
// the marginal CDF, and all threads write P = y / sum y.  Sequential sums in
// each lane keep the pair arithmetic below to about a third of what a
// 32-lane scan per row costs.  Every 8th CDF entry is also written to a
// segment summary that the samplers search first.
//
// Sums, prefixes and quotients carry ~48 significant bits without FP64:
// each value is an unevaluated pair (hi, lo) of FP32 numbers combined with
// error-free transformations (Knuth's TwoSum for additions, an FMA-exact
// product for the quotient's correction step).  GB300 runs FP64 at a small
// fraction of its FP32 rate, and a double-FP32 add is a handful of FP32
// operations.  The pair is rounded to FP32 only when the table is stored.
#include "pg_internal.cuh"

namespace pgi {

namespace {

struct df {
  float hi, lo;
};

// s + e = a + b exactly (any a, b; round-to-nearest).
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Renormalise when |a| >= |b|.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_from(float a) { return {a, 0.0f}; }

// x / y to ~2^-45 relative, rounded to FP32 (x, y >= 0, y > 0).
__device__ __forceinline__ float df_div_to_f32(df x, df y) {
  float q1 = __fdiv_rn(x.hi, y.hi);
  float p = __fmul_rn(q1, y.hi);
  float pe = __fmaf_rn(q1, y.hi, -p);  // exact low part of q1 * y.hi
  float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), __fsub_rn(x.lo, __fmul_rn(q1, y.lo)));
  float q2 = __fdiv_rn(r, y.hi);
  return __fadd_rn(q1, q2);
}

// 1 / y as a pair (y > 0).
__device__ __forceinline__ df df_recip(df y) {
  float r1 = __fdiv_rn(1.0f, y.hi);
  float p = __fmul_rn(r1, y.hi);
  float pe = __fmaf_rn(r1, y.hi, -p);
  float res = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(r1, y.lo));
  return fast_two_sum(r1, __fdiv_rn(res, y.hi));
}

// x * r rounded to FP32, with the product's error term kept (x, r pairs).
__device__ __forceinline__ float df_mul_to_f32(df x, df r) {
  float p = __fmul_rn(x.hi, r.hi);
  float pe = __fmaf_rn(x.hi, r.hi, -p);
  float t = __fmaf_rn(x.hi, r.lo, __fmaf_rn(x.lo, r.hi, pe));
  return __fadd_rn(p, t);
}

__device__ __forceinline__ df shfl_up_df(df v, int o) {
  return {__shfl_up_sync(0xFFFFFFFFu, v.hi, o), __shfl_up_sync(0xFFFFFFFFu, v.lo, o)};
}

__device__ __forceinline__ df warp_incl_scan_df(df x) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    df y = shfl_up_df(x, o);
    if (lane >= o) x = df_add(x, y);
  }
  return x;
}

template <int N>
__device__ __forceinline__ void load_seg(const float *__restrict__ p, float (&v)[N]) {
#pragma unroll
  for (int e = 0; e < N; e += 4) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p + e));
    v[e] = t.x; v[e + 1] = t.y; v[e + 2] = t.z; v[e + 3] = t.w;
  }
}

template <int N>
__device__ __forceinline__ void store_seg(float *__restrict__ p, const float (&v)[N]) {
#pragma unroll
  for (int e = 0; e < N; e += 4) *reinterpret_cast<float4 *>(p + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
}

// Warp 0: the marginal CDF over the row sums and the map total.
__device__ __forceinline__ void marginal_cdf(int H, const float *mrow_hi, const float *mrow_lo, float *__restrict__ cz,
                                             float *__restrict__ sz, uint8_t *__restrict__ valid, df *s_total) {
  const int lane = threadIdx.x & 31;
  const int EH = (H + 31) >> 5;
  df pref[8], run = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    int i = lane * EH + e;
    if (e < EH && i < H) run = df_add(run, df{mrow_hi[i], mrow_lo[i]});
    pref[e] = run;
  }
  df incl = warp_incl_scan_df(run);
  df off = {__shfl_up_sync(0xFFFFFFFFu, incl.hi, 1), __shfl_up_sync(0xFFFFFFFFu, incl.lo, 1)};
  if (lane == 0) off = {0.0f, 0.0f};
  df total = {__shfl_sync(0xFFFFFFFFu, incl.hi, 31), __shfl_sync(0xFFFFFFFFu, incl.lo, 31)};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    int i = lane * EH + e;
    if (e < EH && i < H) {
      const float f = i == H - 1 ? 1.0f : (total.hi > 0.0f ? df_div_to_f32(df_add(off, pref[e]), total) : 0.0f);
      cz[(size_t)blockIdx.x * H + i] = f;
      if (sz && (i & 7) == 7) sz[(size_t)blockIdx.x * (H >> 3) + (i >> 3)] = f;  // segment summary
    }
  }
  if (lane == 0) {
    *s_total = total;
    valid[blockIdx.x] = total.hi > 0.0f ? 1 : 0;
  }
}

// One CTA (256 threads) per map.  A row of W = N*T bins belongs to T
// consecutive lanes, each holding N consecutive bins (N = min(W, 16)), so a
// pass covers 256/T rows: a 64x64 map is one pass with every bin loaded
// once.  A lane sums its N bins in sequence, a T-lane shuffle scan gives its
// offset and the row sum, and a second sweep of its bins forms the prefixes.
// When the map fits one pass the bins stay in registers for P = y / sum y;
// taller maps re-read them.
// With W >= 16 (N = 16) every lane also writes entries 7 and 15 of its
// segment to the row's segment summary (sphi); sz likewise for the marginal.
template <int N, int T>
__global__ void __launch_bounds__(256) k_cdf(const float *__restrict__ y, int H, int W, float *__restrict__ P,
                                             float *__restrict__ cphi, float *__restrict__ cz,
                                             float *__restrict__ sphi, float *__restrict__ sz,
                                             uint8_t *__restrict__ valid) {
  constexpr int RP = 256 / T;
  __shared__ float mrow_hi[256], mrow_lo[256];
  __shared__ df s_total;
  const int tid = threadIdx.x;
  const int q = tid % T;  // = lane % T: the T lanes of a row are one shuffle segment
  const size_t HW = (size_t)H * W, base = (size_t)blockIdx.x * HW;
  float v[N];
  int i = 0;
  for (int r0 = 0; r0 < H; r0 += RP) {
    i = r0 + tid / T;
    const bool has = i < H;  // lanes past the last row still join the shuffles
    const size_t o = base + (size_t)i * W + q * N;
    if (has) load_seg<N>(y + o, v);
    else
#pragma unroll
      for (int e = 0; e < N; ++e) v[e] = 0.0f;
    df tot = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < N; ++e) tot = df_add(tot, df_from(v[e]));
    df incl = tot;
#pragma unroll
    for (int s = 1; s < T; s <<= 1) {
      df u = {__shfl_up_sync(0xFFFFFFFFu, incl.hi, s, T), __shfl_up_sync(0xFFFFFFFFu, incl.lo, s, T)};
      if (q >= s) incl = df_add(incl, u);
    }
    df off = {__shfl_up_sync(0xFFFFFFFFu, incl.hi, 1, T), __shfl_up_sync(0xFFFFFFFFu, incl.lo, 1, T)};
    if (q == 0) off = {0.0f, 0.0f};
    const df m = {__shfl_sync(0xFFFFFFFFu, incl.hi, T - 1, T), __shfl_sync(0xFFFFFFFFu, incl.lo, T - 1, T)};
    if (!has) continue;
    if (q == 0) {
      mrow_hi[i] = m.hi;
      mrow_lo[i] = m.lo;
    }
    float out[N];
    if (m.hi > 0.0f) {
      const df rm = df_recip(m);
      df run = off;
#pragma unroll
      for (int e = 0; e < N; ++e) {
        run = df_add(run, df_from(v[e]));
        out[e] = q * N + e == W - 1 ? 1.0f : df_mul_to_f32(run, rm);
      }
    } else {
#pragma unroll
      for (int e = 0; e < N; ++e) out[e] = (float)(q * N + e + 1) / (float)W;
    }
    store_seg<N>(cphi + o, out);
    if constexpr (N == 16) {
      if (sphi)
        *reinterpret_cast<float2 *>(sphi + ((size_t)blockIdx.x * H + i) * (W >> 3) + 2 * q) = make_float2(out[7], out[15]);
    }
  }
  __syncthreads();
  if (tid < 32) marginal_cdf(H, mrow_hi, mrow_lo, cz, sz, valid, &s_total);
  __syncthreads();
  const df total = s_total;
  const float inv = total.hi > 0.0f ? df_div_to_f32(df{1.0f, 0.0f}, total) : 0.0f;
  if (H <= RP) {
    if (i < H) {
      float out[N];
#pragma unroll
      for (int e = 0; e < N; ++e) out[e] = total.hi > 0.0f ? v[e] * inv : 0.0f;
      store_seg<N>(P + base + (size_t)i * W + q * N, out);
    }
  } else {
    for (size_t k = 4 * tid; k < HW; k += 4 * blockDim.x) {
      float4 t = total.hi > 0.0f ? __ldg(reinterpret_cast<const float4 *>(y + base + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4 *>(P + base + k) = make_float4(t.x * inv, t.y * inv, t.z * inv, t.w * inv);
    }
  }
}

}  // namespace

pg_status build_cdf(pg_ctx *ctx, const Map *m, Tables *t) {
  if (m->A == 0) return PG_OK;
  const unsigned A = m->A;
  cudaStream_t st = ctx->stream;
  switch (m->W) {
#define PG_CDF_CASE(Wc, Nc, Tc) \
  case Wc:                                                                                                          \
    k_cdf<Nc, Tc><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->sum_phi, t->sum_z, t->valid), \
        PG_COUNT(ctx);                                                                                             \
    break;
    PG_CDF_CASE(4, 4, 1)
    PG_CDF_CASE(8, 8, 1)
    PG_CDF_CASE(16, 16, 1)
    PG_CDF_CASE(32, 16, 2)
    PG_CDF_CASE(64, 16, 4)
    PG_CDF_CASE(128, 16, 8)
    PG_CDF_CASE(256, 16, 16)
#undef PG_CDF_CASE
    default: return PG_ERR_UNSUPPORTED;
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
