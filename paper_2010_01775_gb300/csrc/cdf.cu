// a8-a9: sampling map and CDFs (Eq. energy_target; Sec. 7.3, a CDF built by
// a cumulative sum over the map "like sampling an environment map").
//
// One CTA per map.  Each warp owns rows: every lane holds W/32 consecutive
// bins (one vector load), forms their running sum, and one warp scan joins
// the lanes; the conditional CDF of the row is prefix / row sum (1 in the
// last bin, uniform for an empty row).  Warp 0 then scans the row sums into
// the marginal CDF, and all threads write P = y / sum y.
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

template <int E>
__global__ void __launch_bounds__(256) k_cdf(const float *__restrict__ y, int H, int W, float *__restrict__ P,
                                             float *__restrict__ cphi, float *__restrict__ cz,
                                             uint8_t *__restrict__ valid) {
  __shared__ float mrow_hi[256], mrow_lo[256];
  __shared__ df s_total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t HW = (size_t)H * W, base = (size_t)blockIdx.x * HW;
  for (int i = warp; i < H; i += 8) {
    const float *row = y + base + (size_t)i * W;
    float v[E];
    if (E >= 4) {
#pragma unroll
      for (int e = 0; e < E; e += 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(row + lane * E + e));
        v[e] = t.x; v[e + 1] = t.y; v[e + 2] = t.z; v[e + 3] = t.w;
      }
    } else if (E == 2) {
      float2 t = __ldg(reinterpret_cast<const float2 *>(row + lane * 2));
      v[0] = t.x;
      v[1] = t.y;
    } else {
      v[0] = lane < W ? __ldg(row + lane) : 0.0f;
    }
    df pref[E], run = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      run = df_add(run, df_from(v[e]));
      pref[e] = run;
    }
    df incl = warp_incl_scan_df(run);
    df off = {__shfl_up_sync(0xFFFFFFFFu, incl.hi, 1), __shfl_up_sync(0xFFFFFFFFu, incl.lo, 1)};
    if (lane == 0) off = {0.0f, 0.0f};
    df m = {__shfl_sync(0xFFFFFFFFu, incl.hi, 31), __shfl_sync(0xFFFFFFFFu, incl.lo, 31)};
    if (lane == 0) {
      mrow_hi[i] = m.hi;
      mrow_lo[i] = m.lo;
    }
    float out[E];
    const df rm = m.hi > 0.0f ? df_recip(m) : df{0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      int j = lane * E + e;
      if (m.hi > 0.0f) out[e] = j == W - 1 ? 1.0f : df_mul_to_f32(df_add(off, pref[e]), rm);
      else out[e] = (float)(j + 1) / (float)W;
    }
    float *o = cphi + base + (size_t)i * W + lane * E;
    if (E >= 4) {
#pragma unroll
      for (int e = 0; e < E; e += 4) *reinterpret_cast<float4 *>(o + e) = make_float4(out[e], out[e + 1], out[e + 2], out[e + 3]);
    } else if (E == 2) {
      *reinterpret_cast<float2 *>(o) = make_float2(out[0], out[1]);
    } else if (lane < W) {
      o[0] = out[0];
    }
  }
  __syncthreads();
  if (warp == 0) {
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
      if (e < EH && i < H)
        cz[(size_t)blockIdx.x * H + i] =
            i == H - 1 ? 1.0f : (total.hi > 0.0f ? df_div_to_f32(df_add(off, pref[e]), total) : 0.0f);
    }
    if (lane == 0) {
      s_total = total;
      valid[blockIdx.x] = total.hi > 0.0f ? 1 : 0;
    }
  }
  __syncthreads();
  const df total = s_total;
  if (total.hi > 0.0f) {
    const float inv = df_div_to_f32(df{1.0f, 0.0f}, total);
    for (size_t k = 4 * threadIdx.x; k < HW; k += 4 * blockDim.x) {
      float4 t = __ldg(reinterpret_cast<const float4 *>(y + base + k));
      *reinterpret_cast<float4 *>(P + base + k) = make_float4(t.x * inv, t.y * inv, t.z * inv, t.w * inv);
    }
  } else {
    for (size_t k = 4 * threadIdx.x; k < HW; k += 4 * blockDim.x)
      *reinterpret_cast<float4 *>(P + base + k) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace

pg_status build_cdf(pg_ctx *ctx, const Map *m, Tables *t) {
  if (m->A == 0) return PG_OK;
  const unsigned A = m->A;
  cudaStream_t st = ctx->stream;
  switch (m->W >= 32 ? m->W / 32 : 1) {
    case 1: k_cdf<1><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid), PG_COUNT(ctx); break;
    case 2: k_cdf<2><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid), PG_COUNT(ctx); break;
    case 4: k_cdf<4><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid), PG_COUNT(ctx); break;
    case 8: k_cdf<8><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid), PG_COUNT(ctx); break;
    default: return PG_ERR_UNSUPPORTED;
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
