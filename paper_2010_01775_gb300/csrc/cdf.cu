// a8-a9: sampling map and CDFs (Eq. energy_target; Sec. 7.3, a CDF built by
// a cumulative sum over the map "like sampling an environment map").
//
// One CTA per map.  Each warp owns rows: every lane holds W/32 consecutive
// bins, forms their running sum in FP64, and one FP64 warp scan joins the
// lanes; the conditional CDF of the row is prefix / row sum (1 in the last
// bin, uniform for an empty row).  Warp 0 then scans the row sums into the
// marginal CDF, and all threads write P = y / sum y.  FP64 is used only for
// these sums and prefixes (O(bins) adds per map), never per query.
#include "pg_internal.cuh"

namespace pgi {

namespace {

__device__ __forceinline__ double warp_incl_scan_d(double x) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <int E>
__global__ void __launch_bounds__(256) k_cdf(const float *__restrict__ y, int H, int W, float *__restrict__ P,
                                             float *__restrict__ cphi, float *__restrict__ cz,
                                             uint8_t *__restrict__ valid) {
  __shared__ double mrow[256];
  __shared__ double s_total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t HW = (size_t)H * W, base = (size_t)blockIdx.x * HW;
  for (int i = warp; i < H; i += 8) {
    const float *row = y + base + (size_t)i * W;
    double pref[E], run = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      int j = lane * E + e;
      run += j < W ? (double)row[j] : 0.0;
      pref[e] = run;
    }
    double incl = warp_incl_scan_d(run);
    double off = incl - run;
    double m = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (lane == 0) mrow[i] = m;
    float *out = cphi + base + (size_t)i * W;
    if (m > 0.0) {
      double inv = 1.0 / m;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        int j = lane * E + e;
        if (j < W) out[j] = j == W - 1 ? 1.0f : (float)((off + pref[e]) * inv);
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        int j = lane * E + e;
        if (j < W) out[j] = (float)(j + 1) / (float)W;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    const int EH = (H + 31) >> 5;
    double pref[8], run = 0.0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int i = lane * EH + e;
      run += (e < EH && i < H) ? mrow[i] : 0.0;
      pref[e] = run;
    }
    double incl = warp_incl_scan_d(run);
    double off = incl - run;
    double total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    double inv = total > 0.0 ? 1.0 / total : 0.0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int i = lane * EH + e;
      if (e < EH && i < H) cz[(size_t)blockIdx.x * H + i] = i == H - 1 ? 1.0f : (float)((off + pref[e]) * inv);
    }
    if (lane == 0) {
      s_total = total;
      valid[blockIdx.x] = total > 0.0 ? 1 : 0;
    }
  }
  __syncthreads();
  const float invf = s_total > 0.0 ? (float)(1.0 / s_total) : 0.0f;
  for (size_t k = threadIdx.x; k < HW; k += blockDim.x) P[base + k] = y[base + k] * invf;
}

}  // namespace

pg_status build_cdf(pg_ctx *ctx, const Map *m, Tables *t) {
  if (m->A == 0) return PG_OK;
  const unsigned A = m->A;
  cudaStream_t st = ctx->stream;
  switch (m->W >= 32 ? m->W / 32 : 1) {
    case 1: k_cdf<1><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid); break;
    case 2: k_cdf<2><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid); break;
    case 4: k_cdf<4><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid); break;
    case 8: k_cdf<8><<<A, 256, 0, st>>>(m->y, m->H, m->W, t->P, t->cdf_phi, t->cdf_z, t->valid); break;
    default: return PG_ERR_UNSUPPORTED;
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
