// a6-a7: network input assembly and the reconstruction CNN (Sec. 5, 5.1).
//
// Every convolution is an implicit GEMM over all active leaves at once:
//   M = leaves x output pixels, N = output channels, K = taps x input channels,
// activations channel-last ([leaf][y][x][c]) so that a K-chunk of one tap is
// a contiguous run of channels.  The U-Net's skip concatenations cost
// nothing: the encoder writes its skip output straight into the channel slice
// of the decoder's input buffer, and the layer below the concatenation writes
// its output already upsampled (nearest x2) into the other slice.
//
// FP32 form: SIMT FMA tiles (BM x BN per 256-thread CTA, 8 x TN per thread).
// BF16 / FP8 forms: tcgen05 tensor-core kernels (conv_tc.cu).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "conv.cuh"

namespace pgi {

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- a6
// x[slot][k][0..7] = (S_t, S_{t-1}, log1p(C_t), log1p(C_{t-1}), C_t > 0, 0, 0, 0)
// with S = Phi * HW / sum Phi (0 for a leaf without energy).
__global__ void k_assemble(const uint64_t *__restrict__ pow_cur, const uint32_t *__restrict__ cnt_cur,
                           const uint64_t *__restrict__ pow_prev, const uint32_t *__restrict__ cnt_prev,
                           const uint64_t *__restrict__ tot_cur, const uint64_t *__restrict__ tot_prev,
                           const uint32_t *__restrict__ perm, uint32_t slot0, uint32_t nslots, int HW,
                           float *__restrict__ x) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nslots * HW) return;
  // Position slot0 + i / HW of the order `perm` (the identity when null).
  const uint32_t pos = slot0 + (uint32_t)(i / HW);
  const uint32_t s = perm ? perm[pos] : pos;
  size_t g = (size_t)s * HW + i % HW;
  uint64_t tc = tot_cur[s], tp = tot_prev[s];
  float ic = tc ? (float)HW / __ull2float_rn(tc) : 0.0f;
  float ip = tp ? (float)HW / __ull2float_rn(tp) : 0.0f;
  uint32_t c = cnt_cur[g], cp = cnt_prev[g];
  float4 a = make_float4(__ull2float_rn(pow_cur[g]) * ic, __ull2float_rn(pow_prev[g]) * ip, log1pf((float)c),
                         log1pf((float)cp));
  float4 b = make_float4(c ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
  float4 *o = reinterpret_cast<float4 *>(x + i * 8);
  o[0] = a;
  o[1] = b;
}

// k_assemble fused with the tensor-core first-layer packing for BF16: the
// same five channels, rounded to BF16, in a 32-byte row per pixel (channels
// 5..15 zero).  Bit-identical to k_assemble followed by k_pack_x0.
__global__ void k_assemble_bf16(const uint64_t *__restrict__ pow_cur, const uint32_t *__restrict__ cnt_cur,
                                const uint64_t *__restrict__ pow_prev, const uint32_t *__restrict__ cnt_prev,
                                const uint64_t *__restrict__ tot_cur, const uint64_t *__restrict__ tot_prev,
                                const uint32_t *__restrict__ perm, uint32_t slot0, uint32_t nslots, int HW,
                                uint4 *__restrict__ out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nslots * HW) return;
  const uint32_t pos = slot0 + (uint32_t)(i / HW);
  const uint32_t s = perm ? perm[pos] : pos;
  if (s == 0xFFFFFFFFu) {  // a padding position of an expert group: zero input
    out[2 * i] = out[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  size_t g = (size_t)s * HW + i % HW;
  uint64_t tc = tot_cur[s], tp = tot_prev[s];
  float ic = tc ? (float)HW / __ull2float_rn(tc) : 0.0f;
  float ip = tp ? (float)HW / __ull2float_rn(tp) : 0.0f;
  uint32_t c = cnt_cur[g], cp = cnt_prev[g];
  __nv_bfloat162 q0 = __floats2bfloat162_rn(__ull2float_rn(pow_cur[g]) * ic, __ull2float_rn(pow_prev[g]) * ip);
  __nv_bfloat162 q1 = __floats2bfloat162_rn(log1pf((float)c), log1pf((float)cp));
  __nv_bfloat162 q2 = __floats2bfloat162_rn(c ? 1.0f : 0.0f, 0.0f);
  out[2 * i] = make_uint4(*reinterpret_cast<uint32_t *>(&q0), *reinterpret_cast<uint32_t *>(&q1),
                          *reinterpret_cast<uint32_t *>(&q2), 0u);
  out[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ float activate(float v, int act) {
  if (act == 1) return v > 0.0f ? v : expm1f(v);
  if (act == 2) return fmaxf(v, 0.0f) + log1pf(expf(-fabsf(v)));
  return v;
}

// ---------------------------------------------------------------- a7, FP32 SIMT
// CTA tile BM x BN, K chunk 16.  Thread (tx, ty): rows tx*4+{0..3} and
// BM/2+tx*4+{0..3}, columns ty*TN..ty*TN+TN-1.  A is gathered channel-last
// with 16-byte loads (4 channels of one tap), staged k-major in shared memory.
template <int BM, int BN, int TN>
__global__ void __launch_bounds__(256) k_conv_f32(ConvArgs a) {
  constexpr int BK = 16;
  constexpr int TX = BM / 8;  // threads along M
  static_assert(TX * (BN / TN) == 256, "256 threads");
  constexpr int A_VEC = BM * BK / 4 / 256;  // float4 loads of A per thread
  constexpr int B_VEC = (BN * BK / 4 + 255) / 256;
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const long m0 = (long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int K = a.k * a.k * a.Cin;
  const int HWo = a.Hout * a.Wout;

  // Per-thread A rows: fixed across the K loop.
  int a_kq = tid & 3;  // which 4-channel quad of the 16-chunk
  int a_base[A_VEC], a_iy[A_VEC], a_ix[A_VEC];
#pragma unroll
  for (int v = 0; v < A_VEC; ++v) {
    int m = (tid >> 2) + v * 64;
    long mg = m0 + m;
    if (mg < a.M) {
      int leaf = (int)(mg / HWo), r = (int)(mg % HWo);
      int oy = r / a.Wout, ox = r % a.Wout;
      a_iy[v] = oy * a.stride - a.pad;
      a_ix[v] = ox * a.stride - a.pad;  // pad = dil * (k / 2)
      a_base[v] = leaf * a.Hin;
    } else {
      a_iy[v] = -100000;
      a_ix[v] = -100000;
      a_base[v] = 0;
    }
  }

  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

  float4 ra[A_VEC], rb[B_VEC];
  auto load = [&](int k0) {
    int kk = k0 + a_kq * 4;
    int tap = kk / a.Cin, c = kk - tap * a.Cin;
    const int dl = a.dil > 1 ? a.dil : 1;
    int ky = (tap / a.k) * dl, kx = (tap - (tap / a.k) * a.k) * dl;
#pragma unroll
    for (int v = 0; v < A_VEC; ++v) {
      int iy = a_iy[v] + ky, ix = a_ix[v] + kx;
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (kk < K && iy >= 0 && iy < a.Hin && ix >= 0 && ix < a.Win) {
        const float *p = ((const float *)a.in) + ((size_t)(a_base[v] + iy) * a.Win + ix) * a.in_cs + a.in_co + c;
        val = __ldg(reinterpret_cast<const float4 *>(p));
      }
      ra[v] = val;
    }
#pragma unroll
    for (int v = 0; v < B_VEC; ++v) {
      int idx = tid + v * 256;  // float4 index within BK x BN
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < BN * BK / 4) {
        int r = idx / (BN / 4), cq = idx % (BN / 4);
        int kr = k0 + r, n = n0 + cq * 4;
        if (kr < K && n < a.Cout) val = __ldg(reinterpret_cast<const float4 *>(a.w + (size_t)kr * a.Cout + n));
      }
      rb[v] = val;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int v = 0; v < A_VEC; ++v) {
      int m = (tid >> 2) + v * 64;
      As[a_kq * 4 + 0][m] = ra[v].x;
      As[a_kq * 4 + 1][m] = ra[v].y;
      As[a_kq * 4 + 2][m] = ra[v].z;
      As[a_kq * 4 + 3][m] = ra[v].w;
    }
#pragma unroll
    for (int v = 0; v < B_VEC; ++v) {
      int idx = tid + v * 256;
      if (idx < BN * BK / 4) {
        int r = idx / (BN / 4), cq = idx % (BN / 4);
        *reinterpret_cast<float4 *>(&Bs[r][cq * 4]) = rb[v];
      }
    }
  };

  load(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + BK < K) load(k0 + BK);
    // Blocked accumulation: each 16-term chunk is summed on its own and then
    // added to the running total, which keeps FP32 rounding growth at about
    // (K/16 + 16) ulps instead of K ulps over long reductions.
    float part[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) part[i][j] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][tx * 4]);
      float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][BM / 2 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[TN];
      if constexpr (TN % 4 == 0) {
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
          float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][ty * TN + j]);
          bv[j] = b4.x; bv[j + 1] = b4.y; bv[j + 2] = b4.z; bv[j + 3] = b4.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][ty * TN + j];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] += part[i][j];
  }

  // Epilogue: bias + activation, channel-last store (optionally upsampled x2).
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int m = (i < 4) ? tx * 4 + i : BM / 2 + tx * 4 + (i - 4);
    long mg = m0 + m;
    if (mg >= a.M) continue;
    int leaf = (int)(mg / HWo), r = (int)(mg % HWo);
    int oy = r / a.Wout, ox = r % a.Wout;
    float o[TN];
    const float ps = a.scale ? __ldg(a.scale + mg) : 1.0f;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + ty * TN + j;
      const float bn = n < a.Cout ? __ldg(a.bias + n) : 0.0f;
      const float v = a.scale ? (ps > 0.0f ? acc[i][j] * ps + bn : 0.0f) : acc[i][j] + bn;
      o[j] = n < a.Cout ? activate(v, a.act) : 0.0f;
    }
    int nb = n0 + ty * TN;
    if (nb >= a.Cout) continue;
    if (a.res) {
      const float *rp = ((const float *)a.res) + (size_t)mg * a.res_cs + a.res_co + nb;
#pragma unroll
      for (int j = 0; j < TN; ++j)
        if (nb + j < a.Cout) o[j] += __ldg(rp + j);
    }
    int reps = a.ups ? 2 : 1;
    int Ho = a.Hout * reps, Wo = a.Wout * reps;
    for (int dy = 0; dy < reps; ++dy)
      for (int dx = 0; dx < reps; ++dx) {
        float *p = ((float *)a.out) + ((size_t)(leaf * Ho + oy * reps + dy) * Wo + ox * reps + dx) * a.out_cs + a.out_co + nb;
        if constexpr (TN % 4 == 0) {
#pragma unroll
          for (int j = 0; j < TN; j += 4)
            if (nb + j < a.Cout) *reinterpret_cast<float4 *>(p + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < TN; ++j)
            if (nb + j < a.Cout) p[j] = o[j];
        }
      }
  }
}

// Single-output-channel conv (3x3 or 1x1) + activation into the map y.
__global__ void k_conv_cout1(ConvArgs a) {
  long mg = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (mg >= a.M) return;
  int HWo = a.Hout * a.Wout;
  int leaf = (int)(mg / HWo), r = (int)(mg % HWo);
  int oy = r / a.Wout, ox = r % a.Wout;
  float acc = 0.0f;
  for (int ky = 0; ky < a.k; ++ky) {
    int iy = oy * a.stride + ky - a.pad;
    if (iy < 0 || iy >= a.Hin) continue;
    for (int kx = 0; kx < a.k; ++kx) {
      int ix = ox * a.stride + kx - a.pad;
      if (ix < 0 || ix >= a.Win) continue;
      const float *p = ((const float *)a.in) + ((size_t)(leaf * a.Hin + iy) * a.Win + ix) * a.in_cs + a.in_co;
      const float *w = a.w + (size_t)(ky * a.k + kx) * a.Cin;  // [K][1]
      for (int c = 0; c < a.Cin; c += 4) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p + c));
        acc = fmaf(v.x, __ldg(w + c), acc);
        acc = fmaf(v.y, __ldg(w + c + 1), acc);
        acc = fmaf(v.z, __ldg(w + c + 2), acc);
        acc = fmaf(v.w, __ldg(w + c + 3), acc);
      }
    }
  }
  ((float *)a.out)[(size_t)mg * a.out_cs + a.out_co] = activate(acc + __ldg(a.bias), a.act);
}

template <int BM, int BN, int TN>
void launch_f32(pg_ctx *ctx, const ConvArgs &a, cudaStream_t st) {
  dim3 grid((unsigned)((a.M + BM - 1) / BM), (unsigned)((a.Cout + BN - 1) / BN));
  k_conv_f32<BM, BN, TN><<<grid, 256, 0, st>>>(a), PG_COUNT(ctx);
}

}  // namespace

pg_status conv_f32(pg_ctx *ctx, const ConvArgs &a, cudaStream_t st) {
  if (a.M == 0) return PG_OK;
  // Channel counts must be multiples of 4 (16-byte vector access).
  if (a.Cin % 4 || a.in_cs % 4 || a.in_co % 4 || (a.Cout != 1 && (a.Cout % 4 || a.out_cs % 4 || a.out_co % 4)))
    return PG_ERR_UNSUPPORTED;
  if (a.Cout == 1) {
    k_conv_cout1<<<ceil_div(a.M, 256), 256, 0, st>>>(a), PG_COUNT(ctx);
  } else if (a.Cout >= 128) {
    launch_f32<128, 128, 8>(ctx, a, st);
  } else if (a.Cout > 32) {
    launch_f32<256, 64, 8>(ctx, a, st);
  } else if (a.Cout > 16) {
    launch_f32<256, 32, 4>(ctx, a, st);
  } else if (a.Cout > 8) {
    launch_f32<256, 16, 2>(ctx, a, st);
  } else {
    launch_f32<256, 8, 1>(ctx, a, st);
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status net_prepare(pg_ctx *ctx, Net *net, pg_precision prec) {
  if (prec != PG_FP32) return tc_prepare(ctx, net, prec);
  return PG_OK;
}

static size_t act_floats_per_leaf(const Net *net, int H, int W) {
  size_t HW = (size_t)H * W;
  if (net->arch == 0) return HW * (8 + 2 * (size_t)net->widths[0]);
  if (net->arch == 2) {
    const size_t c0 = net->widths[0], c1 = net->widths[1];
    return HW * (c0 + (c1 + c0) + 2 * c0) + HW / 4 * (c1 + 2 * c1 + 2 * c1) + HW / 16 * 2 * c1 +
           paper_mask_floats_per_leaf(H, W);
  }
  size_t c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2], c3 = net->widths[3];
  return HW * (8 + (c1 + c0) + 2 * c0) + HW / 4 * ((c2 + c1) + c1) + HW / 16 * ((c3 + c2) + c2) + HW / 64 * c3;
}

// ---------------------------------------------------------------- paper-style net (arch 2)
// Partial-convolution masks (Liu et al. 2018, the masked convolutions of
// Sec. 5.1): for each output pixel the number c of valid input pixels under
// its 3x3 window (taps dil apart, stride, zero outside the map); scale =
// 9 / c where c > 0, else 0; the output mask is c > 0.
__global__ void k_pconv_mask(const float *__restrict__ m_in, int in_cs, int Hin, int Win, int stride, int dil,
                             long M, int Hout, int Wout, float *__restrict__ scale, float *__restrict__ m_out) {
  const long mg = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (mg >= M) return;
  const int HWo = Hout * Wout;
  const int leaf = (int)(mg / HWo), r = (int)(mg % HWo), oy = r / Wout, ox = r % Wout;
  int c = 0;
  for (int ky = -1; ky <= 1; ++ky)
    for (int kx = -1; kx <= 1; ++kx) {
      const int iy = oy * stride + ky * dil, ix = ox * stride + kx * dil;
      if (iy >= 0 && iy < Hin && ix >= 0 && ix < Win)
        c += m_in[((size_t)(leaf * Hin + iy) * Win + ix) * in_cs] > 0.0f ? 1 : 0;
    }
  scale[mg] = c ? 9.0f / (float)c : 0.0f;
  if (m_out) m_out[mg] = c ? 1.0f : 0.0f;
}

// Mask of a decoder concatenation: the union of the upsampled (nearest x2)
// deeper mask and the skip's mask.
__global__ void k_mask_union_up(const float *__restrict__ deep, const float *__restrict__ skip, long M, int H, int W,
                                float *__restrict__ out) {
  const long mg = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (mg >= M) return;
  const int HW = H * W, leaf = (int)(mg / HW), r = (int)(mg % HW), y = r / W, x = r % W;
  const float d = deep[((size_t)leaf * (H / 2) + y / 2) * (W / 2) + x / 2];
  out[mg] = fmaxf(d, skip[mg]);
}

size_t paper_mask_floats_per_leaf(int H, int W) {
  const size_t HW = (size_t)H * W;
  // 11 scales and 11 masks: 4 + 4 at full resolution, 4 + 4 at half, 3 + 3 at quarter; 2 unions.
  return 8 * HW + 8 * HW / 4 + 6 * HW / 16 + HW + HW / 4;
}

pg_status paper_masks(pg_ctx *ctx, const float *x0, uint32_t ns, int H, int W, float *buf, PaperMasks *pm,
                      cudaStream_t st) {
  const long M0 = (long)ns * H * W, M1 = M0 / 4, M2 = M0 / 16;
  float *q = buf;
  auto take = [&](long n) { float *p = q; q += n; return p; };
  float *s[12] = {}, *m[12] = {};
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
  auto mask = [&](int l, const float *in, int in_cs, int Hin, int Win, int stride, int dil, long M, int Ho, int Wo) {
    s[l] = take(M);
    m[l] = take(M);
    k_pconv_mask<<<ceil_div(M, 256), 256, 0, st>>>(in, in_cs, Hin, Win, stride, dil, M, Ho, Wo, s[l], m[l]),
        PG_COUNT(ctx);
  };
  mask(0, x0 + 4, 8, H, W, 1, 1, M0, H, W);        // input mask: the B channel
  mask(1, m[0], 1, H, W, 1, 1, M0, H, W);          // e0
  mask(2, m[1], 1, H, W, 2, 1, M1, H1, W1);
  mask(3, m[2], 1, H1, W1, 1, 1, M1, H1, W1);      // e1
  mask(4, m[3], 1, H1, W1, 2, 1, M2, H2, W2);
  mask(5, m[4], 1, H2, W2, 1, 2, M2, H2, W2);
  mask(6, m[5], 1, H2, W2, 1, 4, M2, H2, W2);
  float *u7 = take(M1);
  k_mask_union_up<<<ceil_div(M1, 256), 256, 0, st>>>(m[6], m[3], M1, H1, W1, u7), PG_COUNT(ctx);
  mask(7, u7, 1, H1, W1, 1, 1, M1, H1, W1);
  mask(8, m[7], 1, H1, W1, 1, 1, M1, H1, W1);
  float *u9 = take(M0);
  k_mask_union_up<<<ceil_div(M0, 256), 256, 0, st>>>(m[8], m[1], M0, H, W, u9), PG_COUNT(ctx);
  mask(9, u9, 1, H, W, 1, 1, M0, H, W);
  mask(10, m[9], 1, H, W, 1, 1, M0, H, W);
  PG_CUDA(cudaGetLastError());
  for (int l = 0; l < 12; ++l) pm->scale[l] = s[l];
  return PG_OK;
}

// Per-leaf photon count: the sum of the leaf's current count plane.
__global__ void k_leaf_counts(const uint32_t *__restrict__ cnt, int HW, uint32_t *__restrict__ out) {
  __shared__ uint32_t part[8];
  const uint32_t *row = cnt + (size_t)blockIdx.x * HW;
  uint32_t v = 0;
  for (int k = threadIdx.x; k < HW; k += blockDim.x) v += row[k];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += part[w];
    out[blockIdx.x] = t;
  }
}

// y[perm[k]] = yp[k] for rows of HW floats.
__global__ void k_scatter_rows(const float *__restrict__ yp, const uint32_t *__restrict__ perm, uint32_t A, int HW,
                               float *__restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)A * HW / 4) return;
  const size_t k = (4 * i) / HW, c = (4 * i) % HW;
  const uint32_t s = perm[k];
  if (s == 0xFFFFFFFFu) return;  // padding position
  *reinterpret_cast<float4 *>(y + (size_t)s * HW + c) = *reinterpret_cast<const float4 *>(yp + 4 * i);
}

// Leaves grouped by expert on the device (one CTA): the expert of slot k is
// the number of count bounds <= counts[k]; expert e's positions are
// [range[e], range[e+1]), its leaf count rounded up to a multiple of pad;
// pos_slot[p] is the slot at position p (an expert's slots in slot order)
// or ~0 at a padding position.
struct ExpertBounds {
  uint32_t b[16];
};

__global__ void __launch_bounds__(1024) k_group_experts(const uint32_t *__restrict__ counts, uint32_t A,
                                                        ExpertBounds eb, int E, uint32_t pad, uint32_t npos,
                                                        int *__restrict__ range, uint32_t *__restrict__ pos_slot) {
  __shared__ uint32_t n[16], base[16], wcnt[32], wofs[32];
  __shared__ int srange[17];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto expert = [&](uint32_t c) {
    int e = 0;
    while (e + 1 < E && c >= eb.b[e]) ++e;
    return e;
  };
  if (tid < 16) n[tid] = base[tid] = 0u;
  __syncthreads();
  for (uint32_t k = tid; k < A; k += blockDim.x) atomicAdd(&n[expert(counts[k])], 1u);
  for (uint32_t p = tid; p < npos; p += blockDim.x) pos_slot[p] = 0xFFFFFFFFu;
  __syncthreads();
  if (tid == 0) {
    int r = 0;
    for (int e = 0; e < E; ++e) {
      srange[e] = r;
      range[e] = r;
      r += (int)(((n[e] + pad - 1) / pad) * pad);
    }
    srange[E] = r;
    range[E] = r;
  }
  __syncthreads();
  for (uint32_t c0 = 0; c0 < A; c0 += blockDim.x) {
    const uint32_t k = c0 + tid;
    const int ek = k < A ? expert(counts[k]) : -1;
    for (int e = 0; e < E; ++e) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, ek == e);
      if (lane == 0) wcnt[warp] = __popc(m);
      __syncthreads();
      if (warp == 0) {
        const uint32_t v = wcnt[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (lane >= o) x += y;
        }
        wofs[lane] = x - v;
      }
      __syncthreads();
      if (ek == e) pos_slot[srange[e] + base[e] + wofs[warp] + __popc(m & ((1u << lane) - 1u))] = k;
      __syncthreads();
      if (tid == 0) base[e] += wofs[31] + wcnt[31];
      __syncthreads();
    }
  }
}

pg_status leaf_counts(pg_ctx *ctx, const Hist *h, uint32_t *d_counts) {
  if (h->A == 0) return PG_OK;
  k_leaf_counts<<<h->A, 256, 0, ctx->stream>>>(h->cnt_cur, h->H * h->W, d_counts), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status scatter_rows(pg_ctx *ctx, const float *yp, const uint32_t *d_perm, uint32_t A, int HW, float *y) {
  if (A == 0) return PG_OK;
  const size_t n4 = (size_t)A * HW / 4;
  k_scatter_rows<<<ceil_div(n4, 256), 256, 0, ctx->stream>>>(yp, d_perm, A, HW, y), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status reconstruct_experts_grouped(pg_ctx *ctx, const Hist *h, const Net *const *nets, int E,
                                     const uint32_t *count_bounds, float *y) {
  const uint32_t A = h->A;
  if (A == 0) return PG_OK;
  if (E < 2 || E > 16 || E > tc_max_experts()) return PG_ERR_UNSUPPORTED;
  for (int e = 0; e < E; ++e)
    if (nets[e]->arch != 1 || nets[e]->n_layers != nets[0]->n_layers) return PG_ERR_UNSUPPORTED;
  const int H = h->H, W = h->W, HW = H * W;
  // No tile may span two experts: the coarsest level's maps hold HW / 64
  // pixels, and a tile at most 256.
  const uint32_t pad = (uint32_t)std::max(1, (256 * 64) / HW);
  const uint32_t npos = A + (uint32_t)E * (pad - 1);
  ExpertBounds eb;
  memset(&eb, 0, sizeof(eb));
  for (int e = 0; e + 1 < E; ++e) eb.b[e] = count_bounds[e];
  const size_t b_cnt = align256(4ull * A), b_rng = align256(4ull * (E + 1)), b_pos = align256(4ull * npos);
  const size_t b_y = align256((size_t)npos * HW * 4);
  const size_t gbytes = b_cnt + b_rng + b_pos + b_y;
  void *gblock;
  PG_TRY(ctx_alloc(ctx, gbytes, &gblock));
  struct Guard {
    pg_ctx *c; void *p; size_t b;
    ~Guard() { ctx_free(c, p, b); }
  } gguard{ctx, gblock, gbytes};
  uint8_t *q = (uint8_t *)gblock;
  uint32_t *d_cnt = (uint32_t *)q; q += b_cnt;
  int *d_range = (int *)q; q += b_rng;
  uint32_t *d_pos = (uint32_t *)q; q += b_pos;
  float *yp = (float *)q;
  cudaStream_t st = ctx->stream;
  PG_TRY(leaf_counts(ctx, h, d_cnt));
  k_group_experts<<<1, 1024, 0, st>>>(d_cnt, A, eb, E, pad, npos, d_range, d_pos), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  const size_t per_leaf = tc_bytes_per_leaf(nets[0], PG_BF16, H, W);
  uint32_t chunk = 0;
  size_t bytes = 0;
  void *scratch = nullptr;
  pg_status as = PG_ERR_OOM;
  for (size_t limit : {16ull << 30, 6ull << 30, 2ull << 30, 512ull << 20}) {
    chunk = (uint32_t)std::min<size_t>(npos, std::max<size_t>(pad, (limit / per_leaf) / pad * pad));
    bytes = per_leaf * chunk + 4096;
    as = ctx_alloc(ctx, bytes, &scratch);
    if (as != PG_ERR_OOM || chunk == pad) break;
  }
  PG_TRY(as);
  struct Guard2 {
    pg_ctx *c; void *p; size_t b;
    ~Guard2() { ctx_free(c, p, b); }
  } guard{ctx, scratch, bytes};
  for (uint32_t p0 = 0; p0 < npos; p0 += chunk) {
    const uint32_t ns = std::min(chunk, npos - p0);
    const size_t nx = (size_t)ns * HW;
    k_assemble_bf16<<<ceil_div(nx, 256), 256, 0, st>>>(h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev, h->tot_cur,
                                                       h->tot_prev, d_pos, p0, ns, HW, (uint4 *)scratch), PG_COUNT(ctx);
    PG_CUDA(cudaGetLastError());
    PG_TRY(forward_tc_experts(ctx, nets, E, d_range, (int)p0, scratch, ns, H, W, yp + (size_t)p0 * HW, st));
  }
  return scatter_rows(ctx, yp, d_pos, npos, HW, y);
}

pg_status reconstruct(pg_ctx *ctx, const Hist *h, const Net *net, pg_precision prec, Map *m, bool tune) {
  return reconstruct_range(ctx, h, net, prec, m->y, nullptr, 0, h->A, tune);
}

pg_status reconstruct_range(pg_ctx *ctx, const Hist *h, const Net *net, pg_precision prec, float *y_out,
                            const uint32_t *d_perm, uint32_t first, uint32_t count, bool tune) {
  const uint32_t A = count;
  if (A == 0) return PG_OK;
  const int H = h->H, W = h->W, HW = H * W;
  // BF16 assembles straight into the packed first-layer input (no FP32 x0).
  const bool packed = prec == PG_BF16 && net->arch != 2;  // the paper-style net reads its mask from x0
  const size_t x0_per_leaf = packed ? 0 : 8 * (size_t)HW * 4;
  const size_t per_leaf = x0_per_leaf + (prec == PG_FP32 ? act_floats_per_leaf(net, H, W) * 4
                                                         : tc_bytes_per_leaf(net, prec, H, W));
  // Activation working set: leaves are processed in chunks.  The
  // tensor-core forms take up to 16 GB at once (fewer, larger launches;
  // their indexing is 64-bit throughout), falling back to smaller chunks
  // when the budget or the device refuses; the FP32 and paper-style paths
  // keep 6 GB chunks (their element offsets stay below 2^31).
  const bool big = prec != PG_FP32 && net->arch != 2;
  uint32_t chunk = 0;
  size_t bytes = 0;
  void *scratch = nullptr;
  pg_status as = PG_ERR_OOM;
  for (size_t limit : {big ? (16ull << 30) : (6ull << 30), 6ull << 30, 2ull << 30, 512ull << 20}) {
    chunk = (uint32_t)std::max<size_t>(1, std::min<size_t>(A, limit / per_leaf));
    bytes = per_leaf * chunk + 4096;
    as = ctx_alloc(ctx, bytes, &scratch);
    if (as != PG_ERR_OOM || chunk == 1) break;
  }
  PG_TRY(as);
  struct Guard {
    pg_ctx *c; void *p; size_t b;
    ~Guard() { ctx_free(c, p, b); }
  } guard{ctx, scratch, bytes};
  cudaStream_t st = ctx->stream;
  for (uint32_t s0 = 0; s0 < A; s0 += chunk) {
    uint32_t ns = std::min(chunk, A - s0);
    size_t nx = (size_t)ns * HW;
    float *y = y_out + (size_t)s0 * HW;
    if (packed) {
      // The packed input is the first region of the activation buffer.
      k_assemble_bf16<<<ceil_div(nx, 256), 256, 0, st>>>(h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev,
                                                         h->tot_cur, h->tot_prev, d_perm, first + s0, ns, HW,
                                                         (uint4 *)scratch), PG_COUNT(ctx);
      PG_CUDA(cudaGetLastError());
      PG_TRY(forward_tc(ctx, net, prec, nullptr, scratch, ns, H, W, y, st, tune));
      if (tune) break;
      continue;
    }
    float *x0 = (float *)scratch;  // FP32 input, 8 channels
    k_assemble<<<ceil_div(nx, 256), 256, 0, st>>>(h->pow_cur, h->cnt_cur, h->pow_prev, h->cnt_prev, h->tot_cur,
                                                  h->tot_prev, d_perm, first + s0, ns, HW, x0), PG_COUNT(ctx);
    PG_CUDA(cudaGetLastError());
    uint8_t *act = (uint8_t *)scratch + align256(nx * 8 * 4);
    if (prec == PG_FP32) PG_TRY(forward_f32(ctx, net, x0, act, ns, H, W, y, st));
    else PG_TRY(forward_tc(ctx, net, prec, x0, act, ns, H, W, y, st, tune));
    if (tune) break;  // the first chunk is representative of every later one
  }
  return PG_OK;
}

// Plain FP32 forward of one chunk: activations carved from `act`.
pg_status forward_f32(pg_ctx *ctx, const Net *net, const float *x0, void *actv, uint32_t ns, int H, int W, float *y,
                      cudaStream_t st) {
  float *act = (float *)actv;
  const Layer *Ls = net->layers;
  auto conv = [&](const Layer &L, const float *in, int in_cs, int in_co, int Hin, int Win, float *out, int out_cs,
                  int out_co, int ups, const float *scale = nullptr, const float *res = nullptr, int res_cs = 0,
                  int res_co = 0) -> pg_status {
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.in = in; a.in_cs = in_cs; a.in_co = in_co; a.Hin = Hin; a.Win = Win; a.Cin = L.cin;
    a.out = out; a.out_cs = out_cs; a.out_co = out_co;
    a.Hout = Hin / L.stride; a.Wout = Win / L.stride; a.Cout = L.cout;
    a.dil = L.dil > 1 ? L.dil : 1;
    a.k = L.k; a.stride = L.stride; a.pad = a.dil * (L.k / 2);
    a.w = L.w; a.bias = L.b; a.act = L.act; a.ups = ups;
    a.scale = scale;
    a.res = res; a.res_cs = res_cs; a.res_co = res_co;
    a.M = (long)ns * a.Hout * a.Wout;
    return conv_f32(ctx, a, st);
  };
  const size_t HW = (size_t)H * W;
  if (net->arch == 2) {
    const int c0 = net->widths[0], c1 = net->widths[1];
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    const int k0c = c1 + c0, k1c = 2 * c1;
    float *a0 = act;                               // [ns][H][W][c0]
    float *cat0 = a0 + ns * HW * c0;               // [ns][H][W][c1+c0]   up(d1b) | e0
    float *d0 = cat0 + ns * HW * k0c;              // [ns][H][W][c0]
    float *d0b = d0 + ns * HW * c0;                // [ns][H][W][c0]
    float *a1 = d0b + ns * HW * c0;                // [ns][H1][W1][c1]
    float *cat1 = a1 + ns * HW / 4 * c1;           // [ns][H1][W1][2c1]   up(b2) | e1
    float *d1 = cat1 + ns * HW / 4 * k1c;          // [ns][H1][W1][c1]
    float *b0 = d1 + ns * HW / 4 * c1;             // [ns][H2][W2][c1]
    float *b1 = b0 + ns * HW / 16 * c1;            // [ns][H2][W2][c1]
    float *mbuf = b1 + ns * HW / 16 * c1;
    PaperMasks pm;
    PG_TRY(paper_masks(ctx, x0, ns, H, W, mbuf, &pm, st));
    // Encoder (residual links within a level), dilated bottleneck, decoder.
    PG_TRY(conv(Ls[0], x0, 8, 0, H, W, a0, c0, 0, 0, pm.scale[0]));
    PG_TRY(conv(Ls[1], a0, c0, 0, H, W, cat0, k0c, c1, 0, pm.scale[1], a0, c0, 0));            // e0
    PG_TRY(conv(Ls[2], cat0, k0c, c1, H, W, a1, c1, 0, 0, pm.scale[2]));
    PG_TRY(conv(Ls[3], a1, c1, 0, H1, W1, cat1, k1c, c1, 0, pm.scale[3], a1, c1, 0));          // e1
    PG_TRY(conv(Ls[4], cat1, k1c, c1, H1, W1, b0, c1, 0, 0, pm.scale[4]));
    PG_TRY(conv(Ls[5], b0, c1, 0, H2, W2, b1, c1, 0, 0, pm.scale[5], b0, c1, 0));              // dilation 2
    PG_TRY(conv(Ls[6], b1, c1, 0, H2, W2, cat1, k1c, 0, 1, pm.scale[6], b1, c1, 0));           // dilation 4, up
    PG_TRY(conv(Ls[7], cat1, k1c, 0, H1, W1, d1, c1, 0, 0, pm.scale[7]));
    PG_TRY(conv(Ls[8], d1, c1, 0, H1, W1, cat0, k0c, 0, 1, pm.scale[8], d1, c1, 0));           // up
    PG_TRY(conv(Ls[9], cat0, k0c, 0, H, W, d0, c0, 0, 0, pm.scale[9]));
    PG_TRY(conv(Ls[10], d0, c0, 0, H, W, d0b, c0, 0, 0, pm.scale[10], d0, c0, 0));
    PG_TRY(conv(Ls[11], d0b, c0, 0, H, W, y, 1, 0, 0));                                          // 1x1 head
    return PG_OK;
  }
  if (net->arch == 0) {
    int c = net->widths[0];
    float *t0 = act, *t1 = act + ns * HW * c;
    PG_TRY(conv(Ls[0], x0, 8, 0, H, W, t0, c, 0, 0));
    PG_TRY(conv(Ls[1], t0, c, 0, H, W, t1, c, 0, 0));
    PG_TRY(conv(Ls[2], t1, c, 0, H, W, y, 1, 0, 0));
    return PG_OK;
  }
  const int c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2], c3 = net->widths[3];
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  float *cat0 = act;                               // [ns][H][W][c1+c0]   up(d1) | e0
  float *t0 = cat0 + ns * HW * (c1 + c0);          // [ns][H][W][c0]
  float *t0b = t0 + ns * HW * c0;                  // [ns][H][W][c0]
  float *cat1 = t0b + ns * HW * c0;                // [ns][H1][W1][c2+c1] up(d2) | e1
  float *t1 = cat1 + ns * HW / 4 * (c2 + c1);      // [ns][H1][W1][c1]
  float *cat2 = t1 + ns * HW / 4 * c1;             // [ns][H2][W2][c3+c2] up(e3) | e2
  float *t2 = cat2 + ns * HW / 16 * (c3 + c2);     // [ns][H2][W2][c2]
  float *t3 = t2 + ns * HW / 16 * c2;              // [ns][H3][W3][c3]
  const int k0c = c1 + c0, k1c = c2 + c1, k2c = c3 + c2;
  // Encoder.
  PG_TRY(conv(Ls[0], x0, 8, 0, H, W, t0, c0, 0, 0));
  PG_TRY(conv(Ls[1], t0, c0, 0, H, W, cat0, k0c, c1, 0));          // e0
  PG_TRY(conv(Ls[2], cat0, k0c, c1, H, W, t1, c1, 0, 0));          // stride 2
  PG_TRY(conv(Ls[3], t1, c1, 0, H1, W1, cat1, k1c, c2, 0));        // e1
  PG_TRY(conv(Ls[4], cat1, k1c, c2, H1, W1, t2, c2, 0, 0));        // stride 2
  PG_TRY(conv(Ls[5], t2, c2, 0, H2, W2, cat2, k2c, c3, 0));        // e2
  PG_TRY(conv(Ls[6], cat2, k2c, c3, H2, W2, t3, c3, 0, 0));        // stride 2
  PG_TRY(conv(Ls[7], t3, c3, 0, H3, W3, cat2, k2c, 0, 1));         // up(e3)
  // Decoder.
  PG_TRY(conv(Ls[8], cat2, k2c, 0, H2, W2, t2, c2, 0, 0));
  PG_TRY(conv(Ls[9], t2, c2, 0, H2, W2, cat1, k1c, 0, 1));         // up(d2)
  PG_TRY(conv(Ls[10], cat1, k1c, 0, H1, W1, t1, c1, 0, 0));
  PG_TRY(conv(Ls[11], t1, c1, 0, H1, W1, cat0, k0c, 0, 1));        // up(d1)
  PG_TRY(conv(Ls[12], cat0, k0c, 0, H, W, t0, c0, 0, 0));
  PG_TRY(conv(Ls[13], t0, c0, 0, H, W, t0b, c0, 0, 0));
  PG_TRY(conv(Ls[14], t0b, c0, 0, H, W, y, 1, 0, 0));              // 1x1 head + softplus
  return PG_OK;
}

}  // namespace pgi
