// a7 on tensor cores: BF16 (and FP8 E4M3) implicit-GEMM convolutions with
// tcgen05 (5th-generation tensor cores, accumulators in TMEM), fed by TMA.
//
// GEMM view of one layer: M = leaves x output pixels (tiles of 128 pixels =
// whole output rows of one or more leaves), N = output channels (the whole
// layer, 16..256), K = taps x input channels.  One pipeline stage holds one
// (tap, channel chunk): a 4-D TMA box {chunk, Wt, Ht, Lt} of the channel-last
// activation tensor at the tap-shifted origin (out-of-range coordinates are
// zero-filled by TMA, which implements the "same" zero padding; strided
// layers use TMA element strides), and a 2-D TMA box of the K-major weights.
// Both land in shared memory in the canonical K-major swizzled layout that
// the MMA descriptors describe.
//
// Persistent, warp-specialised CTA (192 threads):
//   warp 0   one thread issues TMA loads into a ring of stages
//   warp 1   one thread issues tcgen05.mma (M=128, N=Cout) and commits each
//            stage back to the producer; owns TMEM allocation
//   warps 2-5 epilogue: tcgen05.ld the accumulator (one pixel row per thread),
//            bias + ELU, convert, store channel-last (optionally upsampled x2)
// The accumulator is double-buffered in TMEM so the epilogue of one tile
// overlaps the main loop of the next.
//
// Operand staging modes for the A (activation) tile of a 3x3 stride-1 layer:
//   0  one box per (tap, channel chunk) at the tap-shifted origin;
//   1  per channel chunk, three x-shifted boxes of the tile plus a one-row
//      halo; tap (ky, kx) is rows ky*Wt.. of copy kx;
//   2  per channel chunk, ONE box of whole zero-padded rows (P = W + 2
//      pixels: x = -1 .. W) covering the tile and its halo.  Output pixels are
//      indexed in the same padded row space (q = y * P + x), so tap (ky, kx)
//      of output q is input row q + ky * P + kx of the box: every tap is the
//      same box read from another starting row.  The two pad columns of each
//      output row are computed and discarded (2 / (W + 2) extra MMA rows);
//      the TMA moves each input pixel about once instead of 3 or 9 times.  Every mbarrier wait is bounded (2 s):
// on expiry the CTA raises PG_ERR_TIMEOUT in the context status word, drains
// what it issued and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "conv.cuh"

namespace pgi {

namespace {

constexpr int kThreads = 320;  // producer warp, MMA warp, 8 epilogue warps
constexpr int kMaxExperts = 8;  // networks of one grouped launch (mixture of experts)

// The B (weight) tensor maps of a launch: one per expert network of a
// grouped launch, [0] only otherwise.
struct TcMapsB {
  CUtensorMap b[kMaxExperts];
};
constexpr int kEpiWarps = 8;
constexpr int kBM = 128;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

struct TcArgs {
  int k, stride, pad;
  int Cin, chunk, cchunks;
  int Hout, Wout, HWo;
  long M;
  int BN;
  int mt;           // 128-pixel M-subtiles per CTA tile (each its own accumulator)
  int halo;         // 3x3 stride-1 layers: one stage = one channel chunk, all 9 taps
  uint32_t bytes_ver;  // halo mode: bytes of one x-shifted input box (Ht + 2 rows)
  int Wt, Ht, Lt;
  int P, Hb, tpl;   // mode 2: padded row pitch, box rows, tiles per leaf
  uint32_t p_magic;  // floor(2^32 / P) + 1: q / P = umulhi(q, p_magic) for q < 2^16 (0: divide)
  // Mode 3 (phase form of a decoder convolution over [upsample(U), S]): the
  // tile is 128 padded-row positions of the half-resolution grid (pitch P)
  // in npt of the 4 output phases (py, px), one subtile per phase; output
  // pixel (2y + py, 2x + px).  kS stages read S, the full-resolution skip
  // input, as four parity sub-grids (boxes of box_a bytes); kU stages read
  // U, the half-resolution input, as one box.
  int npt, kS, kU, CinU;
  uint32_t box_a, btap, tx_u;
  int num_tiles, kiters, stages;
  uint32_t bytes_a, bytes_b;  // per stage (A rounded up to 1 KB in mode 2)
  uint32_t tx_bytes;          // bytes the TMA copies of one stage deliver
  int chunk_bytes;            // bytes of one operand row (the swizzle row)
  int stage_out;              // epilogue stores: 0 direct, 1 staged through shared memory (coalesced),
                              // 2 staged and written by bulk async copies (dense rows of 64-byte pixels)
  uint32_t idesc;
  uint32_t sbo;
  int swz;
  uint32_t sbo_b;  // B operand's stride between 8-row groups and swizzle mode (A's, except in mode 4)
  int swz_b;
  int mma_per_stage, mma_kind;  // 0: kind::f16, 1: kind::f8f6f4
  uint32_t tmem_cols;
  // epilogue
  void *out;
  int out_cs, out_co, ups, act, out_fp8;
  float out_mul;   // value multiplier before the output conversion (1/scale for FP8 outputs)
  float acc_mul;   // accumulator multiplier (product of the FP8 operand scales, 1 otherwise)
  // Mixture of experts in one launch: tiles of leaf positions
  // [exp_range[e], exp_range[e+1]) (chunk positions offset by pos0) take
  // expert e's weights, bias and head; n_exp = 1 otherwise.
  int n_exp, pos0;
  const int *exp_range;
  const float *bias[kMaxExperts];
  // Weight images (per expert): each stage's weight blocks of btap bytes as
  // they lie in shared memory, in the K order of the operand mode, copied
  // by one bulk copy per stage; null: per-block tensor loads.
  const uint8_t *bimg[kMaxExperts];
  uint32_t *status;
  unsigned int *amax;  // optional: running max |output| (float bits) for FP8 calibration
  unsigned long long *stats;  // optional: per-role cycle counters (diagnostics)
  // Optional fused 1x1 head (Cout 1) + softplus: the epilogue writes the FP32
  // map y instead of the layer's activations.
  const float *head_w[kMaxExperts], *head_b[kMaxExperts];
  float *head_y;
  // Paper-style layers: taps dil apart (operand mode 0 only); per output
  // pixel partial-convolution scale (null: plain layer; 0: output act(0));
  // residual link (BF16, same pixel indexing as the output) added after the
  // activation.
  int dil;
  const float *pscale;
  const void *res;
  int res_cs, res_co;
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.  Returns false when the
// CTA is aborting (this wait timed out, or another role already gave up).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long limit_ns = kTimeoutNs) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_4d(const CUtensorMap *map, uint64_t *bar, void *dst, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
      "%6}], [%2];" ::"r"(saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap *map, uint64_t *bar, void *dst, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Plain bulk copy global -> shared (16-byte aligned, a multiple of 16
// bytes), completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One MMA with descriptors given as (low, high) words.
template <bool kFp8>
__device__ __forceinline__ void mma_issue(uint32_t d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                          uint32_t idesc, uint32_t acc) {
  if (kFp8)
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 da, db;\n mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n"
        " setp.ne.b32 p, %6, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], da, db, %5, p;\n}\n" ::"r"(d),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 da, db;\n mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n"
        " setp.ne.b32 p, %6, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(d),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Output-tile origin of tile t: first leaf, row and column of the tile.
__device__ __forceinline__ void tile_origin(const TcArgs &a, int t, int &l0, int &y0, int &x0) {
  long m0 = (long)t * kBM * a.mt;
  l0 = (int)(m0 / a.HWo);
  int r = (int)(m0 % a.HWo);
  y0 = r / a.Wout;
  x0 = r % a.Wout;
}

// Expert of the tile whose first leaf is chunk position l0 (s_range: the
// experts' position ranges, n_exp + 1 boundaries).
__device__ __forceinline__ int tile_expert(const TcArgs &a, const int *s_range, int l0) {
  int e = 0;
  const int pos = a.pos0 + l0;
  while (e + 1 < a.n_exp && pos >= s_range[e + 1]) ++e;
  return e;
}

// ELU for the reduced-precision forms: exp(v) - 1 through the fast exponential
// (its ~1e-7 absolute error is far below a BF16 or E4M3 output's rounding).
__device__ __forceinline__ float elu_lp(float v) { return v > 0.0f ? v : __expf(v) - 1.0f; }

// 2^x by the PTX ex2.approx instruction (relative error at most 2^-22,
// subnormal results flushed to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// e^v - 1 of two values on packed FP32 pairs: e^v = 2^(v log2 e), one
// multiply and one add for both values.
__device__ __forceinline__ float2 expm1_pair(float2 v) {
  constexpr float kLog2e = 1.4426950408889634f;
  const float2 u = __fmul2_rn(v, make_float2(kLog2e, kLog2e));
  return __fadd2_rn(make_float2(ex2_approx(u.x), ex2_approx(u.y)), make_float2(-1.0f, -1.0f));
}

// ELU of two values without a branch: e^v - 1 >= v for every v, so
// min(e^v - 1, max(v, 0)) is v above zero and e^v - 1 at or below it.
__device__ __forceinline__ float2 elu_pair(float2 v) {
  const float2 e = expm1_pair(v);
  return make_float2(fminf(e.x, fmaxf(v.x, 0.0f)), fminf(e.y, fmaxf(v.y, 0.0f)));
}

// BF16 output of 16 accumulator columns of one pixel without partial-conv
// scales, residuals or calibration: bias add and the ELU's arithmetic on
// packed FP32 pairs (one instruction per two columns), and the ELU's min/max
// on packed BF16 pairs after the conversion (rounding to BF16 is monotone,
// so min and max commute with it; the max with 0 is the conversion's .relu).
__device__ __forceinline__ void epi_bf16_pairs(const TcArgs &a, const uint32_t *r, const float *bias, uint4 *chunk) {
  const float2 m2 = make_float2(a.acc_mul, a.acc_mul);
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const float4 b = *reinterpret_cast<const float4 *>(bias + 2 * j);
    float2 v[2];
    v[0] = __ffma2_rn(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])), m2,
                      make_float2(b.x, b.y));
    v[1] = __ffma2_rn(make_float2(__uint_as_float(r[2 * j + 2]), __uint_as_float(r[2 * j + 3])), m2,
                      make_float2(b.z, b.w));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      __nv_bfloat162 o;
      if (a.act == 1) {
        // max(v, 0) comes from the conversion itself (cvt .relu).
        uint32_t pos;
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(pos) : "f"(v[h].y), "f"(v[h].x));
        const float2 e = expm1_pair(v[h]);
        o = __hmin2(__floats2bfloat162_rn(e.x, e.y), *reinterpret_cast<const __nv_bfloat162 *>(&pos));
      } else {
        o = __floats2bfloat162_rn(v[h].x, v[h].y);
      }
      w[j + h] = *reinterpret_cast<uint32_t *>(&o);
    }
  }
  chunk[0] = make_uint4(w[0], w[1], w[2], w[3]);
  chunk[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Bias + activation + conversion of 16 accumulator columns of one pixel into
// output bytes: one 16-byte chunk (E4M3) or two (BF16).
template <bool kFp8Out, bool kCalib>
__device__ __forceinline__ void epi_convert16(const TcArgs &a, const uint32_t *r, const float *s_bias, int c,
                                              float &amax, uint4 *chunk, float ps = 1.0f,
                                              const __nv_bfloat16 *resp = nullptr) {
  if (!kFp8Out && !kCalib && !a.pscale && !resp) {
    epi_bf16_pairs(a, r, s_bias + c, chunk);
    return;
  }
  float v[16];
  if (a.pscale) {
    // Partial convolution: acc * scale + bias where a valid input lies under
    // the window, else 0 (before the activation).
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = ps > 0.0f ? fmaf(__uint_as_float(r[j]) * a.acc_mul, ps, s_bias[c + j]) : 0.0f;
  } else {
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
      const float4 b = *reinterpret_cast<const float4 *>(s_bias + c + j);
      v[j] = fmaf(__uint_as_float(r[j]), a.acc_mul, b.x);
      v[j + 1] = fmaf(__uint_as_float(r[j + 1]), a.acc_mul, b.y);
      v[j + 2] = fmaf(__uint_as_float(r[j + 2]), a.acc_mul, b.z);
      v[j + 3] = fmaf(__uint_as_float(r[j + 3]), a.acc_mul, b.w);
    }
  }
  if (a.act == 1) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = elu_lp(v[j]);
  }
  if (resp) {
    const uint4 q0 = *reinterpret_cast<const uint4 *>(resp), q1 = *reinterpret_cast<const uint4 *>(resp + 8);
    const uint32_t qw[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&qw[j]));
      v[2 * j] += f.x;
      v[2 * j + 1] += f.y;
    }
  }
  if (kCalib) {
#pragma unroll
    for (int j = 0; j < 16; ++j) amax = fmaxf(amax, fabsf(v[j]));
  }
  if (kFp8Out) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_fp8x4_e4m3 p(make_float4(v[4 * j] * a.out_mul, v[4 * j + 1] * a.out_mul, v[4 * j + 2] * a.out_mul,
                                    v[4 * j + 3] * a.out_mul));
      w[j] = *reinterpret_cast<uint32_t *>(&p);
    }
    chunk[0] = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      w[j] = *reinterpret_cast<uint32_t *>(&p);
    }
    chunk[0] = make_uint4(w[0], w[1], w[2], w[3]);
    chunk[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// Direct output of one work item: each lane stores its own pixel's chunks.
__device__ __forceinline__ void store_direct(const TcArgs &a, const uint4 *chunk, int cpp, int c0, size_t pix0,
                                             int Wo, int reps, int es) {
  uint8_t *out = (uint8_t *)a.out;
  for (int dy = 0; dy < reps; ++dy)
    for (int dx = 0; dx < reps; ++dx) {
      const size_t pix = pix0 + (size_t)dy * Wo + dx;
      uint4 *o = reinterpret_cast<uint4 *>(out + (pix * a.out_cs + a.out_co + c0) * es);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < cpp) o[k] = chunk[k];
    }
}

// Coalesced output of one work item: every lane holds `cpp` 16-byte chunks
// of its own pixel (channels c0.. of the layer's output).  The chunks go
// through a per-warp staging buffer (chunk slots XOR-swizzled by pixel so
// that neither side conflicts on banks) and leave as runs of 16 * cpp
// contiguous bytes per pixel, 32 / cpp pixels per store instruction,
// instead of one scattered 16-byte store per lane.
__device__ __forceinline__ void store_staged(const TcArgs &a, uint8_t *stg, const uint4 *chunk, int cpp, int c0,
                                             size_t pix0, bool valid, int Wo, int reps, int lane, int es) {
  const int sh = cpp == 4 ? 1 : 2;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < cpp) {
      const int slot = k ^ ((lane >> sh) & (cpp - 1));
      *reinterpret_cast<uint4 *>(stg + (lane * cpp + slot) * 16) = chunk[k];
    }
  __syncwarp();
  const int ppi = 32 / cpp;  // pixels per store instruction
  const int c = lane & (cpp - 1);
  uint8_t *out = (uint8_t *)a.out;
  for (int it = 0; it < cpp; ++it) {
    const int p = it * ppi + lane / cpp;
    const uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)pix0, p);
    const uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(pix0 >> 32), p);
    const int ok = __shfl_sync(0xFFFFFFFFu, valid ? 1 : 0, p);
    const uint4 v = *reinterpret_cast<const uint4 *>(stg + (p * cpp + (c ^ ((p >> sh) & (cpp - 1)))) * 16);
    if (ok) {
      const size_t px = ((size_t)hi << 32) | lo;
      for (int dy = 0; dy < reps; ++dy)
        for (int dx = 0; dx < reps; ++dx) {
          const size_t pix = px + (size_t)dy * Wo + dx;
          *reinterpret_cast<uint4 *>(out + (pix * a.out_cs + a.out_co + c0) * es + c * 16) = v;
        }
    }
  }
  __syncwarp();
}

// Bulk output of one work item (mode 2, a dense output of 32 BF16 channels:
// every pixel is 64 contiguous bytes, and consecutive valid positions of a
// padded row are consecutive pixels).  Each lane puts its pixel into the
// warp's staging buffer; every lane that starts a run of consecutive valid
// pixels then writes the run with one bulk async copy, so the global stores
// leave the epilogue's critical path.  A lane waits for the shared-memory
// reads of its earlier copies before the buffer is rewritten.
__device__ __forceinline__ void store_bulk(uint8_t *stg, const uint4 *chunk, size_t pix0, bool valid, int lane,
                                           uint8_t *out) {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncwarp();
  // Chunk k of the pixel goes out in round (k - lane) mod 4, so that lanes
  // L and L + 1 of an 8-lane phase hit different banks.
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int kk = (k + lane) & 3;
    const uint4 v = kk == 0 ? chunk[0] : (kk == 1 ? chunk[1] : (kk == 2 ? chunk[2] : chunk[3]));
    *reinterpret_cast<uint4 *>(stg + lane * 64 + kk * 16) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
  const unsigned long long prev = __shfl_up_sync(0xFFFFFFFFu, (unsigned long long)pix0, 1);
  const bool start = valid && (lane == 0 || !((vmask >> (lane - 1)) & 1u) || prev + 1ull != (unsigned long long)pix0);
  const unsigned smask = __ballot_sync(0xFFFFFFFFu, start);
  if (start) {
    const unsigned brk = (smask | ~vmask) & ~((2u << lane) - 1u);  // lanes after this one that end the run
    const int end = (lane == 31 || brk == 0u) ? 32 : __ffs(brk) - 1;
    const uint32_t bytes = (uint32_t)(end - lane) * 64u;
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(out + pix0 * 64ull),
                 "r"(saddr(stg + lane * 64)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
}

// Descriptor words and offsets of one pipeline stage (see the MMA issuer).
struct StageOps {
  uint32_t d, BN, alo, blo, a_byte0;
  int off0, P;
  uint32_t cb, sub_step, row_step, ver16, tap_b16, desc_hi, idesc;
  bool first;
  uint32_t desc_hi_b;  // B descriptor's high word (A's, except in mode 4)
  int sub;  // the 128-row subtile (and accumulator) this issuing lane owns
  uint32_t box_a;  // mode 3: bytes between the parity sub-grid boxes
};

// The MMAs of one stage for one subtile, as straight-line code: a
// tcgen05.mma stream issued from a loop with run-time trip counts runs about
// 3x slower per instruction than the same stream unrolled, so every (mode,
// K steps) combination gets its own fully unrolled sequence.  The K order of
// an accumulator is (tap, K step) in every mode.
template <bool kFp8, int kMode, int kMPS>
__device__ __forceinline__ void issue_stage(const StageOps &o) {
  const uint32_t d = o.d + (uint32_t)o.sub * o.BN;
  if constexpr (kMode == 0) {
    const uint32_t a0 = o.alo + (uint32_t)o.sub * o.sub_step;
#pragma unroll
    for (int j = 0; j < kMPS; ++j)
      mma_issue<kFp8>(d, a0 + 2u * j, o.desc_hi, o.blo + 2u * j, o.desc_hi_b, o.idesc, (o.first && j == 0) ? 0u : 1u);
  } else {
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const uint32_t b_tap = o.blo + (uint32_t)(ky * 3 + kx) * o.tap_b16;
        uint32_t a_tap;
        if constexpr (kMode == 1) {
          // Copy kx of the haloed tile, from row ky * Wt on.
          a_tap = o.alo + (uint32_t)kx * o.ver16 + (uint32_t)ky * o.row_step + (uint32_t)o.sub * o.sub_step;
        } else {
          // Padded row off0 + ky * P + kx of the box.  Any starting row
          // works: the MMA, like the TMA that wrote the box, applies the
          // swizzle to absolute shared-memory address bits of the
          // 1-KB-aligned buffer (base offset 0).
          const uint32_t addr = o.a_byte0 + ((uint32_t)(o.off0 + ky * o.P + kx) + (uint32_t)(o.sub * kBM)) * o.cb;
          a_tap = ((addr & 0x3FFFFu) >> 4) | (1u << 16);
        }
#pragma unroll
        for (int j = 0; j < kMPS; ++j) {
          const uint32_t acc = (o.first && ky == 0 && kx == 0 && j == 0) ? 0u : 1u;
          mma_issue<kFp8>(d, a_tap + 2u * j, o.desc_hi, b_tap + 2u * j, o.desc_hi_b, o.idesc, acc);
        }
      }
    }
  }
}

// Mode 3: the MMAs of one stage for the subtile of output phase (py, px).
// An S stage holds the four parity sub-grids of the full-resolution input:
// tap (ky, kx) reads row 2y + py + ky - 1 = 2 (y + sy / 2 - 1) + sy % 2 with
// sy = py + ky + 1, i.e. box row sy / 2 of parity sub-grid sy % 2 (likewise
// for columns).  A U stage holds the half-resolution input: the phase's 2x2
// taps (i, j) read box row py + i and column px + j, with weights that sum
// the 3x3 taps falling on the same upsampled pixel.
template <int kMPS>
__device__ __forceinline__ void issue_stage3(const StageOps &o, bool u_stage, int py, int px) {
  const uint32_t d = o.d + (uint32_t)o.sub * o.BN;
  const uint32_t row0 = o.a_byte0 + (uint32_t)o.off0 * o.cb;
  if (!u_stage) {
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int sy = py + ky + 1;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int sx = px + kx + 1;
        const uint32_t addr = row0 + (uint32_t)((sy & 1) * 2 + (sx & 1)) * o.box_a +
                              (uint32_t)((sy >> 1) * o.P + (sx >> 1)) * o.cb;
        const uint32_t a_tap = ((addr & 0x3FFFFu) >> 4) | (1u << 16);
        const uint32_t b_tap = o.blo + (uint32_t)(ky * 3 + kx) * o.tap_b16;
#pragma unroll
        for (int j = 0; j < kMPS; ++j) {
          const uint32_t acc = (o.first && ky == 0 && kx == 0 && j == 0) ? 0u : 1u;
          mma_issue<false>(d, a_tap + 2u * j, o.desc_hi, b_tap + 2u * j, o.desc_hi_b, o.idesc, acc);
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
      for (int jx = 0; jx < 2; ++jx) {
        const uint32_t addr = row0 + (uint32_t)((py + i) * o.P + px + jx) * o.cb;
        const uint32_t a_tap = ((addr & 0x3FFFFu) >> 4) | (1u << 16);
        const uint32_t b_tap = o.blo + (uint32_t)(o.sub * 4 + i * 2 + jx) * o.tap_b16;
#pragma unroll
        for (int j = 0; j < kMPS; ++j)
          mma_issue<false>(d, a_tap + 2u * j, o.desc_hi, b_tap + 2u * j, o.desc_hi_b, o.idesc, 1u);
      }
    }
  }
}

// Mode 4 (a stride-2 3x3 layer over 32 BF16 channels): the input is read as
// pixel pairs, one 128-byte row (pixels 2x and 2x + 1) per output column x.
// Stage 2 ky holds the pairs at x - 1, whose second pixel 2x - 1 is tap
// (ky, 0) (K steps 2-3 of the row); stage 2 ky + 1 holds the pairs at x: taps
// (ky, 1) and (ky, 2) are the first and the second 64 bytes of each row (K
// steps 0-1 and 2-3 against the two taps' weight blocks).  The MMAs follow
// mode 0's K order (tap, K step), so the accumulators are the same.
__device__ __forceinline__ void issue_stage4(const StageOps &o, bool prev_pair) {
  const uint32_t d = o.d + (uint32_t)o.sub * o.BN;
  const uint32_t a0 = o.alo + (uint32_t)o.sub * o.sub_step;
  if (prev_pair) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
      mma_issue<false>(d, a0 + 2u * (2 + j), o.desc_hi, o.blo + 2u * j, o.desc_hi_b, o.idesc,
                       (o.first && j == 0) ? 0u : 1u);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      mma_issue<false>(d, a0 + 2u * j, o.desc_hi, o.blo + (uint32_t)(j >> 1) * o.tap_b16 + 2u * (j & 1), o.desc_hi_b,
                       o.idesc, 1u);
  }
}

// Mode 3 tile t: leaf l0, phase group g (phases g * npt ..) and first
// position q0 of the half-resolution padded rows.
__device__ __forceinline__ void tile_origin3(const TcArgs &a, int t, int &l0, int &g, int &q0) {
  const int groups = 4 / a.npt, per_leaf = groups * a.tpl;
  l0 = t / per_leaf;
  const int r = t - l0 * per_leaf;
  g = r / a.tpl;
  q0 = (r - g * a.tpl) * kBM;
}

template <bool kFp8Out, bool kCalib>
__global__ void __launch_bounds__(kThreads, 2)
    k_conv_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapU,
              const __grid_constant__ TcMapsB mapsB, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;
  uint8_t *sB = sA + (size_t)a.stages * a.bytes_a;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + (size_t)a.stages * a.bytes_b);
  uint64_t *empty = full + a.stages;
  uint64_t *acc_full = empty + a.stages;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  // Per expert: BN bias floats, then (fused head only) BN head weights and
  // the head's bias in a block of BN + 4 floats (16-byte aligned per expert);
  // then the experts' position ranges.
  const int head_n = a.head_y ? a.BN + 4 : 0;
  float *s_bias = reinterpret_cast<float *>(((uintptr_t)(tmem_slot + 2) + 15) & ~(uintptr_t)15);  // n_exp x BN
  float *s_head = s_bias + a.n_exp * a.BN;                                                         // n_exp x head_n
  int *s_range = reinterpret_cast<int *>(s_head + a.n_exp * head_n);                              // n_exp + 1
  uint8_t *s_stage =
      reinterpret_cast<uint8_t *>(((uintptr_t)(s_range + a.n_exp + 1) + 15) & ~(uintptr_t)15);  // 8 x 2 KB
  for (int e = 0; e < a.n_exp; ++e) {
    for (int k = threadIdx.x; k < a.BN; k += blockDim.x) s_bias[e * a.BN + k] = a.bias[e][k];
    if (a.head_y) {
      for (int k = threadIdx.x; k < a.BN; k += blockDim.x) s_head[e * head_n + k] = a.head_w[e][k];
      if (threadIdx.x == 0) s_head[e * head_n + a.BN] = a.head_b[e][0];
    }
  }
  for (int k = threadIdx.x; k <= a.n_exp; k += blockDim.x) s_range[k] = a.n_exp > 1 ? a.exp_range[k] : 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], a.mt);  // one commit per issuing lane
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], a.mt);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, a.mt);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    if (a.halo == 3) asm volatile("prefetch.tensormap [%0];" ::"l"(&mapU) : "memory");
    for (int e = 0; e < a.n_exp; ++e) asm volatile("prefetch.tensormap [%0];" ::"l"(&mapsB.b[e]) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer: lane 0 owns the ring; the copies of one
    // stage are issued by separate lanes so they enter the TMA unit together.
    int stage = 0;
    uint32_t phase = 0;
    long issued = 0;
    bool ok = true;
    long long prod_wait = 0;
    const long long prod_t0 = clock64();
    const int ntma = a.halo == 3 ? 17 : (a.halo == 2 ? 10 : (a.halo ? 12 : 2));
    for (int t = blockIdx.x; t < a.num_tiles && ok; t += gridDim.x) {
      int l0, y0, x0, g = 0;
      if (a.halo == 3) {
        int q0;
        tile_origin3(a, t, l0, g, q0);
        y0 = q0 / a.P - 1;
        x0 = -1;
      } else if (a.halo == 2) {
        // Leaf of the tile, and the first box row: the image row above the
        // tile's first output row (row -1 and rows >= H are zero-filled).
        l0 = t / a.tpl;
        y0 = ((t - l0 * a.tpl) * kBM * a.mt) / a.P - 1;
        x0 = -1;
      } else {
        tile_origin(a, t, l0, y0, x0);
      }
      const int te = a.n_exp > 1 ? tile_expert(a, s_range, l0) : 0;
      const CUtensorMap *mapB = &mapsB.b[te];
      const uint8_t *img = a.bimg[te];
      for (int ki = 0; ki < a.kiters; ++ki) {
        int got = 1;
        if (lane == 0) {
          const long long c0 = clock64();
          got = mbar_wait(&empty[stage], phase ^ 1u, abort_flag) ? 1 : 0;
          prod_wait += clock64() - c0;
          if (got)
            mbar_expect_tx(&full[stage], ((a.halo == 3 && ki >= a.kS) || (a.halo == 4 && !(ki & 1))) ? a.tx_u
                                                                                                   : a.tx_bytes);
        }
        got = __shfl_sync(0xFFFFFFFFu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
        __syncwarp();
        if (img && lane == 31) {
          // The stage's weight blocks, contiguous in the image: mode 0 one
          // block per (tap, chunk); modes 1-2 the 9 taps of chunk ki; mode 3
          // the 9 taps of skip chunk ki, or the 2x2 taps of the tile's phases
          // for U chunk ki - kS (16 blocks per U chunk, 4 per phase).
          int b0 = ki, nb = 1;
          if (a.halo == 4) {
            // Row ky's tap 0 (pairs at x - 1) or taps 1-2 (pairs at x).
            b0 = 3 * (ki >> 1) + ((ki & 1) ? 1 : 0);
            nb = (ki & 1) ? 2 : 1;
          } else if (a.halo == 3 && ki >= a.kS) {
            b0 = 9 * a.kS + (ki - a.kS) * 16 + g * 4 * a.npt;
            nb = 4 * a.npt;
          } else if (a.halo) {
            b0 = 9 * ki;
            nb = 9;
          }
          bulk_load(sB + (size_t)stage * a.bytes_b, img + (size_t)b0 * a.btap, (uint32_t)nb * a.btap, &full[stage]);
        }
        if (lane < ntma) {
          if (a.halo == 4) {
            const int ky = ki >> 1, prev = (ki & 1) ^ 1;
            if (lane == 0)
              tma_load_4d(&mapA, &full[stage], sA + (size_t)stage * a.bytes_a, 0, x0 - prev, 2 * y0 + ky - 1, l0);
            else if (lane <= 2 - prev && !img)
              tma_load_2d(mapB, &full[stage], sB + (size_t)stage * a.bytes_b + (size_t)(lane - 1) * a.btap,
                          (3 * ky + (prev ? 0 : 1) + lane - 1) * a.Cin, 0);
          } else if (a.halo == 3) {
            uint8_t *dA = sA + (size_t)stage * a.bytes_a, *dB = sB + (size_t)stage * a.bytes_b;
            if (ki < a.kS) {
              // Lane b loads parity sub-grid b (rows 2r + b / 2, columns
              // 2c + b % 2) of the skip input; lanes 4..12 the 9 taps' weights.
              const int cc = ki;
              if (lane < 4)
                tma_load_4d(&mapA, &full[stage], dA + (size_t)lane * a.box_a, cc * a.chunk, 2 * x0 + (lane & 1),
                            2 * y0 + (lane >> 1), l0);
              else if (lane < 13 && !img)
                tma_load_2d(mapB, &full[stage], dB + (size_t)(lane - 4) * a.btap, (lane - 4) * a.Cin + cc * a.chunk, 0);
            } else {
              // Lane 0 loads the half-resolution box; lanes 1..4 npt the 2x2
              // taps' combined weights of the tile's phases.
              const int cc = ki - a.kS;
              if (lane == 0) {
                tma_load_4d(&mapU, &full[stage], dA, cc * a.chunk, x0, y0, l0);
              } else if (lane <= 4 * a.npt && !img) {
                const int j = lane - 1, ph = g * a.npt + (j >> 2);
                tma_load_2d(mapB, &full[stage], dB + (size_t)j * a.btap,
                            9 * a.Cin + (ph * 4 + (j & 3)) * a.CinU + cc * a.chunk, 0);
              }
            }
          } else if (a.halo == 2) {
            const int cc = ki;
            if (lane == 0)
              tma_load_4d(&mapA, &full[stage], sA + (size_t)stage * a.bytes_a, cc * a.chunk, x0, y0, l0);
            else if (!img)
              tma_load_2d(mapB, &full[stage], sB + (size_t)stage * a.bytes_b + (size_t)(lane - 1) * (a.bytes_b / 9),
                          (lane - 1) * a.Cin + cc * a.chunk, 0);
          } else if (a.halo) {
            // Three copies of the haloed input tile (rows y0-1 .. y0+Ht),
            // shifted by kx - 1 columns; out-of-range columns and rows are
            // zero-filled.  Tap (ky, kx) is then rows ky*Wt.. of copy kx.
            const int cc = ki;
            if (lane < 3)
              tma_load_4d(&mapA, &full[stage], sA + (size_t)stage * a.bytes_a + (size_t)lane * a.bytes_ver,
                          cc * a.chunk, x0 + lane - 1, y0 - 1, l0);
            else if (!img)
              tma_load_2d(mapB, &full[stage], sB + (size_t)stage * a.bytes_b + (size_t)(lane - 3) * (a.bytes_b / 9),
                          (lane - 3) * a.Cin + cc * a.chunk, 0);
          } else {
            int tap = ki / a.cchunks, cc = ki - tap * a.cchunks;
            int ky = tap / a.k, kx = tap - ky * a.k;
            if (lane == 0)
              tma_load_4d(&mapA, &full[stage], sA + (size_t)stage * a.bytes_a, cc * a.chunk,
                          x0 * a.stride + kx * a.dil - a.pad, y0 * a.stride + ky * a.dil - a.pad, l0);
            else if (!img)
              tma_load_2d(mapB, &full[stage], sB + (size_t)stage * a.bytes_b, tap * a.Cin + cc * a.chunk, 0);
          }
        }
        ++issued;
        if (++stage == a.stages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (lane == 0 && a.stats) {
      atomicAdd(&a.stats[0], (unsigned long long)prod_wait);
      atomicAdd(&a.stats[1], (unsigned long long)(clock64() - prod_t0));
    }
    if (lane == 0 && *abort_flag) {
      // Drain: let the last stages' copies land before the CTA exits.
      long back = issued < a.stages ? issued : a.stages;
      for (long q = 0; q < back; ++q) {
        if (--stage < 0) {
          stage = a.stages - 1;
          phase ^= 1u;
        }
        volatile int never = 0;
        mbar_wait(&full[stage], phase, &never, 100000000ull);
      }
    }
  } else if (warp == 1) {
    if (lane < a.mt) {
      // ---------------- MMA issuers: lane s issues subtile s (the converged
      // lanes issue their MMAs together).
      int stage = 0;
      uint32_t phase = 0;
      int i = 0;
      const uint32_t a_base = saddr(sA), b_base = saddr(sB);
      // Descriptor words (see smem_desc): low = start address >> 4 | LBO,
      // high = SBO >> 4 | version | swizzle mode.
      const uint32_t desc_hi = ((a.sbo >> 4) & 0x3FFFu) | (1u << 14) | ((uint32_t)(a.swz & 7) << 29);
      const uint32_t desc_hi_b = ((a.sbo_b >> 4) & 0x3FFFu) | (1u << 14) | ((uint32_t)(a.swz_b & 7) << 29);
      const uint32_t a_lo0 = ((a_base & 0x3FFFFu) >> 4) | (1u << 16), b_lo0 = ((b_base & 0x3FFFFu) >> 4) | (1u << 16);
      const uint32_t row16 = a.sbo / 8 / 16;                 // one operand row, in 16-byte units
      const uint32_t sub_step = (uint32_t)kBM * row16;       // next 128-row subtile
      const uint32_t row_step = (uint32_t)a.Wt * row16;      // halo mode: next tap row
      const uint32_t ver16 = a.bytes_ver >> 4;               // halo mode: next x-shifted copy
      const uint32_t tap_b16 = (a.halo >= 3 ? a.btap : a.bytes_b / 9) >> 4;  // next tap's weights
      long long mma_wait_acc = 0, mma_wait_full = 0;
      const long long mma_t0 = clock64();
      for (int t = blockIdx.x; t < a.num_tiles && !*abort_flag; t += gridDim.x, ++i) {
        const int buf = i & 1;
        const uint32_t use = (uint32_t)(i >> 1) & 1u;
        long long c0 = clock64();
        if (!mbar_wait(&acc_empty[buf], use ^ 1u, abort_flag)) break;
        mma_wait_acc += clock64() - c0;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * a.mt * a.BN);
        int off0 = a.halo == 2 ? ((t % a.tpl) * kBM * a.mt) % a.P : 0;
        int py = 0, px = 0;
        if (a.halo == 3) {
          int l0, g, q0;
          tile_origin3(a, t, l0, g, q0);
          off0 = q0 % a.P;
          const int ph = g * a.npt + lane;  // this lane's subtile is one output phase
          py = ph >> 1;
          px = ph & 1;
        }
        bool ok = true;
        for (int ki = 0; ki < a.kiters; ++ki) {
          c0 = clock64();
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          mma_wait_full += clock64() - c0;
          // No tcgen05 fence here: the TMA writes this stage's operands
          // through the async proxy and the mbarrier's transaction count
          // already orders them before the MMAs that read them.
          // Descriptors move by adding (byte offset >> 4) to the 14-bit
          // start-address field of the low word (shared memory < 256 KB, so
          // the field never carries); the high word is fixed per launch.
          const uint32_t alo_s = a_lo0 + (uint32_t)stage * (a.bytes_a >> 4);
          const uint32_t blo_s = b_lo0 + (uint32_t)stage * (a.bytes_b >> 4);
          const bool first = ki == 0;
          const StageOps so{d,         (uint32_t)a.BN, alo_s,        blo_s,   a_base + (uint32_t)stage * a.bytes_a,
                            off0,      a.P,            (uint32_t)a.chunk_bytes, sub_step, row_step, ver16, tap_b16,
                            desc_hi,   a.idesc,        first,   desc_hi_b,              lane,     a.box_a};
          // The MMA kind follows the operands (a.mma_kind), which may differ
          // from the output type (a layer at a BF16/E4M3 boundary).
          if (a.halo == 4) {
            issue_stage4(so, (ki & 1) == 0);
          } else if (a.halo == 3) {
            const bool u_stage = ki >= a.kS;
            if (a.mma_per_stage == 1)
              issue_stage3<1>(so, u_stage, py, px);
            else if (a.mma_per_stage == 2)
              issue_stage3<2>(so, u_stage, py, px);
            else if (a.mma_per_stage == 4)
              issue_stage3<4>(so, u_stage, py, px);
          } else
          switch ((a.mma_kind ? 16 : 0) + a.halo * 4 + (a.mma_per_stage >> 1)) {
#define PG_STAGE_CASE(K, H, MPS) \
  case (K ? 16 : 0) + H * 4 + (MPS >> 1): issue_stage<K, H, MPS>(so); break;
            PG_STAGE_CASE(false, 0, 1) PG_STAGE_CASE(false, 0, 2) PG_STAGE_CASE(false, 0, 4)
            PG_STAGE_CASE(false, 1, 1) PG_STAGE_CASE(false, 1, 2) PG_STAGE_CASE(false, 1, 4)
            PG_STAGE_CASE(false, 2, 1) PG_STAGE_CASE(false, 2, 2) PG_STAGE_CASE(false, 2, 4)
            PG_STAGE_CASE(true, 0, 1) PG_STAGE_CASE(true, 0, 2) PG_STAGE_CASE(true, 0, 4)
            PG_STAGE_CASE(true, 1, 1) PG_STAGE_CASE(true, 1, 2) PG_STAGE_CASE(true, 1, 4)
            PG_STAGE_CASE(true, 2, 1) PG_STAGE_CASE(true, 2, 2) PG_STAGE_CASE(true, 2, 4)
#undef PG_STAGE_CASE
            default: break;
          }
          mma_commit(&empty[stage]);
          if (++stage == a.stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
      }
      if (a.stats && lane == 0) {
        atomicAdd(&a.stats[2], (unsigned long long)mma_wait_acc);
        atomicAdd(&a.stats[3], (unsigned long long)mma_wait_full);
        atomicAdd(&a.stats[4], (unsigned long long)(clock64() - mma_t0));
      }
      // All issued MMAs complete before TMEM is released.
      mma_commit(drain);
      volatile int never = 0;
      mbar_wait(drain, 0, &never, 200000000ull);
    }
  } else {
    // ---------------- epilogue: warps 2..9; warp w reads TMEM lane quarter
    // w % 4, and the two warps of a quarter split the tile's work items
    // (subtile, column chunk) between them.
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int m = q * 32 + lane;
    int i = 0;
    const int reps = a.ups ? 2 : 1;
    const int Ho = a.Hout * reps, Wo = a.Wout * reps;
    const int cw = (a.BN % 32 == 0 && a.mt * a.BN >= 64) ? 32 : 16;  // columns per work item
    const int per_sub = a.BN / cw, items = a.mt * per_sub;
    // Lean paths (uniform per launch): padded-row positions (mode 2) without
    // the x2 upsample, BF16 outputs without partial-conv scales, residuals
    // or calibration; rows found by one multiply-high instead of a division.
    const bool lean_in = a.halo == 2 && !a.ups && a.p_magic && !kFp8Out && !kCalib && !a.pscale && !a.res;
    const bool lean = lean_in && !a.head_y && cw == 32 && (per_sub & (per_sub - 1)) == 0 && a.stage_out < 2;
    const bool lean_head = lean_in && a.head_y;
    const int lg_ps = __ffs(per_sub) - 1;
    float amax_local = 0.0f;
    long long epi_wait = 0;
    const long long epi_t0 = clock64();
    for (int t = blockIdx.x; t < a.num_tiles; t += gridDim.x, ++i) {
      const int buf = i & 1;
      const uint32_t use = (uint32_t)(i >> 1) & 1u;
      const long long c0 = clock64();
      if (!mbar_wait(&acc_full[buf], use, abort_flag)) break;
      epi_wait += clock64() - c0;
      tc_fence_after();
      int l0 = 0, y0 = 0, x0 = 0, q0 = 0, g = 0;
      if (a.halo == 3) {
        tile_origin3(a, t, l0, g, q0);
      } else if (a.halo == 2) {
        l0 = t / a.tpl;
        q0 = (t - l0 * a.tpl) * kBM * a.mt;
      } else {
        tile_origin(a, t, l0, y0, x0);
      }
      // The tile's expert: its bias and head.
      const int te = a.n_exp > 1 ? tile_expert(a, s_range, l0) : 0;
      const float *eb = s_bias + te * a.BN, *eh = s_head + te * head_n;
      if (lean_head) {
        // Fused head, one whole pixel per thread: bias, ELU and the head's
        // dot product on FP32 pairs.
        const float2 m2 = make_float2(a.acc_mul, a.acc_mul);
        for (int sub = h; sub < a.mt; sub += 2) {
          const uint32_t qq = (uint32_t)(q0 + sub * kBM + m);
          const int y = (int)__umulhi(qq, a.p_magic), x = (int)qq - y * a.P;
          const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * a.mt * a.BN + sub * a.BN);
          float2 hacc2 = make_float2(0.0f, 0.0f);
          for (int c = 0; c < a.BN; c += 16) {
            uint32_t r[16];
            tmem_ld16(trow + (uint32_t)c, r);
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 b = *reinterpret_cast<const float4 *>(eb + c + j);
              const float4 w = *reinterpret_cast<const float4 *>(eh + c + j);
              float2 v0 = __ffma2_rn(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])), m2,
                                     make_float2(b.x, b.y));
              float2 v1 = __ffma2_rn(make_float2(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])), m2,
                                     make_float2(b.z, b.w));
              if (a.act == 1) {
                v0 = elu_pair(v0);
                v1 = elu_pair(v1);
              }
              hacc2 = __ffma2_rn(make_float2(w.x, w.y), v0, hacc2);
              hacc2 = __ffma2_rn(make_float2(w.z, w.w), v1, hacc2);
            }
          }
          if (y < a.Hout && x < a.Wout) {
            const float v = (hacc2.x + hacc2.y) + eh[a.BN];
            a.head_y[((size_t)l0 * a.Hout + y) * a.Wout + x] = fmaxf(v, 0.0f) + log1pf(__expf(-fabsf(v)));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        continue;
      }
      if (lean) {
        for (int it = h; it < items; it += 2) {
          const int sub = it >> lg_ps, c = (it & (per_sub - 1)) * 32;
          const uint32_t qq = (uint32_t)(q0 + sub * kBM + m);
          const int y = (int)__umulhi(qq, a.p_magic), x = (int)qq - y * a.P;
          const bool valid = y < a.Hout && x < a.Wout;
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * a.mt * a.BN + sub * a.BN + c), r);
          uint4 chunk[4];
          epi_bf16_pairs(a, r, eb + c, chunk);
          epi_bf16_pairs(a, r + 16, eb + c + 16, chunk + 2);
          const size_t pix0 = ((size_t)l0 * a.Hout + y) * a.Wout + x;
          if (a.stage_out) {
            store_staged(a, s_stage + (warp - 2) * 2048, chunk, 4, c, pix0, valid, a.Wout, 1, lane, 2);
          } else if (valid) {
            uint4 *o = reinterpret_cast<uint4 *>((__nv_bfloat16 *)a.out + pix0 * a.out_cs + a.out_co + c);
            o[0] = chunk[0];
            o[1] = chunk[1];
            o[2] = chunk[2];
            o[3] = chunk[3];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        continue;
      }
      if (a.head_y) {
        // Fused head: each thread owns whole pixels (all BN channels), so
        // the two warps of a lane quarter take alternate subtiles.
        for (int sub = h; sub < a.mt; sub += 2) {
          const int qq = q0 + sub * kBM + m;
          int leaf, y, x;
          bool valid;
          if (a.halo == 2) {
            leaf = l0;
            y = qq / a.P;
            x = qq - y * a.P;
            valid = y < a.Hout && x < a.Wout;
          } else {
            const int mm = sub * kBM + m;
            const int xx = mm % a.Wt, yy = (mm / a.Wt) % a.Ht, ll = mm / (a.Wt * a.Ht);
            leaf = l0 + ll;
            y = y0 + yy;
            x = x0 + xx;
            valid = (long)leaf * a.HWo + (long)y * a.Wout + x < a.M;
          }
          const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * a.mt * a.BN + sub * a.BN);
          const size_t hpix = ((size_t)leaf * a.Hout + y) * a.Wout + x;
          const float hps = (a.pscale && valid) ? a.pscale[hpix] : 0.0f;
          const __nv_bfloat16 *hres =
              (a.res && valid) ? (const __nv_bfloat16 *)a.res + hpix * a.res_cs + a.res_co : nullptr;
          float hacc = 0.0f;
          float2 hacc2 = make_float2(0.0f, 0.0f);
          for (int c = 0; c < a.BN; c += 16) {
            uint32_t r[16];
            tmem_ld16(trow + (uint32_t)c, r);
            if (!a.pscale && !hres && !kCalib) {
              // Bias, ELU and the head's dot product on packed FP32 pairs.
              const float2 m2 = make_float2(a.acc_mul, a.acc_mul);
#pragma unroll
              for (int j = 0; j < 16; j += 2) {
                float2 v = __ffma2_rn(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])), m2,
                                      make_float2(eb[c + j], eb[c + j + 1]));
                if (a.act == 1) v = elu_pair(v);
                hacc2 = __ffma2_rn(make_float2(eh[c + j], eh[c + j + 1]), v, hacc2);
              }
              continue;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float v = a.pscale ? (hps > 0.0f ? fmaf(__uint_as_float(r[j]) * a.acc_mul, hps, eb[c + j]) : 0.0f)
                                 : fmaf(__uint_as_float(r[j]), a.acc_mul, eb[c + j]);
              if (a.act == 1) v = elu_lp(v);
              if (hres) v += __bfloat162float(hres[c + j]);
              if (kCalib) amax_local = fmaxf(amax_local, fabsf(v));
              hacc = fmaf(eh[c + j], v, hacc);
            }
          }
          if (valid) {
            const float v = hacc + (hacc2.x + hacc2.y) + eh[a.BN];
            a.head_y[((size_t)leaf * a.Hout + y) * a.Wout + x] = fmaxf(v, 0.0f) + log1pf(__expf(-fabsf(v)));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        continue;
      }
      for (int it = h; it < items; it += 2) {
      const int sub = it / per_sub, c = (it - sub * per_sub) * cw;
      const int mm = sub * kBM + m;
      int leaf, y, x;
      bool valid;
      size_t pix0;
      if (a.halo == 3) {
        // Half-resolution padded rows; subtile sub is output phase
        // (py, px) = g * npt + sub, written to pixel (2y + py, 2x + px).
        const int qq = q0 + m, ph = g * a.npt + sub;
        leaf = l0;
        y = qq / a.P;
        x = qq - y * a.P;
        valid = y < a.Hout && x < a.Wout;
        pix0 = ((size_t)leaf * (2 * a.Hout) + (size_t)(2 * y + (ph >> 1))) * (size_t)(2 * a.Wout) +
               (size_t)(2 * x + (ph & 1));
      } else if (a.halo == 2) {
        // Padded row space: q = y * P + x; the pad columns and rows past the
        // map are discarded.
        const int qq = q0 + mm;
        leaf = l0;
        y = qq / a.P;
        x = qq - y * a.P;
        valid = y < a.Hout && x < a.Wout;
      } else {
        const int xx = mm % a.Wt, yy = (mm / a.Wt) % a.Ht, ll = mm / (a.Wt * a.Ht);
        leaf = l0 + ll;
        y = y0 + yy;
        x = x0 + xx;
        valid = (long)leaf * a.HWo + (long)y * a.Wout + x < a.M;
      }
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * a.mt * a.BN + sub * a.BN + c);
      if (a.halo != 3) pix0 = ((size_t)leaf * Ho + (size_t)(y * reps)) * Wo + (size_t)(x * reps);
      const size_t opix = ((size_t)leaf * a.Hout + y) * a.Wout + x;  // before the x2 upsampled store
      const float ps = (a.pscale && valid) ? a.pscale[opix] : 0.0f;
      const __nv_bfloat16 *resp =
          (a.res && valid) ? (const __nv_bfloat16 *)a.res + opix * a.res_cs + a.res_co + c : nullptr;
      uint4 chunk[4];
      int cpp;
      if (cw == 32) {
        uint32_t r[32];
        tmem_ld32(trow, r);
        epi_convert16<kFp8Out, kCalib>(a, r, eb, c, amax_local, chunk, ps, resp);
        epi_convert16<kFp8Out, kCalib>(a, r + 16, eb, c + 16, amax_local, chunk + (kFp8Out ? 1 : 2), ps,
                                       resp ? resp + 16 : nullptr);
        cpp = kFp8Out ? 2 : 4;
      } else {
        uint32_t r[16];
        tmem_ld16(trow, r);
        epi_convert16<kFp8Out, kCalib>(a, r, eb, c, amax_local, chunk, ps, resp);
        cpp = kFp8Out ? 1 : 2;
      }
      if (a.stage_out == 2 && cpp == 4)
        store_bulk(s_stage + (warp - 2) * 2048, chunk, pix0, valid, lane, (uint8_t *)a.out);
      else if (a.stage_out)
        store_staged(a, s_stage + (warp - 2) * 2048, chunk, cpp, c, pix0, valid, Wo, reps, lane, kFp8Out ? 1 : 2);
      else if (valid)
        store_direct(a, chunk, cpp, c, pix0, Wo, reps, kFp8Out ? 1 : 2);
      }  // work items
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    // Bulk output copies complete before the CTA exits.
    if (a.stage_out == 2) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (a.stats && lane == 0 && warp == 2) {
      atomicAdd(&a.stats[5], (unsigned long long)epi_wait);
      atomicAdd(&a.stats[6], (unsigned long long)(clock64() - epi_t0));
      atomicAdd(&a.stats[7], (unsigned long long)i);
    }
    if (kCalib) {
#pragma unroll
      for (int o = 16; o; o >>= 1) amax_local = fmaxf(amax_local, __shfl_xor_sync(0xFFFFFFFFu, amax_local, o));
      if (lane == 0) atomicMax(a.amax, __float_as_uint(amax_local));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  if (threadIdx.x == 0 && *abort_flag) atomicOr(a.status, ST_TIMEOUT);
}

// Weight image builder: block j (btap bytes, the Cout rows of one K chunk,
// swizzled exactly as a tensor load writes them) holds the weights' K
// columns [koff(j), koff(j) + chunk), loaded with the tensor map of the
// per-block path.  Block orders: 0 (mode 0) block = tap * cchunks + chunk;
// 1 (modes 1, 2) block = 9 * chunk + tap; 2 (mode 3) the 9 skip taps of
// each skip chunk, then per U chunk the 16 (phase, 2x2 tap) blocks.
__global__ void __launch_bounds__(128) k_build_bimage(const __grid_constant__ CUtensorMap mapB, int order, int cchunks,
                                                      int Cin, int CinU, int chunk, uint32_t btap, uint8_t *out,
                                                      uint32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *buf = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar;
  __shared__ int ok;
  const int j = blockIdx.x;
  int koff;
  if (order == 0) {
    koff = (j / cchunks) * Cin + (j % cchunks) * chunk;
  } else if (order == 1 || j < 9 * cchunks) {
    koff = (j % 9) * Cin + (j / 9) * chunk;
  } else {
    const int jj = j - 9 * cchunks;
    koff = 9 * Cin + (jj % 16) * CinU + (jj / 16) * chunk;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, btap);
    tma_load_2d(&mapB, &bar, buf, koff, 0);
    volatile int never = 0;
    ok = mbar_wait(&bar, 0, &never, 1000000000ull) ? 1 : 0;
    if (!ok) {
      atomicOr(status, ST_TIMEOUT);
      mbar_wait(&bar, 0, &never, 1000000000ull);  // the copy in flight lands before the CTA exits
    }
  }
  __syncthreads();
  if (!ok) return;
  for (uint32_t i = threadIdx.x * 16u; i < btap; i += blockDim.x * 16u)
    *reinterpret_cast<uint4 *>(out + (size_t)j * btap + i) = *reinterpret_cast<const uint4 *>(buf + i);
}

// ---------------------------------------------------------------- small SIMT kernels
// First-layer input in the tensor-core layout: the FP32 8-channel x0 as
// 32-byte rows of T per pixel (16 BF16 or 32 E4M3 channels; channels 8.. are
// zero), scaled by `mul`.  The first layer then runs as an ordinary 3x3
// layer over it.
template <typename T>
__global__ void k_pack_x0(const float *__restrict__ x0, long M, T *__restrict__ out, float mul) {
  long m = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const float4 *p = reinterpret_cast<const float4 *>(x0 + m * 8);
  const float4 a = __ldg(p), b = __ldg(p + 1);
  uint4 *o = reinterpret_cast<uint4 *>(out) + m * 2;
  if constexpr (sizeof(T) == 2) {
    __nv_bfloat162 q0 = __floats2bfloat162_rn(a.x * mul, a.y * mul), q1 = __floats2bfloat162_rn(a.z * mul, a.w * mul);
    __nv_bfloat162 q2 = __floats2bfloat162_rn(b.x * mul, b.y * mul), q3 = __floats2bfloat162_rn(b.z * mul, b.w * mul);
    o[0] = make_uint4(*reinterpret_cast<uint32_t *>(&q0), *reinterpret_cast<uint32_t *>(&q1),
                      *reinterpret_cast<uint32_t *>(&q2), *reinterpret_cast<uint32_t *>(&q3));
  } else {
    __nv_fp8x4_e4m3 q0(make_float4(a.x * mul, a.y * mul, a.z * mul, a.w * mul));
    __nv_fp8x4_e4m3 q1(make_float4(b.x * mul, b.y * mul, b.z * mul, b.w * mul));
    o[0] = make_uint4(*reinterpret_cast<uint32_t *>(&q0), *reinterpret_cast<uint32_t *>(&q1), 0u, 0u);
  }
  o[1] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ float load_act(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float load_act(const __nv_fp8_e4m3 *p) { return float(*p); }

// Single-output-channel conv (3x3 or 1x1) + softplus into the map y (FP32).
template <typename T>
__global__ void k_cout1_lp(const T *__restrict__ in, int in_cs, int H, int W, int Cin, int k, const float *__restrict__ w,
                           const float *__restrict__ bias, float in_scale, long M, float *__restrict__ y) {
  long mg = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (mg >= M) return;
  int HW = H * W;
  long leaf = mg / HW;
  int r = (int)(mg % HW), oy = r / W, ox = r % W, pad = k / 2;
  float acc = 0.0f;
  for (int ky = 0; ky < k; ++ky) {
    int iy = oy + ky - pad;
    if (iy < 0 || iy >= H) continue;
    for (int kx = 0; kx < k; ++kx) {
      int ix = ox + kx - pad;
      if (ix < 0 || ix >= W) continue;
      const T *p = in + ((leaf * H + iy) * W + ix) * in_cs;
      const float *wk = w + (size_t)(ky * k + kx) * Cin;
      for (int c = 0; c < Cin; ++c) acc = fmaf(load_act(p + c), __ldg(wk + c), acc);
    }
  }
  float v = acc * in_scale + __ldg(bias);
  y[mg] = fmaxf(v, 0.0f) + log1pf(expf(-fabsf(v)));
}

// Per-tensor absolute maximum (FP8 activation scale calibration).
__global__ void k_absmax(const float *__restrict__ x, size_t n, unsigned int *__restrict__ out) {
  float m = 0.0f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  // Looked up once per process (thread-safe static initialisation).
  static const EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

struct LpLayer {
  const void *in;
  int in_cs, in_co, Hin, Win, Cin;
  void *out;
  int out_cs, out_co, ups;
  int Cout, k, stride, act;
  const void *w;  // [Cout][k*k*Cin] reduced precision, K contiguous
  const float *bias;
  // Mixture of experts in one launch (see TcArgs): experts 1.. of the
  // group; expert 0 is w / bias / head_w / head_b.
  int n_exp = 1, pos0 = 0;
  const int *exp_range = nullptr;
  const void *w_e[kMaxExperts] = {};
  const float *bias_e[kMaxExperts] = {}, *head_w_e[kMaxExperts] = {}, *head_b_e[kMaxExperts] = {};
  float acc_mul, out_mul;
  unsigned int *amax;
  const float *head_w = nullptr, *head_b = nullptr;  // fused 1x1 head (see TcArgs)
  float *head_y = nullptr;
  int dil = 1;                                         // paper-style layers (see TcArgs)
  const float *pscale = nullptr;
  const void *res = nullptr;
  int res_cs = 0, res_co = 0;
  // Phase form (operand mode 3): the layer's input is [upsample2(U), S]
  // with S = in (Cin channels, full resolution) and U = in_u (CinU channels,
  // half resolution); w is then the phase weight layout (see make_phase_weights).
  const void *in_u = nullptr;
  int u_cs = 0, u_co = 0, CinU = 0;
  // The nets' layers (expert e; 0: this net) and the contexts that own the
  // nets, which hold and are charged for the weight images.
  Layer *own[kMaxExperts] = {};
  pg_ctx *own_ctx[kMaxExperts] = {};
};

// Launch shape: CTAs resident per SM and pipeline stages per CTA.  Zero
// fields select the built-in heuristic.
struct TcCfg {
  int ctas = 0, stages = 0, mt = 0, halo = 0, cb = 0, so = 0;
};

constexpr size_t kSmemPerSM = 228 * 1024;

// CTAs per SM that the register file holds (65,536 registers per SM).
int ctas_by_registers() {
  static const int n = [] {
    int regs = 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_conv_tc<false, false>) == cudaSuccess) regs = std::max(regs, fa.numRegs);
    if (cudaFuncGetAttributes(&fa, k_conv_tc<false, true>) == cudaSuccess) regs = std::max(regs, fa.numRegs);
    if (cudaFuncGetAttributes(&fa, k_conv_tc<true, false>) == cudaSuccess) regs = std::max(regs, fa.numRegs);
    cudaGetLastError();
    regs = (std::max(regs, 1) + 7) & ~7;
    return std::max(1, 65536 / (regs * kThreads));
  }();
  return n;
}

// Guards the nets' weight-image caches (a lock of its own: the E4M3
// calibration pass runs under the net-state lock).
std::mutex &bimg_mutex() {
  static std::mutex mu;
  return mu;
}

// The weight image of a layer's weights w (element size es) in block order
// `order` with chunks of cb bytes (see k_build_bimage), built on first use
// on stream st and cached in the layer; held outside the stream-ordered
// pool and charged to the context owning the net.  Returns null (the per-block tensor loads then serve) while st is
// being captured into a graph or when the image cannot be allocated.
const uint8_t *get_bimage(Layer *Lw, pg_ctx *owner, const void *w, int es, int order, int cb, int Cout, int K,
                          int nblk, int cchunks, int Cin, int CinU, cudaStream_t st, uint32_t *status) {
  if (!Lw || !owner || !w) return nullptr;
  const int ei = es == 1 ? 1 : 0, ci = cb == 128 ? 0 : (cb == 64 ? 1 : 2);
  std::lock_guard<std::mutex> lock(bimg_mutex());
  if (Lw->bimg[ei][order][ci]) return (const uint8_t *)Lw->bimg[ei][order][ci];
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  EncodeTiledFn enc = encode_fn();
  if (!enc) return nullptr;
  const int chunk = cb / es;
  const uint32_t btap = (uint32_t)(Cout * cb);
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)Cout};
  cuuint64_t strides[1] = {(cuuint64_t)K * es};
  cuuint32_t box[2] = {(cuuint32_t)chunk, (cuuint32_t)Cout};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw =
      cb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (cb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  if (enc(&map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(w),
          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return nullptr;
  const size_t bytes = (size_t)nblk * btap;
  void *p = nullptr;
  if (ctx_alloc_static(owner, bytes, &p) != PG_OK) return nullptr;
  k_build_bimage<<<nblk, 128, btap + 1024, st>>>(map, order, cchunks, Cin, CinU, chunk, btap, (uint8_t *)p, status);
  // Other streams may use the image as soon as it is cached.
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    ctx_free_static(owner, p, bytes);
    return nullptr;
  }
  Lw->bimg[ei][order][ci] = p;
  Lw->bimg_bytes[ei][order][ci] = bytes;
  if (getenv("PG_TC_LOG"))
    fprintf(stderr, "pg: weight image of %d blocks (order %d, %d-byte chunks): %zu bytes\n", nblk, order, cb, bytes);
  return (const uint8_t *)p;
}

pg_status launch_tc(const LpLayer &L, uint32_t ns, int es, bool fp8_out, cudaStream_t st, uint32_t *status,
                    TcCfg cfg = TcCfg()) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return PG_ERR_UNSUPPORTED;
  const int Hout = L.Hin / L.stride, Wout = L.Win / L.stride, HWo = Hout * Wout;
  const long M = (long)ns * HWo;
  if (M == 0) return PG_OK;
  if (L.Cout % 16 || L.Cout < 16 || L.Cout > 256) return PG_ERR_UNSUPPORTED;
  // K chunk per stage: one swizzle row of 128, 64 or 32 bytes.
  int cb = 0;
  for (int c : {128, 64, 32})
    if ((L.Cin * es) % c == 0 && (cfg.cb == 0 || cfg.cb == c)) {
      cb = c;
      break;
    }
  if (!cb) return PG_ERR_UNSUPPORTED;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.k = L.k;
  a.stride = L.stride;
  a.dil = L.dil > 1 ? L.dil : 1;
  a.pad = a.dil * (L.k / 2);
  a.Cin = L.Cin;
  a.chunk = cb / es;
  a.cchunks = L.Cin / a.chunk;
  a.Hout = Hout;
  a.Wout = Wout;
  a.HWo = HWo;
  a.M = M;
  a.BN = L.Cout;
  a.mt = cfg.mt > 0 ? cfg.mt : 1;
  if (cfg.halo < 2 && a.mt > 2) return PG_ERR_UNSUPPORTED;  // up to 4 subtiles: the padded-row modes only
  if (a.mt != 1 && a.mt != 2 && a.mt != 4) return PG_ERR_UNSUPPORTED;
  const int TP = kBM * a.mt;  // pixels per CTA tile
  if (Wout >= TP) {
    a.Wt = TP; a.Ht = 1; a.Lt = 1;
  } else if (HWo >= TP) {
    a.Wt = Wout; a.Ht = TP / Wout; a.Lt = 1;
  } else {
    a.Wt = Wout; a.Ht = Hout; a.Lt = TP / HWo;
  }
  if (a.Wt * a.Ht * a.Lt != TP || a.Wt * L.stride > 256 || a.Ht * L.stride > 256 || a.Lt > 256)
    return PG_ERR_UNSUPPORTED;
  a.num_tiles = (int)((M + TP - 1) / TP);
  a.halo = cfg.halo;
  if (a.dil > 1 && a.halo) return PG_ERR_UNSUPPORTED;  // haloed operand modes assume adjacent taps
  if ((L.pscale || L.res) && fp8_out) return PG_ERR_UNSUPPORTED;  // paper-style layers run in BF16
  if (a.halo == 1 && (L.k != 3 || L.stride != 1 || a.Lt != 1 || a.Ht + 2 > 256)) return PG_ERR_UNSUPPORTED;
  a.chunk_bytes = cb;
  a.kiters = a.halo ? a.cchunks : L.k * L.k * a.cchunks;
  a.bytes_ver = (uint32_t)((a.Ht + 2) * a.Wt * cb);
  a.bytes_a = a.halo ? 3u * a.bytes_ver : (uint32_t)(TP * cb);
  a.bytes_b = (uint32_t)(L.Cout * cb) * (a.halo ? 9u : 1u);
  a.tx_bytes = a.bytes_a + a.bytes_b;
  if (a.halo == 2) {
    // One box of Hb padded rows per channel chunk: the tile's TP rows start
    // anywhere in their first image row, and the taps read up to 2P + 2 rows
    // further, so Hb = ceil((TP + 1) / P) + 3 image rows always cover them.
    if (L.k != 3 || L.stride != 1 || HWo < TP || Wout + 2 > 256) return PG_ERR_UNSUPPORTED;
    a.P = Wout + 2;
    a.Hb = (TP + a.P) / a.P + 3;
    if (a.Hb > 256) return PG_ERR_UNSUPPORTED;
    a.tpl = (Hout * a.P + TP - 1) / TP;
    a.num_tiles = (int)ns * a.tpl;
    // Exact for every position index below 2^16 and pitches up to 258
    // (checked exhaustively on the host).
    a.p_magic = (long)a.tpl * TP <= 65536 ? (uint32_t)((1ull << 32) / (uint64_t)a.P + 1ull) : 0u;
    const uint32_t box = (uint32_t)(a.Hb * a.P * cb);
    a.bytes_a = (box + 1023u) & ~1023u;
    a.tx_bytes = box + a.bytes_b;
  }
  if (a.halo == 3) {
    // Phase form of a decoder layer: the tile grid is U's half-resolution
    // map in padded rows (as mode 2), one subtile per output phase.  Each
    // box holds Hb rows of P positions: Hb = ceil((128 + 1) / P) + 3 rows
    // cover the tile and every tap's row and column offset of -1..1.
    if (!L.in_u || es != 2 || fp8_out || L.k != 3 || L.stride != 1 || a.dil != 1 || L.pscale || L.res || L.head_y ||
        L.ups || (L.Hin & 1) || (L.Win & 1) || L.CinU <= 0 || (L.CinU * es) % cb)
      return PG_ERR_UNSUPPORTED;
    if (cfg.mt <= 0) a.mt = L.Cout <= 64 ? 4 : (L.Cout <= 128 ? 2 : 1);  // all phases whose accumulators fit
    if (a.mt != 1 && a.mt != 2 && a.mt != 4) return PG_ERR_UNSUPPORTED;
    a.npt = a.mt;
    a.Hout = L.Hin / 2;
    a.Wout = L.Win / 2;
    a.HWo = a.Hout * a.Wout;
    a.P = a.Wout + 2;
    a.Hb = (kBM + a.P) / a.P + 3;
    if (2 * a.P > 256 || 2 * a.Hb > 256) return PG_ERR_UNSUPPORTED;
    a.tpl = (a.Hout * a.P + kBM - 1) / kBM;
    a.num_tiles = (int)ns * (4 / a.npt) * a.tpl;
    a.p_magic = (long)a.tpl * kBM <= 65536 ? (uint32_t)((1ull << 32) / (uint64_t)a.P + 1ull) : 0u;
    a.CinU = L.CinU;
    a.kS = a.cchunks;
    a.kU = L.CinU / a.chunk;
    a.kiters = a.kS + a.kU;
    const uint32_t box = (uint32_t)(a.Hb * a.P * cb);
    a.box_a = (box + 1023u) & ~1023u;
    a.bytes_a = 4u * a.box_a;
    a.btap = (uint32_t)(L.Cout * cb);
    a.bytes_b = a.btap * (uint32_t)std::max(9, 4 * a.npt);
    a.tx_bytes = 4u * box + 9u * a.btap;
    a.tx_u = box + 4u * (uint32_t)a.npt * a.btap;
  }
  if (a.halo == 4) {
    // Stride-2 3x3 layer over 32 dense BF16 channels, read as pixel pairs
    // (issue_stage4): six stages per tile -- kernel row ky, pairs at x - 1
    // then pairs at x -- each one box of TP rows of 128 bytes plus the weight
    // blocks of one tap or two.
    if (L.k != 3 || L.stride != 2 || es != 2 || cb != 64 || L.Cin != 32 || L.in_cs != 32 || L.in_co != 0 ||
        (L.Win & 1) || (L.Hin & 1) || L.pscale || L.res || L.in_u || 2 * a.Ht > 256)
      return PG_ERR_UNSUPPORTED;
    a.kiters = 6;
    a.bytes_a = (uint32_t)TP * 128u;
    a.bytes_b = 2u * (uint32_t)(L.Cout * cb);
    a.tx_bytes = a.bytes_a + a.bytes_b;
    a.tx_u = a.bytes_a + (uint32_t)(L.Cout * cb);
  }
  a.btap = (uint32_t)(L.Cout * cb);
  a.sbo = 8u * (uint32_t)cb;
  a.swz = cb == 128 ? 2 : (cb == 64 ? 4 : 6);
  a.sbo_b = a.sbo;
  a.swz_b = a.swz;
  if (a.halo == 4) {  // A rows of 128 bytes (128-byte swizzle); B keeps the taps' 64-byte rows
    a.sbo = 8u * 128u;
    a.swz = 2;
  }
  a.mma_per_stage = cb / 32;
  a.mma_kind = es == 1 ? 1 : 0;
  // Instruction descriptor: D = F32, A/B = BF16 (kind::f16) or E4M3
  // (kind::f8f6f4), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
  a.idesc = (1u << 4) | ((es == 2 ? 1u : 0u) << 7) | ((es == 2 ? 1u : 0u) << 10) | ((uint32_t)(L.Cout >> 3) << 17) |
            ((uint32_t)(kBM >> 4) << 24);
  uint32_t cols = 32;
  while (cols < 2u * (uint32_t)(a.mt * L.Cout)) cols <<= 1;
  if (cols > 512) return PG_ERR_UNSUPPORTED;
  a.tmem_cols = cols;
  // CTAs per SM: TMEM holds 512 columns per SM, and shared memory is sized
  // so that no more CTAs than that can be resident (a CTA that found no free
  // TMEM columns would wait inside tcgen05.alloc).
  const int max_ctas = std::min((int)std::min<uint32_t>(4, 512u / cols), ctas_by_registers());
  int per_sm = cfg.ctas > 0 ? std::min(cfg.ctas, max_ctas) : std::min(2, max_ctas);
  const size_t stage_bytes = a.bytes_a + a.bytes_b;
  a.stage_out = (cfg.so && !L.head_y) ? 1 : 0;
  // Bulk stores: padded-row tiles of a dense 32-channel BF16 output, with
  // work items of all 32 columns (two or more subtiles); other layers asked
  // for them take the staged stores.
  if (cfg.so == 2 && a.halo == 2 && a.mt >= 2 && es == 2 && !fp8_out && L.Cout == 32 && L.out_cs == 32 &&
      L.out_co == 0 && !L.ups && !L.head_y && !L.pscale && !L.res && !L.amax)
    a.stage_out = 2;
  // align, barriers, per-expert bias + head and ranges, staging, reserve
  const size_t head_n = L.head_y ? (size_t)L.Cout + 4 : 0;
  const size_t bias_head = 4 * (size_t)L.n_exp * ((size_t)L.Cout + head_n) + 4 * (L.n_exp + 1) + 16;
  size_t stage_smem = 0;
  int max_stages = 0;
  for (;;) {
    stage_smem = a.stage_out ? (size_t)kEpiWarps * 2048 : 0;
    const size_t fixed = 1024 + 8 * 5 + 16 + bias_head + 32 + stage_smem + 1024;
    const size_t cap = kSmemPerSM / per_sm - 1024;
    max_stages = cap > fixed ? (int)std::min<size_t>(24, (cap - fixed) / (stage_bytes + 16)) : 0;
    if (max_stages >= 2) break;
    // A shape tuned for one net may not fit beside several experts' bias
    // and head tables: give up the staged stores, then a resident CTA.
    if (L.n_exp > 1 && a.stage_out) {
      a.stage_out = 0;
    } else if (L.n_exp > 1 && per_sm > 1) {
      --per_sm;
    } else {
      return PG_ERR_UNSUPPORTED;
    }
  }
  a.stages = cfg.stages > 0 ? std::min(cfg.stages, max_stages) : std::min(8, max_stages);
  size_t smem = 1024 + a.stages * stage_bytes + 8 * (2 * a.stages + 5) + 16 + bias_head + 16 + stage_smem;
  smem = std::max(smem, kSmemPerSM / (per_sm + 1) + 1024);  // at most per_sm CTAs resident
  a.out = L.out;
  a.out_cs = L.out_cs;
  a.out_co = L.out_co;
  a.ups = L.ups;
  a.act = L.act;
  a.out_fp8 = fp8_out ? 1 : 0;
  a.out_mul = L.out_mul;
  a.acc_mul = L.acc_mul;
  a.n_exp = L.n_exp;
  a.pos0 = L.pos0;
  a.exp_range = L.exp_range;
  if (L.n_exp < 1 || L.n_exp > kMaxExperts || (L.n_exp > 1 && !L.exp_range)) return PG_ERR_UNSUPPORTED;
  for (int e = 0; e < L.n_exp; ++e) a.bias[e] = e ? L.bias_e[e] : L.bias;
  a.status = status;
  a.amax = L.amax;
  for (int e = 0; e < L.n_exp; ++e) {
    a.head_w[e] = e ? L.head_w_e[e] : L.head_w;
    a.head_b[e] = e ? L.head_b_e[e] : L.head_b;
  }
  a.head_y = L.head_y;
  a.pscale = L.pscale;
  a.res = L.res;
  a.res_cs = L.res_cs;
  a.res_co = L.res_co;
  if (a.head_y && (L.ups || L.Cout % 16)) return PG_ERR_UNSUPPORTED;
  a.stats = nullptr;
  static unsigned long long *d_stats = nullptr;
  const bool want_stats = getenv("PG_TC_STATS") != nullptr;
  if (want_stats) {
    if (!d_stats) PG_CUDA(cudaMalloc(&d_stats, 8 * sizeof(unsigned long long)));
    PG_CUDA(cudaMemsetAsync(d_stats, 0, 8 * sizeof(unsigned long long), st));
    a.stats = d_stats;
  }

  const CUtensorMapDataType dt = es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const CUtensorMapSwizzle sw =
      cb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (cb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  CUtensorMap mA;
  TcMapsB mB;
  memset(&mB, 0, sizeof(mB));
  {
    cuuint64_t dims[4] = {(cuuint64_t)L.Cin, (cuuint64_t)L.Win, (cuuint64_t)L.Hin, (cuuint64_t)ns};
    cuuint64_t strides[3] = {(cuuint64_t)L.in_cs * es, (cuuint64_t)L.Win * L.in_cs * es,
                             (cuuint64_t)L.Hin * L.Win * L.in_cs * es};
    cuuint32_t box[4] = {(cuuint32_t)a.chunk, (cuuint32_t)(a.Wt * L.stride),
                         (cuuint32_t)(a.halo ? a.Ht + 2 : a.Ht * L.stride), (cuuint32_t)a.Lt};
    if (a.halo == 2) {
      box[1] = (cuuint32_t)a.P;
      box[2] = (cuuint32_t)a.Hb;
      box[3] = 1;
    }
    cuuint32_t estr[4] = {1, (cuuint32_t)L.stride, (cuuint32_t)L.stride, 1};
    if (a.halo == 3) {
      // One parity sub-grid: every second column and row of the skip input.
      box[1] = (cuuint32_t)(2 * a.P);
      box[2] = (cuuint32_t)(2 * a.Hb);
      box[3] = 1;
      estr[1] = estr[2] = 2;
    }
    CUtensorMapSwizzle swA = sw;
    if (a.halo == 4) {
      // Pixel pairs: 64 channels (two pixels of 32) per 128-byte row, every
      // second image row; the leaf and pair index carry the zero padding.
      dims[0] = 64;
      dims[1] = (cuuint64_t)(L.Win / 2);
      strides[0] = 128;
      box[0] = 64;
      box[1] = (cuuint32_t)a.Wt;
      box[2] = (cuuint32_t)(2 * a.Ht);
      box[3] = (cuuint32_t)a.Lt;
      estr[1] = 1;
      estr[2] = 2;
      swA = CU_TENSOR_MAP_SWIZZLE_128B;
    }
    void *base = (uint8_t *)L.in + (size_t)L.in_co * es;
    if (enc(&mA, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swA,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PG_ERR_UNSUPPORTED;
  }
  CUtensorMap mU;
  memset(&mU, 0, sizeof(mU));
  if (a.halo == 3) {
    const int Hu = L.Hin / 2, Wu = L.Win / 2;
    cuuint64_t dims[4] = {(cuuint64_t)L.CinU, (cuuint64_t)Wu, (cuuint64_t)Hu, (cuuint64_t)ns};
    cuuint64_t strides[3] = {(cuuint64_t)L.u_cs * es, (cuuint64_t)Wu * L.u_cs * es, (cuuint64_t)Hu * Wu * L.u_cs * es};
    cuuint32_t box[4] = {(cuuint32_t)a.chunk, (cuuint32_t)a.P, (cuuint32_t)a.Hb, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    void *base = (uint8_t *)L.in_u + (size_t)L.u_co * es;
    if (enc(&mU, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PG_ERR_UNSUPPORTED;
  }
  {
    const int K = a.halo == 3 ? 9 * L.Cin + 16 * L.CinU : L.k * L.k * L.Cin;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)L.Cout};
    cuuint64_t strides[1] = {(cuuint64_t)K * es};
    cuuint32_t box[2] = {(cuuint32_t)a.chunk, (cuuint32_t)L.Cout};
    cuuint32_t estr[2] = {1, 1};
    for (int e = 0; e < L.n_exp; ++e) {
      const void *w = e ? L.w_e[e] : L.w;
      if (!w || enc(&mB.b[e], dt, 2, const_cast<void *>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return PG_ERR_UNSUPPORTED;
    }
  }
  if (smem > 227 * 1024) return PG_ERR_UNSUPPORTED;
  // Weight images: one bulk copy per stage instead of one tensor load per
  // weight block (all experts or none).
  {
    const int order = a.halo == 3 ? 2 : ((a.halo == 1 || a.halo == 2) ? 1 : 0);
    const int K = a.halo == 3 ? 9 * L.Cin + 16 * L.CinU : L.k * L.k * L.Cin;
    const int nblk = a.halo == 3 ? 9 * a.kS + 16 * a.kU : (a.halo ? 9 * a.cchunks : L.k * L.k * a.cchunks);
    bool all = !getenv("PG_TC_NO_IMAGE");
    for (int e = 0; e < L.n_exp && all; ++e) {
      a.bimg[e] = get_bimage(L.own[e], L.own_ctx[e], e ? L.w_e[e] : L.w, es, order, cb, L.Cout, K, nblk,
                             a.halo == 3 ? a.kS : a.cchunks, L.Cin, L.CinU, st, status);
      all = a.bimg[e] != nullptr;
    }
    if (!all)
      for (int e = 0; e < kMaxExperts; ++e) a.bimg[e] = nullptr;
  }
  const int grid = std::min(a.num_tiles, per_sm * num_sms());
  if (fp8_out) {
    PG_CUDA(cudaFuncSetAttribute(k_conv_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k_conv_tc<true, false><<<grid, kThreads, smem, st>>>(mA, mU, mB, a);
  } else if (a.amax) {
    PG_CUDA(cudaFuncSetAttribute(k_conv_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k_conv_tc<false, true><<<grid, kThreads, smem, st>>>(mA, mU, mB, a);
  } else {
    PG_CUDA(cudaFuncSetAttribute(k_conv_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k_conv_tc<false, false><<<grid, kThreads, smem, st>>>(mA, mU, mB, a);
  }
  if (want_stats) {
    unsigned long long h[8];
    PG_CUDA(cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
    PG_CUDA(cudaStreamSynchronize(st));
    const double g = (double)grid;
    fprintf(stderr,
            "pg_tc_stats: %dx%d cin %d cout %d halo %d cb %d mt %d ctas %d stages %d tiles %d | per CTA kcycles: "
            "producer wait %.0f / %.0f, mma wait acc %.0f full %.0f / %.0f, epilogue wait %.0f / %.0f (tiles %.0f)\n",
            L.Hin, L.Win, L.Cin, L.Cout, a.halo, cb, a.mt, per_sm, a.stages, a.num_tiles, h[0] / g / 1e3,
            h[1] / g / 1e3, h[2] / g / 1e3, h[3] / g / 1e3, h[4] / g / 1e3, h[5] / g / 1e3, h[6] / g / 1e3, h[7] / g);
  }
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace

// Reduced-precision weight copies: [Cout][k*k*Cin] (K contiguous); the first
// layer's input channels are padded to the 32-byte rows of k_pack_x0 (16
// BF16 or 32 E4M3 channels, zero weights past the net's own).  FP8 weights
// carry one per-tensor scale (amax / 448).
static pg_status make_lp_weights(pg_ctx *ctx, Layer &L, bool first, pg_precision prec) {
  const int taps = L.k * L.k;
  const size_t Kf = (size_t)taps * L.cin;  // rows of the FP32 [K][Cout] copy
  std::vector<float> wf(Kf * L.cout);
  PG_CUDA(cudaMemcpyAsync(wf.data(), L.w, wf.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  PG_CUDA(cudaStreamSynchronize(ctx->stream));
  const int cp = first ? (prec == PG_FP8_E4M3 ? 32 : 16) : L.cin;
  const size_t K = (size_t)taps * cp;
  std::vector<float> wt((size_t)L.cout * K, 0.0f);
  for (int o = 0; o < L.cout; ++o)
    for (int tap = 0; tap < taps; ++tap)
      for (int c = 0; c < L.cin; ++c) wt[(size_t)o * K + (size_t)tap * cp + c] = wf[((size_t)tap * L.cin + c) * L.cout + o];
  const int es = prec == PG_FP8_E4M3 ? 1 : 2;
  std::vector<uint8_t> host(wt.size() * es);
  float scale = 1.0f;
  if (es == 2) {
    for (size_t i = 0; i < wt.size(); ++i) {
      __nv_bfloat16 b = __float2bfloat16_rn(wt[i]);
      memcpy(&host[2 * i], &b, 2);
    }
  } else {
    float amax = 0.0f;
    for (float v : wt) amax = std::max(amax, fabsf(v));
    scale = amax > 0.0f ? amax / 448.0f : 1.0f;
    for (size_t i = 0; i < wt.size(); ++i) {
      __nv_fp8_e4m3 q(wt[i] / scale);
      memcpy(&host[i], &q, 1);
    }
  }
  void *p;
  PG_TRY(ctx_alloc(ctx, host.size(), &p));
  PG_CUDA(cudaMemcpyAsync(p, host.data(), host.size(), cudaMemcpyHostToDevice, ctx->stream));
  PG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (es == 2) {
    L.w_bf16 = p;
    L.w_bf16_bytes = host.size();
  } else {
    L.w_fp8 = p;
    L.w_fp8_bytes = host.size();
    L.w_scale = scale;
  }
  return PG_OK;
}

// Phase-form weights of a decoder layer whose input is the concatenation
// [upsample2(U) (Cu channels), S (Cs channels)], nearest-neighbour x2.  The
// 3x3 tap (ky, kx) of output pixel (2y + py, 2x + px) falls on upsampled
// pixel row 2y + py + ky - 1, i.e. U row y + floor((py + ky - 1) / 2): for
// py = 0 the taps ky = 0 | 1, 2 land on U rows y - 1 | y, for py = 1 the
// taps ky = 0, 1 | 2 on U rows y | y + 1 (columns likewise).  So each of the
// four output phases convolves U with a 2x2 kernel whose taps sum the 3x3
// taps landing on the same U pixel (the zero padding agrees: upsampled row
// -1 or 2H is U row -1 or H), and S keeps its 3x3 taps.  Layout, K
// contiguous: [cout][9 Cs (tap, channel) | 16 Cu (phase, 2x2 tap, channel)],
// the sums taken in double and rounded to BF16 once.
static pg_status make_phase_weights(pg_ctx *ctx, Layer &L, int Cu) {
  const int Cs = L.cin - Cu;
  if (L.k != 3 || L.stride != 1 || Cu <= 0 || Cs <= 0) return PG_ERR_UNSUPPORTED;
  std::vector<float> wf((size_t)9 * L.cin * L.cout);
  PG_CUDA(cudaMemcpyAsync(wf.data(), L.w, wf.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  PG_CUDA(cudaStreamSynchronize(ctx->stream));
  const size_t K = (size_t)9 * Cs + (size_t)16 * Cu;
  std::vector<double> wt((size_t)L.cout * K, 0.0);
  auto w_at = [&](int tap, int c, int o) { return (double)wf[((size_t)tap * L.cin + c) * L.cout + o]; };
  for (int o = 0; o < L.cout; ++o) {
    double *row = &wt[(size_t)o * K];
    for (int tap = 0; tap < 9; ++tap)
      for (int c = 0; c < Cs; ++c) row[(size_t)tap * Cs + c] = w_at(tap, Cu + c, o);
    for (int ph = 0; ph < 4; ++ph) {
      const int py = ph >> 1, px = ph & 1;
      for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
          const int i = ((py + ky + 1) >> 1) - py, j = ((px + kx + 1) >> 1) - px;  // U row / column offset + 1 - py
          double *dst = row + (size_t)9 * Cs + (size_t)(ph * 4 + i * 2 + j) * Cu;
          for (int c = 0; c < Cu; ++c) dst[c] += w_at(ky * 3 + kx, c, o);
        }
    }
  }
  std::vector<__nv_bfloat16> host(wt.size());
  for (size_t i = 0; i < wt.size(); ++i) host[i] = __float2bfloat16_rn((float)wt[i]);
  void *p;
  PG_TRY(ctx_alloc(ctx, host.size() * 2, &p));
  PG_CUDA(cudaMemcpyAsync(p, host.data(), host.size() * 2, cudaMemcpyHostToDevice, ctx->stream));
  PG_CUDA(cudaStreamSynchronize(ctx->stream));
  L.w_ph_bf16 = p;
  L.w_ph_bytes = host.size() * 2;
  return PG_OK;
}

// Serialises the one-time state changes of a net (reduced-precision weight
// copies, FP8 activation calibration) between threads that share it.
std::mutex &net_state_mutex() {
  static std::mutex mu;
  return mu;
}

pg_status tc_prepare(pg_ctx *ctx, Net *net, pg_precision prec) {
  if (!encode_fn()) return PG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(net_state_mutex());
  // Weight copies belong to the net, so they are charged to the context that
  // owns it (the one that frees them), whichever context runs the first call.
  ctx = net->h.ctx;
  for (int l = 0; l < net->n_layers; ++l) {
    Layer &L = net->layers[l];
    // FP8 runs are calibrated by one BF16 pass, so they need both copies.
    if (!L.w_bf16) PG_TRY(make_lp_weights(ctx, L, l == 0, PG_BF16));
    // The U-Net's decoder layers over [upsample2(U), S] (layers 8, 10, 12):
    // U is the previous layer's c3, c2 or c1 channels.
    if (net->arch == 1 && (l == 8 || l == 10 || l == 12) && !L.w_ph_bf16)
      PG_TRY(make_phase_weights(ctx, L, net->widths[(14 - l) / 2]));
    if ((prec == PG_FP8_E4M3 || prec == PG_FP8_MIXED) && !L.w_fp8) PG_TRY(make_lp_weights(ctx, L, l == 0, PG_FP8_E4M3));
  }
  return PG_OK;
}

namespace {

// FP8 activation groups: every tensor a layer reads has one per-tensor scale,
// so layers that write into the same buffer instance (the two halves of a
// U-Net concatenation) share a group.  out_group[l] / in_group[l]; group 0 is
// the network input (the packed first-layer input).
const int kUnetOut[15] = {1, 2, 3, 4, 5, 6, 7, 6, 8, 4, 9, 2, 10, 11, -1};
const int kUnetIn[15] = {0, 1, 2, 3, 4, 5, 6, 7, 6, 8, 4, 9, 2, 10, 11};
const int kTinyOut[3] = {1, 2, -1};
const int kTinyIn[3] = {0, 1, 2};

// Times every feasible launch shape of one layer on its real operands
// (CUDA events on the launching stream) and returns the fastest.  The layer
// is left computed (every candidate writes the same output).
pg_status tune_layer(const LpLayer &L, uint32_t ns, int es, bool fp8, cudaStream_t st, uint32_t *status,
                     TcCfg *best, float *best_ms_out) {
  cudaEvent_t e0, e1;
  PG_CUDA(cudaEventCreate(&e0));
  PG_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  pg_status last_err = PG_ERR_UNSUPPORTED;
  *best = TcCfg();
  // The phase form (operand mode 3) is the only mode of its layers, with
  // one to four output phases per tile.
  const std::vector<int> halos = L.in_u ? std::vector<int>{3} : std::vector<int>{0, 1, 2, 4};
  for (int so : {0, 1, 2})
  for (int halo : halos)
  for (int cb : {128, 64, 32})
  for (int mt : {1, 2, 4})
  for (int ctas : {1, 2, 3, 4})
    for (int stages : {2, 3, 4, 6, 8, 12, 16}) {
      if (halo && stages > 6) continue;
      if (mt == 4 && halo < 2) continue;  // four subtiles: the padded-row modes only
      // Bulk stores serve padded-row layers with dense 32-channel BF16
      // outputs; elsewhere they would repeat the staged candidate.
      if (so == 2 && !(halo == 2 && mt >= 2 && es == 2 && !fp8 && L.Cout == 32 && L.out_cs == 32 && L.out_co == 0 &&
                       !L.ups && !L.head_y && !L.pscale && !L.res && !L.amax))
        continue;
      if (!halo && cb != 128 && stages < 3) continue;
      TcCfg c;
      c.ctas = ctas;
      c.stages = stages;
      c.mt = mt;
      c.halo = halo;
      c.cb = cb;
      c.so = so;
      const pg_status w = launch_tc(L, ns, es, fp8, st, status, c);  // warm-up / feasibility
      if (w != PG_OK) {
        if (w != PG_ERR_UNSUPPORTED) last_err = w;
        continue;
      }
      cudaEventRecord(e0, st);
      pg_status s = launch_tc(L, ns, es, fp8, st, status, c);
      cudaEventRecord(e1, st);
      if (s != PG_OK) continue;
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        *best = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PG_CUDA(cudaGetLastError());
  *best_ms_out = best_ms;
  return best->ctas ? PG_OK : last_err;
}

template <typename T>
pg_status forward_lp(pg_ctx *ctx, const Net *netc, bool fp8, const float *x0, void *actv, uint32_t ns, int H, int W,
                     float *y, cudaStream_t st, const float *scale, unsigned int *amax, bool tune = false,
                     bool mixed = false, const Net *const *experts = nullptr, int n_exp = 1,
                     const int *exp_range = nullptr, int pos0 = 0) {
  Net *net = const_cast<Net *>(netc);
  // Mixture of experts in one launch per layer (BF16 U-Net only): experts[0]
  // is net; the others share its layer shapes and launch shapes.
  if (n_exp > 1 && (fp8 || mixed || scale || amax || tune || net->arch != 1 || n_exp > kMaxExperts)) return PG_ERR_UNSUPPORTED;
  // Mixed form (U-Net only): E4M3 operands inside the network (layers 3-11
  // read E4M3, layers 2-10 write it); the full-resolution level, its skip
  // concatenation and the head stay BF16.
  if (mixed && (net->arch != 1 || fp8 || !scale)) return PG_ERR_UNSUPPORTED;
  auto in8_of = [&](int li) { return mixed ? (li >= 3 && li <= 11) : fp8; };
  auto out8_of = [&](int li) { return mixed ? (li >= 2 && li <= 10) : fp8; };
  const int es = sizeof(T);
  const size_t HW = (size_t)H * W;
  const long M0 = (long)ns * HW;
  const Layer *Ls = net->layers;
  const int *og = net->arch == 0 ? kTinyOut : kUnetOut;
  const int *ig = net->arch == 0 ? kTinyIn : kUnetIn;
  uint8_t *act = (uint8_t *)actv;
  const int cp = 32 / es;  // first-layer channels per pixel (32-byte rows)
  T *xcol = (T *)act;
  act += align256(M0 * 32);
  if (x0) {  // null: the caller assembled the packed input into xcol already
    k_pack_x0<T><<<ceil_div(M0, 256), 256, 0, st>>>(x0, M0, xcol, fp8 ? 1.0f / scale[0] : 1.0f);
    PG_COUNT(ctx);
    PG_CUDA(cudaGetLastError());
  }
  auto conv = [&](int li, const void *in, int in_cs, int in_co, int Hin, int Win, int Cin, void *out, int out_cs,
                  int out_co, int ups, const Layer *head = nullptr, const float *pscale = nullptr,
                  const void *res = nullptr, int res_cs = 0, int res_co = 0, const void *in_u = nullptr,
                  int u_cs = 0, int CinU = 0) -> pg_status {
    const Layer &Lr = Ls[li];
    const bool phase = in_u != nullptr;  // operand mode 3 over [upsample2(in_u), in]
    LpLayer L;
    L.own[0] = &net->layers[li];
    L.own_ctx[0] = net->h.ctx;
    if (phase) {
      L.in_u = in_u;
      L.u_cs = u_cs;
      L.CinU = CinU;
    }
    if (head) {
      L.head_w = head->w;
      L.head_b = head->b;
      L.head_y = y;
    }
    L.dil = Lr.dil;
    L.pscale = pscale;
    L.res = res;
    L.res_cs = res_cs;
    L.res_co = res_co;
    L.in = in; L.in_cs = in_cs; L.in_co = in_co; L.Hin = Hin; L.Win = Win; L.Cin = Cin;
    L.out = out; L.out_cs = out_cs; L.out_co = out_co; L.ups = ups;
    L.Cout = Lr.cout; L.k = Lr.k; L.stride = Lr.stride; L.act = Lr.act;
    L.bias = Lr.b;
    if (n_exp > 1) {
      L.n_exp = n_exp;
      L.exp_range = exp_range;
      L.pos0 = pos0;
      for (int e = 1; e < n_exp; ++e) {
        const Layer &Le = experts[e]->layers[li];
        if (!Le.w_bf16 || Le.cout != Lr.cout || Le.cin != Lr.cin || Le.k != Lr.k || Le.stride != Lr.stride ||
            (phase && !Le.w_ph_bf16))
          return PG_ERR_UNSUPPORTED;
        L.w_e[e] = phase ? Le.w_ph_bf16 : Le.w_bf16;
        L.own[e] = const_cast<Layer *>(&Le);
        L.own_ctx[e] = experts[e]->h.ctx;
        L.bias_e[e] = Le.b;
        if (head) {
          L.head_w_e[e] = experts[e]->layers[14].w;
          L.head_b_e[e] = experts[e]->layers[14].b;
        }
      }
    }
    L.amax = amax ? amax + og[li] : nullptr;
    const bool in8 = in8_of(li), out8 = out8_of(li);
    const int pi = in8 ? 2 : 1;  // tuned shapes are kept per operand type
    const int les = in8 ? 1 : 2;
    if (in8) {
      L.w = Lr.w_fp8;
      L.acc_mul = scale[ig[li]] * Lr.w_scale;
    } else {
      L.w = phase ? Lr.w_ph_bf16 : Lr.w_bf16;
      L.acc_mul = 1.0f;
    }
    L.out_mul = out8 ? 1.0f / scale[og[li]] : 1.0f;
    Layer &Lw = net->layers[li];
    if (tune) {
      TcCfg best;
      float best_ms = 0;
      PG_TRY(tune_layer(L, ns, les, out8, st, ctx->d_status, &best, &best_ms));
      Lw.tc_ctas[pi] = best.ctas;
      Lw.tc_stages[pi] = best.stages;
      Lw.tc_mt[pi] = best.mt;
      Lw.tc_halo[pi] = best.halo;
      Lw.tc_cb[pi] = best.cb;
      Lw.tc_so[pi] = best.so;
      Lw.tuned_hw[pi] = H * W;
      if (getenv("PG_TC_LOG"))
        fprintf(stderr,
                "pg_autotune: layer %d %dx%d cin %d cout %d stride %d leaves %u -> halo %d chunk %dB mt %d ctas %d "
                "stages %d staged-out %d: %.1f us\n",
                li, Hin, Win, Cin, Lr.cout, Lr.stride, ns, best.halo, best.cb, best.mt, best.ctas, best.stages, best.so,
                best_ms * 1e3f);
    }
    TcCfg cfg;
    if (Lw.tuned_hw[pi] == H * W) {
      cfg.ctas = Lw.tc_ctas[pi];
      cfg.stages = Lw.tc_stages[pi];
      cfg.mt = Lw.tc_mt[pi];
      cfg.halo = Lw.tc_halo[pi];
      cfg.cb = Lw.tc_cb[pi];
      cfg.so = Lw.tc_so[pi];
    }
    // A shape tuned for the other form of this layer (phase form or not)
    // does not apply.
    if (phase != (cfg.halo == 3)) cfg = TcCfg();
    if (phase) cfg.halo = 3;
    // Default shape: the built-in heuristic; in the phase form the first of
    // (chunk bytes, phases per tile) whose two stages fit in shared memory.
    auto launch_default = [&]() -> pg_status {
      if (!phase) return launch_tc(L, ns, les, out8, st, ctx->d_status, TcCfg());
      pg_status r = PG_ERR_UNSUPPORTED;
      static const int kShapes[5][2] = {{64, 4}, {32, 4}, {64, 2}, {32, 2}, {32, 1}};
      for (const auto &cm : kShapes) {
        TcCfg d;
        d.halo = 3;
        d.cb = cm[0];
        d.mt = cm[1];
        r = launch_tc(L, ns, les, out8, st, ctx->d_status, d);
        if (r != PG_ERR_UNSUPPORTED) break;
      }
      return r;
    };
    // Diagnostics: PG_TC_FORCE=<mode>[,cb,mt,ctas,stages,staged] runs every layer
    // that supports it with that operand staging mode and launch shape (zero
    // or missing fields: defaults); other layers run the default shape.  The
    // phase-form layers always run mode 3.
    if (const char *force = getenv("PG_TC_FORCE")) {
      TcCfg f;
      sscanf(force, "%d,%d,%d,%d,%d,%d", &f.halo, &f.cb, &f.mt, &f.ctas, &f.stages, &f.so);
      if (phase) f.halo = 3;
      PG_COUNT(ctx);
      const pg_status s = launch_tc(L, ns, les, out8, st, ctx->d_status, f);
      if (s != PG_ERR_UNSUPPORTED) return s;
      return launch_default();
    }
    PG_COUNT(ctx);
    pg_status s = (cfg.cb || cfg.mt || !phase) ? launch_tc(L, ns, les, out8, st, ctx->d_status, cfg) : launch_default();
    if (s == PG_ERR_UNSUPPORTED && (Lw.tuned_hw[pi] == H * W || phase)) s = launch_default();
    if (s != PG_OK && getenv("PG_TC_LOG"))
      fprintf(stderr, "pg: layer %d (%d experts) launch shape halo %d chunk %dB mt %d ctas %d stages %d staged-out %d: status %d\n",
              li, n_exp, cfg.halo, cfg.cb, cfg.mt, cfg.ctas, cfg.stages, cfg.so, (int)s);
    return s;
  };
  auto head = [&](int li, const T *in, int in_cs, int Cin) -> pg_status {
    const Layer &Lr = Ls[li];
    k_cout1_lp<T><<<ceil_div(M0, 256), 256, 0, st>>>(in, in_cs, H, W, Cin, Lr.k, Lr.w, Lr.b,
                                                     fp8 ? scale[ig[li]] : 1.0f, M0, y);
    PG_COUNT(ctx);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
  };
  if (net->arch == 2) {
    // The paper-style network (BF16 only): partial convolutions with the
    // FP32 scale maps of the mask pyramid, residual links, dilated
    // bottleneck; the 1x1 head runs in layer 10's epilogue.
    if (fp8 || !x0) return PG_ERR_UNSUPPORTED;
    const int c0 = net->widths[0], c1 = net->widths[1];
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4;
    const int k0c = c1 + c0, k1c = 2 * c1;
    T *a0 = (T *)act;
    T *cat0 = a0 + ns * HW * c0;
    T *d0 = cat0 + ns * HW * k0c;
    T *d0b = d0 + ns * HW * c0;
    T *a1 = d0b + ns * HW * c0;
    T *cat1 = a1 + ns * HW / 4 * c1;
    T *d1 = cat1 + ns * HW / 4 * k1c;
    T *b0 = d1 + ns * HW / 4 * c1;
    T *b1 = b0 + ns * HW / 16 * c1;
    float *mbuf = (float *)(b1 + ns * HW / 16 * c1);
    PaperMasks pm;
    PG_TRY(paper_masks(ctx, x0, ns, H, W, mbuf, &pm, st));
    PG_TRY(conv(0, xcol, cp, 0, H, W, cp, a0, c0, 0, 0, nullptr, pm.scale[0]));
    PG_TRY(conv(1, a0, c0, 0, H, W, c0, cat0, k0c, c1, 0, nullptr, pm.scale[1], a0, c0, 0));        // e0
    PG_TRY(conv(2, cat0, k0c, c1, H, W, c0, a1, c1, 0, 0, nullptr, pm.scale[2]));
    PG_TRY(conv(3, a1, c1, 0, H1, W1, c1, cat1, k1c, c1, 0, nullptr, pm.scale[3], a1, c1, 0));      // e1
    PG_TRY(conv(4, cat1, k1c, c1, H1, W1, c1, b0, c1, 0, 0, nullptr, pm.scale[4]));
    PG_TRY(conv(5, b0, c1, 0, H2, W2, c1, b1, c1, 0, 0, nullptr, pm.scale[5], b0, c1, 0));          // dilation 2
    PG_TRY(conv(6, b1, c1, 0, H2, W2, c1, cat1, k1c, 0, 1, nullptr, pm.scale[6], b1, c1, 0));       // dilation 4, up
    PG_TRY(conv(7, cat1, k1c, 0, H1, W1, k1c, d1, c1, 0, 0, nullptr, pm.scale[7]));
    PG_TRY(conv(8, d1, c1, 0, H1, W1, c1, cat0, k0c, 0, 1, nullptr, pm.scale[8], d1, c1, 0));       // up
    PG_TRY(conv(9, cat0, k0c, 0, H, W, k0c, d0, c0, 0, 0, nullptr, pm.scale[9]));
    return conv(10, d0, c0, 0, H, W, c0, d0b, c0, 0, 0, &Ls[11], pm.scale[10], d0, c0, 0);
  }
  if (net->arch == 0) {
    const int c = net->widths[0];
    T *t0 = (T *)act, *t1 = t0 + M0 * c;
    PG_TRY(conv(0, xcol, cp, 0, H, W, cp, t0, c, 0, 0));
    PG_TRY(conv(1, t0, c, 0, H, W, c, t1, c, 0, 0));
    return head(2, t1, c, c);
  }
  const int c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2], c3 = net->widths[3];
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  const int k0c = c1 + c0, k1c = c2 + c1, k2c = c3 + c2;
  T *cat0 = (T *)act;
  T *t0 = cat0 + ns * HW * k0c;
  T *t0b = t0 + ns * HW * c0;
  T *cat1 = t0b + ns * HW * c0;
  T *t1 = cat1 + ns * HW / 4 * k1c;
  T *cat2 = t1 + ns * HW / 4 * c1;
  T *t2 = cat2 + ns * HW / 16 * k2c;
  T *t3 = t2 + ns * HW / 16 * c2;
  // Phase form of decoder level lev (layer 12 - 2 lev over [upsample2(U), S],
  // maps of width W >> lev): the skip S goes to its own dense buffer at the
  // start of the concatenation buffer, and the layer before writes U there
  // too, at half resolution instead of its x2 upsampled copy.  BF16 only
  // (the E4M3 forms and their calibration pass keep the concatenation), and
  // only where the half-resolution grid is at least 32 wide, so the tiles'
  // tail past each leaf's rows stays small.
  bool ph[3];
  for (int lev = 0; lev < 3; ++lev) {
    const int Wl = W >> lev, Hl = H >> lev;
    bool ok = !fp8 && !mixed && !scale && !amax && Ls[12 - 2 * lev].w_ph_bf16 && Wl / 2 >= 32 &&
              2 * (Wl / 2 + 2) <= 256 && Hl % 2 == 0 && Wl % 2 == 0 && getenv("PG_TC_NO_PHASE") == nullptr;
    for (int e = 1; e < n_exp && ok; ++e) ok = experts[e]->layers[12 - 2 * lev].w_ph_bf16 != nullptr;
    ph[lev] = ok;
  }
  T *u0 = cat0 + ns * HW * c0, *u1 = cat1 + ns * HW / 4 * c1, *u2 = cat2 + ns * HW / 16 * c2;
  PG_TRY(conv(0, xcol, cp, 0, H, W, cp, t0, c0, 0, 0));
  if (ph[0]) {
    PG_TRY(conv(1, t0, c0, 0, H, W, c0, cat0, c0, 0, 0));
    PG_TRY(conv(2, cat0, c0, 0, H, W, c0, t1, c1, 0, 0));
  } else {
    PG_TRY(conv(1, t0, c0, 0, H, W, c0, cat0, k0c, c1, 0));
    PG_TRY(conv(2, cat0, k0c, c1, H, W, c0, t1, c1, 0, 0));
  }
  if (ph[1]) {
    PG_TRY(conv(3, t1, c1, 0, H1, W1, c1, cat1, c1, 0, 0));
    PG_TRY(conv(4, cat1, c1, 0, H1, W1, c1, t2, c2, 0, 0));
  } else {
    PG_TRY(conv(3, t1, c1, 0, H1, W1, c1, cat1, k1c, c2, 0));
    PG_TRY(conv(4, cat1, k1c, c2, H1, W1, c1, t2, c2, 0, 0));
  }
  if (ph[2]) {
    PG_TRY(conv(5, t2, c2, 0, H2, W2, c2, cat2, c2, 0, 0));
    PG_TRY(conv(6, cat2, c2, 0, H2, W2, c2, t3, c3, 0, 0));
    PG_TRY(conv(7, t3, c3, 0, H3, W3, c3, u2, c3, 0, 0));
    PG_TRY(conv(8, cat2, c2, 0, H2, W2, c2, t2, c2, 0, 0, nullptr, nullptr, nullptr, 0, 0, u2, c3, c3));
  } else {
    PG_TRY(conv(5, t2, c2, 0, H2, W2, c2, cat2, k2c, c3, 0));
    PG_TRY(conv(6, cat2, k2c, c3, H2, W2, c2, t3, c3, 0, 0));
    PG_TRY(conv(7, t3, c3, 0, H3, W3, c3, cat2, k2c, 0, 1));
    PG_TRY(conv(8, cat2, k2c, 0, H2, W2, k2c, t2, c2, 0, 0));
  }
  if (ph[1]) {
    PG_TRY(conv(9, t2, c2, 0, H2, W2, c2, u1, c2, 0, 0));
    PG_TRY(conv(10, cat1, c1, 0, H1, W1, c1, t1, c1, 0, 0, nullptr, nullptr, nullptr, 0, 0, u1, c2, c2));
  } else {
    PG_TRY(conv(9, t2, c2, 0, H2, W2, c2, cat1, k1c, 0, 1));
    PG_TRY(conv(10, cat1, k1c, 0, H1, W1, k1c, t1, c1, 0, 0));
  }
  if (ph[0]) {
    PG_TRY(conv(11, t1, c1, 0, H1, W1, c1, u0, c1, 0, 0));
    PG_TRY(conv(12, cat0, c0, 0, H, W, c0, t0, c0, 0, 0, nullptr, nullptr, nullptr, 0, 0, u0, c1, c1));
  } else {
    PG_TRY(conv(11, t1, c1, 0, H1, W1, c1, cat0, k0c, 0, 1));
    PG_TRY(conv(12, cat0, k0c, 0, H, W, k0c, t0, c0, 0, 0));
  }
  // The 1x1 head (Cout 1) + softplus runs in layer 13's epilogue.
  if (Ls[14].k == 1 && Ls[14].cout == 1) return conv(13, t0, c0, 0, H, W, c0, t0b, c0, 0, 0, &Ls[14]);
  PG_TRY(conv(13, t0, c0, 0, H, W, c0, t0b, c0, 0, 0));
  return head(14, t0b, c0, c0);
}

}  // namespace

pg_status forward_tc(pg_ctx *ctx, const Net *netc, pg_precision prec, const float *x0, void *actv, uint32_t ns, int H,
                     int W, float *y, cudaStream_t st, bool tune) {
  Net *net = const_cast<Net *>(netc);
  if (net->arch == 2 && prec != PG_BF16) return PG_ERR_UNSUPPORTED;
  if (prec == PG_BF16)
    return forward_lp<__nv_bfloat16>(ctx, net, false, x0, actv, ns, H, W, y, st, nullptr, nullptr, tune);
  if (prec != PG_FP8_E4M3 && prec != PG_FP8_MIXED) return PG_ERR_UNSUPPORTED;
  if (prec == PG_FP8_MIXED && net->arch != 1) return PG_ERR_UNSUPPORTED;
  std::unique_lock<std::mutex> lock(net_state_mutex());
  if (!net->act_calibrated) {
    // Delayed scaling: one BF16 pass over this chunk records the largest
    // |activation| of every group; scale = amax / 448 (E4M3's largest normal).
    unsigned int *d_amax;
    PG_TRY(ctx_alloc(ctx, 64, (void **)&d_amax));
    PG_CUDA(cudaMemsetAsync(d_amax, 0, 64, st));
    k_absmax<<<num_sms() * 4, 256, 0, st>>>(x0, (size_t)ns * H * W * 8, d_amax);
    PG_COUNT(ctx);
    pg_status s = forward_lp<__nv_bfloat16>(ctx, net, false, x0, actv, ns, H, W, y, st, nullptr, d_amax);
    unsigned int h[16];
    if (s == PG_OK && cudaMemcpyAsync(h, d_amax, 64, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess) {
      for (int g = 0; g < 16; ++g) {
        float m;
        memcpy(&m, &h[g], 4);
        net->act_scale[g] = m > 0.0f && isfinite(m) ? m / 448.0f : 1.0f;
      }
      net->act_calibrated = 1;
    } else if (s == PG_OK) {
      s = PG_ERR_CUDA;
    }
    ctx_free(ctx, d_amax, 64);
    PG_TRY(s);
  }
  lock.unlock();
  if (prec == PG_FP8_MIXED)
    return forward_lp<__nv_bfloat16>(ctx, net, false, x0, actv, ns, H, W, y, st, net->act_scale, nullptr, tune,
                                     true);
  return forward_lp<__nv_fp8_e4m3>(ctx, net, true, x0, actv, ns, H, W, y, st, net->act_scale, nullptr, tune);
}

pg_status forward_tc_experts(pg_ctx *ctx, const Net *const *nets, int n_exp, const int *d_range, int pos0, void *actv,
                             uint32_t ns, int H, int W, float *y, cudaStream_t st) {
  if (n_exp < 2 || n_exp > kMaxExperts) return PG_ERR_UNSUPPORTED;
  return forward_lp<__nv_bfloat16>(ctx, nets[0], false, nullptr, actv, ns, H, W, y, st, nullptr, nullptr, false, false,
                                   nets, n_exp, d_range, pos0);
}

int tc_max_experts() { return kMaxExperts; }

size_t tc_bytes_per_leaf(const Net *net, pg_precision prec, int H, int W) {
  // Sized for 2-byte activations in both forms: an FP8 reconstruction may
  // first run the BF16 calibration pass in the same buffer.
  (void)prec;
  const size_t es = 2, HW = (size_t)H * W;
  size_t n = HW * 16;  // first-layer input, 32 bytes per pixel
  if (net->arch == 0) return es * (n + 2 * HW * net->widths[0]) + 1024;
  if (net->arch == 2) {
    const size_t c0 = net->widths[0], c1 = net->widths[1];
    n += HW * (c0 + (c1 + c0) + 2 * c0) + HW / 4 * (c1 + 2 * c1 + c1) + HW / 16 * 2 * c1;
    return es * n + 4 * paper_mask_floats_per_leaf(H, W) + 1024;
  }
  const size_t c0 = net->widths[0], c1 = net->widths[1], c2 = net->widths[2], c3 = net->widths[3];
  n += HW * ((c1 + c0) + 2 * c0) + HW / 4 * ((c2 + c1) + c1) + HW / 16 * ((c3 + c2) + c2) + HW / 64 * c3;
  return es * n + 1024;
}

}  // namespace pgi
