// Internal declarations of libpg: handle layouts, device-side rules shared by
// the kernels (voxel quantisation, Morton codes, direction bins, Philox), and
// the host-side launchers each kernel file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "pg.h"

namespace pgi {

// ---------------------------------------------------------------- errors
// Bits of the per-context device status word.
enum : uint32_t { ST_INVALID_INPUT = 1u, ST_OVERFLOW = 2u, ST_TIMEOUT = 4u, ST_CAPACITY = 8u };

#define PG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      pgi::last_cuda_error() = e_;                      \
      return PG_ERR_CUDA;                               \
    }                                                   \
  } while (0)

#define PG_TRY(call)                    \
  do {                                  \
    pg_status s_ = (call);              \
    if (s_ != PG_OK) return s_;         \
  } while (0)

cudaError_t &last_cuda_error();

// ---------------------------------------------------------------- handles
enum : uint32_t {
  KIND_GRID = 0x50474744u, KIND_HIST = 0x50474848u, KIND_NET = 0x5047484Eu,
  KIND_MAP = 0x5047484Du, KIND_TABLES = 0x50474854u, KIND_MIS = 0x5047494Du, KIND_PROGRESS = 0x50475052u
};

struct Handle {
  uint32_t kind;
  uint32_t borrowed;  // owned by another handle: pg_free leaves it alone
  pg_ctx *ctx;
  size_t bytes;  // charged to the context budget
};

struct Grid {
  Handle h;
  uint64_t n;
  uint32_t L, A;
  int D, min_depth;
  uint32_t thr;
  float lo[3], hi[3], scale[3];
  uint64_t *codes;       // [n]   original order
  uint32_t *perm;        // [n]   sorted slot -> original index
  uint32_t *leaf_of;     // [n]   original index -> leaf
  uint64_t *leaf_code;   // [cap]
  int32_t *leaf_depth;   // [cap]
  uint32_t *leaf_begin;  // [cap]
  uint32_t *leaf_end;    // [cap]
  uint32_t *active;      // [cap] active leaves (count > 0), ascending
  int32_t *slot_of_leaf; // [cap]
  uint32_t *lut;         // [8^lut_depth] leaf containing the first code of each lut_depth cell
  int lut_depth;
  // Scene batch: scene s occupies the top bits of the code (s << 3 D); the
  // tree's first scene_levels levels enumerate scenes.  A single-scene grid
  // has n_scenes = 1, scene_levels = 0.
  uint32_t n_scenes;
  int scene_levels;
  uint32_t *scene_begin;  // [S+1] photon offsets per scene
  uint32_t *scene_leaf_begin;  // [S+1] first leaf per scene, L at S
  float *scene_geom;      // [S][6] lo[3], scale[3] per scene (batched grids)
  // The paper's grid rule (pg_build_grid_kd): R^3 voxels, each a binary tree.
  // Nodes 0 .. R^3-1 are the voxels' roots; kd_link >= 0 is a node's left
  // child (right = left + 1), < 0 is ~leaf.  leaf_code then holds each
  // leaf's voxel, codes each photon's voxel, D the deepest split, and
  // scale R / (hi - lo).
  int kd;
  uint32_t kd_R, kd_nodes;
  int32_t *kd_link;      // [kd_nodes]
  float *kd_tau;         // [kd_nodes] left holds x[axis] < tau
  uint8_t *kd_axis;      // [kd_nodes]
  void *block;           // single allocation holding the arrays above
};

// Host-side description of a scene batch for build_grid.
struct SceneBatch {
  uint32_t S;
  const uint32_t *d_begin;  // device [S+1]
  const float *h_geom;      // host [S][6]
};

struct Hist {
  Handle h;
  uint32_t A;
  int H, W;
  uint64_t *pow_cur, *pow_prev;  // [A][HW]
  uint32_t *cnt_cur, *cnt_prev;  // [A][HW]
  uint64_t *tot_cur, *tot_prev;  // [A]
  void *block;
};

struct Layer {
  int cout, cin, k, stride, act;
  int dil;    // tap spacing (1 except dilated layers)
  float *w;   // device, [k*k*cin][cout] (GEMM B operand, K-major rows)
  float *b;   // device, [cout]
  void *w_bf16;  // device, BF16 copy [cout][K] (tensor-core layout), or null
  void *w_fp8;   // device, FP8 E4M3 copy [cout][K], or null
  // device, BF16 phase-form weights of a U-Net decoder layer over
  // [upsample2(U), S]: [cout][9 Cs + 16 Cu] (see make_phase_weights), or null
  void *w_ph_bf16;
  size_t w_bf16_bytes, w_fp8_bytes, w_ph_bytes;
  // Weight images for the tensor-core layers: every pipeline stage's weight
  // blocks as they lie in shared memory (swizzled), so that one bulk copy
  // fills a stage.  Indexed [BF16 / E4M3][block order][128 / 64 / 32-byte
  // chunk]; built on first use (see conv_tc.cu), freed with the net.
  void *bimg[2][3][3];
  size_t bimg_bytes[2][3][3];
  float w_scale;  // FP8 per-tensor weight scale (w = w_fp8 * w_scale)
  // Tensor-core launch shape picked by pg_autotune, per reduced precision
  // (index 1 = BF16, 2 = FP8) for maps of tuned_hw[i] bins (0 = not tuned).
  int tc_ctas[3], tc_stages[3], tc_mt[3], tc_halo[3], tc_cb[3], tc_so[3];
  int tuned_hw[3];
};

struct Net {
  Handle h;
  int arch, n_layers;
  int widths[4];
  Layer layers[16];
  void *block;
  // FP8 activation scales per activation group (see conv_tc.cu), calibrated
  // on the first FP8 reconstruction with this net and reused afterwards.
  int act_calibrated;
  float act_scale[16];
};

struct Map {
  Handle h;
  uint32_t A;
  int H, W;
  float *y;  // [A][H][W]
  void *block;
};

struct Tables {
  Handle h;
  uint32_t A;
  int H, W;
  float *P;        // [A][HW]
  float *cdf_phi;  // [A][HW]
  float *cdf_z;    // [A][H]
  uint8_t *valid;  // [A]
  // Segment summaries for the samplers' search: every 8th entry of each
  // CDF (F[8k + 7]); null for rows shorter than 16.
  float *sum_phi;  // [A][H][W/8]
  float *sum_z;    // [A][H/8]
  void *block;
};

// First index i in [0, n) with u < F[i] for an ascending F with F[n-1] = 1 > u
// (n a power of two, F 16-byte aligned): the number of entries <= u.  With
// n >= 16, S holds F[8k + 7] for k < n/8 (S 8-byte aligned, 16-byte from n =
// 32): counting over S picks the 8-entry segment, counting over the segment
// picks the entry -- two rounds of independent vector loads (one 32-byte
// sector each for n <= 64) in place of log2(n) dependent probes.  Any
// correct search of a monotone table gives this index.
__device__ __forceinline__ int cdf_count4(float4 v, float u) {
  return (v.x <= u) + (v.y <= u) + (v.z <= u) + (v.w <= u);
}

__device__ __forceinline__ int first_above_seg(const float *__restrict__ F, const float *__restrict__ S, int n,
                                               float u) {
  if (n <= 4) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(F));
    return min(cdf_count4(v, u), n - 1);  // entries past n (n < 4) are never read as answers
  }
  int k = 0;
  if (n >= 16) {
    const int ns = n >> 3;
    if (ns == 2) {
      const float2 v = __ldg(reinterpret_cast<const float2 *>(S));
      k = (v.x <= u) + (v.y <= u);
    } else {
      for (int b = 0; b < ns; b += 4) k += cdf_count4(__ldg(reinterpret_cast<const float4 *>(S + b)), u);
    }
  }
  const float *seg = F + 8 * k;
  const float4 a = __ldg(reinterpret_cast<const float4 *>(seg)), b = __ldg(reinterpret_cast<const float4 *>(seg + 4));
  return 8 * k + cdf_count4(a, u) + cdf_count4(b, u);
}

// One-sample MIS state per leaf of a grid (Sec. 7.3): accumulated bounce
// contributions and counts by the strategy that sampled them, and the BSDF
// selection probability alpha.
struct Mis {
  Handle h;
  uint32_t L;
  double *nu_b, *nu_g;     // [L]
  uint32_t *q_b, *q_g;     // [L]
  float *alpha;            // [L]
  void *block;
};

// Progressive iterations (Sec. 7.1, 7.2; Algorithm 1).  The grid, the
// leaf-indexed planes, maps and tables are handles of their own kinds, lent
// to the caller (borrowed) and replaced as iterations go on.
struct Progress {
  Handle h;
  pg_progress_params p;
  uint32_t t;               // iterations added so far
  uint64_t total;           // photons added so far
  Grid *grid;               // leaf table; slot_of_leaf / active are the state's map slots (A = slots)
  Hist *cum;                // [slots][HW] planes: sums over all iterations, and before the leaf's last update
  Map *map;                 // [slots][H][W]
  Tables *tab;              // tables of map, or null before the first reconstruct
  pg_photon *stored;        // refining iterations keep their photons (the grid is rebuilt)
  float *stored_n;          // and their normals (grid_rule 1), or null
  int normals;              // -1 not yet known, 0 batches without normals, 1 with
  uint64_t n_stored, cap_stored;
  uint32_t cap_slots;       // rows allocated in cum and map (cum->A = map->A = slots in use)
  uint32_t *updated;        // slots whose planes changed in the last add (in leaf order)
  uint32_t n_updated, cap_updated;
};

}  // namespace pgi

namespace pgi {
struct PendingFrees;  // shared-budget bytes whose stream-ordered frees have not run yet
}

struct pg_ctx {
  int device;
  cudaStream_t stream;
  size_t budget, in_use;
  pg_budget *shared;   // optional budget shared with other contexts
  pgi::PendingFrees *pending;
  uint64_t launches;   // kernels launched for this context (pg_launch_count)
  uint32_t *d_status;  // device status word (pgi::ST_* bits)
  // Mapped pinned host words that kernels write small results into (leaf
  // counts, status), so reading them back takes no copy-engine transfer that
  // could queue behind the caller's large copies on other streams.
  volatile uint32_t *h_words;
  uint32_t *d_words;
  float *d_phi[9];     // boundary-ray tables (cos, sin) per log2(W), W <= 256
};

// Counts one kernel launch made for a context.
#define PG_COUNT(ctx) (++(ctx)->launches)

namespace pgi {

// ---------------------------------------------------------------- memory
pg_status ctx_alloc(pg_ctx *ctx, size_t bytes, void **ptr);
void ctx_free(pg_ctx *ctx, void *ptr, size_t bytes);
pg_status ctx_alloc_static(pg_ctx *ctx, size_t bytes, void **ptr);
void ctx_free_static(pg_ctx *ctx, void *ptr, size_t bytes);
// Returns to the shared budget the bytes of every free that has run on the
// GPU (all of them when `all`, which waits for the context's stream).
void ctx_reap_frees(pg_ctx *ctx, bool all);
bool budget_try_charge(pg_budget *b, size_t bytes);
void budget_release(pg_budget *b, size_t bytes);
// Device tables (cos, sin) of the W boundary rays, built once per W on the
// host of the calling process and cached on the context.
pg_status phi_table(pg_ctx *ctx, int W, const float **d_table);
// Reads one or two device words (b / hb may be null) once stream `st` has run
// all work before: a one-thread kernel puts them in the context's mapped host
// words, then the stream synchronises.  No copy-engine transfer is involved,
// so the read does not wait behind the caller's large copies.
pg_status read_words(pg_ctx *ctx, cudaStream_t st, const uint32_t *a, uint32_t *ha, const uint32_t *b = nullptr,
                     uint32_t *hb = nullptr);

// ---------------------------------------------------------------- device rules
// Voxel quantisation (Algorithm 1, voxel location): q = clamp(floor(fl32(
// fl32(x - lo) * s)), 0, top) with IEEE round-to-nearest FP32 operations
// (the __f*_rn intrinsics are never contracted into FMAs).
__device__ __forceinline__ uint32_t quantise(float x, float lo, float s, uint32_t top, uint32_t &bad) {
  if (!isfinite(x)) {
    bad = 1u;
    return 0u;
  }
  float f = floorf(__fmul_rn(__fsub_rn(x, lo), s));
  f = fmaxf(f, 0.0f);
  f = fminf(f, (float)top);
  return (uint32_t)f;
}

// Spread the low 21 bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1FFFFFu;
  x = (x | (x << 32)) & 0x001F00000000FFFFull;
  x = (x | (x << 16)) & 0x001F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint64_t morton3(uint32_t qx, uint32_t qy, uint32_t qz) {
  return spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
}

// The same interleave for cell indices of at most 10 bits (depth <= 10, a
// 30-bit code) in 32-bit arithmetic: bit b of v to bit 3b by four
// shift-or-mask steps (the bit-expansion step of Karras, "Maximizing
// parallelism in the construction of BVHs, octrees and k-d trees", HPG 2012),
// half the instructions of the 64-bit form.
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
  uint32_t x = v & 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

struct GridGeom {
  float lo[3], scale[3];
  uint32_t top;  // 2^D - 1
  int D;
};

__device__ __forceinline__ uint64_t position_code(const GridGeom &g, float x, float y, float z, uint32_t &bad) {
  uint32_t qx = quantise(x, g.lo[0], g.scale[0], g.top, bad);
  uint32_t qy = quantise(y, g.lo[1], g.scale[1], g.top, bad);
  uint32_t qz = quantise(z, g.lo[2], g.scale[2], g.top, bad);
  if (g.D <= 10) return (uint64_t)(spread3_10(qx) | (spread3_10(qy) << 1) | (spread3_10(qz) << 2));
  return morton3(qx, qy, qz);
}

// Leaf of a position in a grid of the paper's form: its voxel's root, then
// left while x[axis] < tau.  Children always have larger indices than their
// parent, and depth is at most 16, so the walk ends; the bound guards it.
struct KdView {
  const int32_t *link;
  const float *tau;
  const uint8_t *axis;
  float lo[3], scale[3];
  uint32_t R;
};

__device__ __forceinline__ uint32_t kd_locate(const KdView &k, float x, float y, float z, uint32_t &bad) {
  const uint32_t qx = quantise(x, k.lo[0], k.scale[0], k.R - 1, bad);
  const uint32_t qy = quantise(y, k.lo[1], k.scale[1], k.R - 1, bad);
  const uint32_t qz = quantise(z, k.lo[2], k.scale[2], k.R - 1, bad);
  int32_t v = (int32_t)(qx + k.R * (qy + k.R * qz));
  int32_t ln = __ldg(k.link + v);
  for (int it = 0; ln >= 0 && it < 64; ++it) {
    const int a = __ldg(k.axis + v);
    const float p = a == 0 ? x : (a == 1 ? y : z);
    v = ln + (p < __ldg(k.tau + v) ? 0 : 1);
    ln = __ldg(k.link + v);
  }
  return ln < 0 ? (uint32_t)~ln : 0u;
}

// Last leaf whose start code is <= code (leaf start codes ascend).
__device__ __forceinline__ uint32_t find_leaf(const uint64_t *__restrict__ leaf_code, uint32_t L, uint64_t code) {
  uint32_t lo = 0, hi = L;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(leaf_code + mid) <= code) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// Leaf of a code through the coarse table: the leaves of a depth-`ld` cell
// lie between the leaves holding its first code and the next cell's first
// code, so the binary search covers only those.
__device__ __forceinline__ uint32_t find_leaf_lut(const uint64_t *__restrict__ leaf_code, uint32_t L,
                                                  const uint32_t *__restrict__ lut, uint32_t ncell, int shift,
                                                  uint64_t code) {
  const uint32_t c = (uint32_t)(code >> shift);
  const uint32_t lo = __ldg(lut + c);
  uint32_t hi = c + 1 < ncell ? __ldg(lut + c + 1) + 1 : L;  // exclusive bound
  // Last l in [lo, hi) with leaf_code[l] <= code (holds at lo).
  uint32_t a = lo + 1;
  while (a < hi) {
    uint32_t mid = a + ((hi - a) >> 1);
    if (__ldg(leaf_code + mid) <= code) a = mid + 1;
    else hi = mid;
  }
  return a - 1;
}

// Cylindrical-map row: clamp(floor(z * H/2) + H/2, 0, H-1).  z * H/2 is exact.
__device__ __forceinline__ int dir_row(float z, int H) {
  int h2 = H >> 1;
  float f = floorf(__fmul_rn(z, (float)h2));
  f = fminf(fmaxf(f, (float)-h2), (float)(h2 - 1));
  return (int)f + h2;
}

// Exact sign test "direction (x, y) is not clockwise of boundary ray (c, s)",
// i.e. c*y - s*x >= 0: the products of two floats are exact in FP64 and the
// rounded FP64 difference keeps the exact sign.
__device__ __forceinline__ bool not_clockwise_exact(float c, float s, float x, float y) {
  double dd = __dsub_rn(__dmul_rn((double)c, (double)y), __dmul_rn((double)s, (double)x));
  return dd >= 0.0;
}

// Cylindrical-map column: the phi sector of (x, y) among W equal sectors,
// phi = atan2(y, x) in [0, 2 pi): the last boundary ray the direction is not
// clockwise of, within the half plane of the direction
// (upper: phi in [0, pi), rays 0..W/2-1; lower: phi in [pi, 2 pi), rays
// W/2..W-1).  tab holds cos at [0, W) and sin at [W, 2W).
static __device__ __noinline__ int dir_col_exact(float x, float y, int W, const float *tab, int lo, int hi) {
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (not_clockwise_exact(tab[mid], tab[W + mid], x, y)) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// FP32 form of the same test; `unsure` is set when the difference does not
// clear its rounding bound (4 ulp of |c y| + |s x|, normal operands).
__device__ __forceinline__ bool not_clockwise_f32(float c, float s, float x, float y, bool &unsure) {
  float a = __fmul_rn(c, y), b = __fmul_rn(s, x);
  float d = __fsub_rn(a, b);
  float mag = fabsf(a) + fabsf(b);
  unsure |= !(mag > 1e-30f && fabsf(d) > 4.8e-7f * mag);
  return d >= 0.0f;
}

// The answer is the last ray of the half plane that the direction is not
// clockwise of: the first ray always is, and the test holds up to the answer
// and fails after it.  A guess from the azimuth is checked against its own ray and
// the next one (one round of table reads, usually the last), and walked from
// there if either test disagrees, so any guess gives the same column.  Any
// unsure FP32 test redoes the search with the exact FP64 test (kept out of
// line: GB300's FP64 rate is a small fraction of FP32's).
// Approximate azimuth of (x, y) in [0, 2 pi) for the column guess: octant
// reduction and atan(t) ~ t / (1 + 0.28086 t^2) on [0, 1] (Rajan, Wang,
// Inkol and Joyal, "Efficient approximations for the arctangent function",
// IEEE Signal Processing Magazine 23(3), 2006; error under 0.005 rad).  The
// exact ray tests below decide the column, so the guess only has to be
// close; it costs a handful of instructions where atan2f costs dozens.
__device__ __forceinline__ float approx_azimuth(float x, float y) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float t = __fdividef(fminf(ax, ay), fmaxf(ax, ay));
  float a = __fdividef(t, fmaf(0.28086f, t * t, 1.0f));
  if (ay > ax) a = 1.5707963267948966f - a;
  if (x < 0.0f) a = 3.1415926535897932f - a;
  if (y < 0.0f) a = 6.2831853071795865f - a;
  return a;
}

__device__ __forceinline__ int dir_col(float x, float y, int W, const float *tab) {
  if (x == 0.0f && y == 0.0f) return 0;
  const bool upper = (y > 0.0f) || (y == 0.0f && x >= 0.0f);
  const int lo0 = upper ? 0 : (W >> 1), hi0 = lo0 + (W >> 1) - 1;
  const float phi = approx_azimuth(x, y);
  int a = (int)(phi * ((float)W * 0.15915494309189535f));
  a = min(max(a, lo0), hi0);
  const int b = a < hi0 ? a + 1 : a;
  const float c0 = tab[a], s0 = tab[W + a], c1 = tab[b], s1 = tab[W + b];
  bool unsure = false;
  if (a > lo0 && !not_clockwise_f32(c0, s0, x, y, unsure)) {
    --a;
    while (a > lo0 && !not_clockwise_f32(tab[a], tab[W + a], x, y, unsure)) --a;
  } else if (a < hi0 && not_clockwise_f32(c1, s1, x, y, unsure)) {
    ++a;
    while (a < hi0 && not_clockwise_f32(tab[a + 1], tab[W + a + 1], x, y, unsure)) ++a;
  }
  if (unsure) a = dir_col_exact(x, y, W, tab, lo0, hi0);
  return a;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// ---------------------------------------------------------------- launchers
// grid.cu
pg_status build_grid(pg_ctx *ctx, const pg_photon *d_ph, uint64_t n, const pg_grid_params *p, Grid *g,
                     const SceneBatch *sb = nullptr);
// A batch of photons binned into the fixed leaves of g (single scene): *view
// is g with this batch's sort permutation, per-leaf ranges and the leaves
// holding its photons (A of them); its arrays live in *scratch (bytes in
// *scratch_bytes, freed by the caller with ctx_free).
pg_status bin_into_grid(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n, Grid *view, void **scratch,
                        size_t *scratch_bytes);
// The paper's grid rule: R^3 voxels refined by binary trees (grid.cu).
pg_status build_grid_kd(pg_ctx *ctx, const pg_photon *d_ph, const float *d_normals, uint64_t n,
                        const pg_kd_params *p, Grid *g);
// progress.cu
pg_status hist_alloc(pg_ctx *ctx, Hist *h, uint32_t A, int H, int W);  // zeroed planes
// Reallocates to cap rows (zeroed), keeping the first `rows`; A becomes rows.
pg_status hist_grow(pg_ctx *ctx, Hist *h, uint32_t rows, uint32_t cap);
pg_status map_grow(pg_ctx *ctx, Map *m, uint32_t rows, uint32_t cap);
// Leaves in d_leaves (ascending) without a slot take slots g->A, g->A+1, ...
// (slot_of_leaf and the active list of g updated); *new_slots gets their
// number (one synchronisation).
pg_status assign_slots(pg_ctx *ctx, uint32_t nA, const uint32_t *d_leaves, Grid *g, uint32_t *new_slots);
pg_status slots_of(pg_ctx *ctx, uint32_t nA, const uint32_t *d_leaves, const Grid *g, uint32_t *d_out);
pg_status iota_slots(pg_ctx *ctx, uint32_t n, uint32_t *d_out);
// A batch binned into the fixed leaves of a grid of the paper's form (tree
// walk per photon, then a sort by leaf); as bin_into_grid otherwise.
pg_status bin_into_grid_kd(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n, Grid *view, void **scratch,
                           size_t *scratch_bytes);
// splat.cu
// A batch binned into a fixed grid (view from bin_into_grid) and merged into
// slot-indexed sums: for every leaf l of the view's active list, with slot
// s = slot_of_leaf[l]: prev[s] = cur[s], then cur[s] += the leaf's batch
// histogram (planes and totals).  n_bound sets the fixed-point bound
// (2^63 - 1) / n_bound.
pg_status splat_merge(pg_ctx *ctx, const Grid *view, const pg_photon *d_ph, uint64_t n_bound, int F,
                      const int32_t *d_slot_of_leaf, Hist *cum);
pg_status splat(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n, uint64_t n_prev, int F, Hist *h,
                const uint32_t *d_scene_nprev = nullptr);
// cnn.cu
pg_status net_prepare(pg_ctx *ctx, Net *net, pg_precision prec);
pg_status reconstruct(pg_ctx *ctx, const Hist *h, const Net *net, pg_precision prec, Map *m, bool tune = false);
// Maps of the leaves at positions [first, first + count) of the slot order
// d_perm (the identity when null), written to y_out in that position order.
pg_status reconstruct_range(pg_ctx *ctx, const Hist *h, const Net *net, pg_precision prec, float *y_out,
                            const uint32_t *d_perm, uint32_t first, uint32_t count, bool tune = false);
// Mixture of experts routed by leaf photon count (BF16 U-Nets): the leaves
// grouped by expert on the device, then one tensor-core launch per layer
// over every expert's tiles; maps y in slot order.  No host read-back.
pg_status reconstruct_experts_grouped(pg_ctx *ctx, const Hist *h, const Net *const *nets, int E,
                                     const uint32_t *count_bounds, float *y);
// Photon count of every active leaf (sum of its current count plane).
pg_status leaf_counts(pg_ctx *ctx, const Hist *h, uint32_t *d_counts);
// y[perm[k]] = yp[k], rows of HW floats (HW a multiple of 4).
pg_status scatter_rows(pg_ctx *ctx, const float *yp, const uint32_t *d_perm, uint32_t A, int HW, float *y);
// cdf.cu
pg_status build_cdf(pg_ctx *ctx, const Map *m, Tables *t);
// sample.cu
// Per-scene query ranges (device [S+1]) and Philox stream ids (device [S])
// of a batched call; null for a single-scene call.
struct QueryScenes {
  const uint32_t *d_qbegin = nullptr;
  const uint32_t *d_streams = nullptr;
};
pg_status sample(pg_ctx *ctx, const Grid *g, const Tables *t, const float *d_pos, uint64_t q, uint64_t seed,
                 uint32_t stream_id, float *d_dir, float *d_pdf, uint32_t *d_leaf, uint32_t *d_bin,
                 QueryScenes qs = QueryScenes());
pg_status eval_pdf(pg_ctx *ctx, const Grid *g, const Tables *t, const float *d_pos, const float *d_dir,
                   uint64_t q, float *d_pdf, QueryScenes qs = QueryScenes());

pg_status mis_init(pg_ctx *ctx, Mis *m);
pg_status mis_accumulate(pg_ctx *ctx, Mis *m, const Grid *g, const float *d_pos, const uint8_t *d_strategy,
                         const float *d_contrib, uint64_t q);
pg_status mis_update(pg_ctx *ctx, Mis *m, uint32_t min_count, float alpha_lo, float alpha_hi);
pg_status mis_sample(pg_ctx *ctx, const Grid *g, const Tables *t, const Mis *m, const float *d_pos,
                     const float *d_normal, uint64_t q, uint64_t seed, uint32_t stream_id, float *d_dir,
                     float *d_pdf, uint8_t *d_strategy);
pg_status mis_eval(pg_ctx *ctx, const Grid *g, const Tables *t, const Mis *m, const float *d_pos,
                   const float *d_normal, const float *d_dir, uint64_t q, float *d_pdf);

inline GridGeom geom_of(const Grid *g) {
  GridGeom gg;
  for (int a = 0; a < 3; ++a) {
    gg.lo[a] = g->lo[a];
    gg.scale[a] = g->scale[a];
  }
  gg.D = g->D;
  gg.top = (uint32_t)((1u << g->D) - 1u);
  return gg;
}

inline unsigned ceil_div(uint64_t a, uint64_t b) { return (unsigned)((a + b - 1) / b); }

// Query-side view of a grid of the paper's form (link null for an octree grid).
inline KdView kd_view_of(const Grid *g) {
  KdView k;
  memset(&k, 0, sizeof(k));
  if (!g->kd) return k;
  k.link = g->kd_link;
  k.tau = g->kd_tau;
  k.axis = g->kd_axis;
  for (int a = 0; a < 3; ++a) {
    k.lo[a] = g->lo[a];
    k.scale[a] = g->scale[a];
  }
  k.R = g->kd_R;
  return k;
}

}  // namespace pgi
