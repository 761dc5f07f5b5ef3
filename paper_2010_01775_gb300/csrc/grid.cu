// a1-a4: voxel location and the adaptive hierarchical grid (Sec. 7.1,
// Algorithm 1: locating a position's voxel and subdividing voxels), octree form.
//
//   k_morton        per photon: FP32 quantisation + Morton code (a1)
//   k_sort_*        stable LSD radix sort of (code, index), 8-bit digits (a2):
//                   upsweep digit histograms per 4096-key tile, per-digit scan
//                   over tiles, then a scatter that ranks keys stably inside
//                   the tile (warp match + per-warp digit counters), stages
//                   them in shared memory and writes digit runs coalesced
//   k_tree_*        top-down split of cells with count > threshold (a3): one
//                   launch per level, 8 lanes per cell find the 7 child
//                   boundaries by binary search inside the parent's range;
//                   bottom-up leaf counts and top-down offsets put the leaves
//                   in Morton order without sorting them
//   k_leaf_assign   per photon: leaf id by binary search of leaf start codes (a4)
//   k_tree_all      the same tree in one cooperative launch:
//                   the levels and phases follow one another through bounded
//                   grid-wide barriers (the per-level launches remain the
//                   fallback where cooperative launches are unavailable)
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include <vector>

#include "pg_internal.cuh"

namespace pgi {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kRadix = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr size_t kScatterSmem =
    (size_t)kSortTile * 8 + (size_t)kSortTile * 4 + (size_t)kSortWarps * kRadix * 4 + 2 * kRadix * 4;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block scan (blockDim a multiple of 32, <= 1024).  `sh` holds 32
// words of shared scratch.  Returns this thread's exclusive prefix; *total is
// the block sum.  Contains __syncthreads: call from all threads.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *total, uint32_t *sh) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = warp_incl_scan(v);
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nw ? sh[lane] : 0u;
    s = warp_incl_scan(s);
    sh[lane] = s;
  }
  __syncthreads();
  uint32_t prefix = (warp ? sh[warp - 1] : 0u) + x - v;
  *total = sh[nw - 1];
  __syncthreads();
  return prefix;
}

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *__restrict__ a, uint32_t n, uint64_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- a1
__global__ void k_morton(const pg_photon *__restrict__ ph, uint32_t n, GridGeom g, uint64_t *__restrict__ codes,
                         uint32_t *status) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = __ldg(reinterpret_cast<const float4 *>(ph + i));
  uint32_t bad = 0;
  codes[i] = position_code(g, a.x, a.y, a.z, bad);
  if (bad) atomicOr(status, ST_INVALID_INPUT);
}

// Scene batches: photon i belongs to the scene whose range holds i; its code
// is the scene index above the scene's own Morton code.
__global__ void k_morton_batched(const pg_photon *__restrict__ ph, uint32_t n, const uint32_t *__restrict__ begin,
                                 uint32_t S, const float *__restrict__ geom, int D, uint64_t *__restrict__ codes,
                                 uint32_t *status) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t lo = 0, hi = S;  // last s with begin[s] <= i
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(begin + mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  const float *gs = geom + 6 * lo;
  GridGeom gg;
  for (int a = 0; a < 3; ++a) {
    gg.lo[a] = __ldg(gs + a);
    gg.scale[a] = __ldg(gs + 3 + a);
  }
  gg.D = D;
  gg.top = (uint32_t)((1u << D) - 1u);
  float4 a = __ldg(reinterpret_cast<const float4 *>(ph + i));
  uint32_t bad = 0;
  codes[i] = ((uint64_t)lo << (3 * D)) | position_code(gg, a.x, a.y, a.z, bad);
  if (bad) atomicOr(status, ST_INVALID_INPUT);
}

// ---------------------------------------------------------------- a2: radix sort
// Lanes of the warp whose value d has the same low kBits bits: one ballot
// per bit (the lanes that share the bit with this lane), ANDed together.
// Cheaper than a warp match on this GPU (the sort's ranking and digit
// counting are bound by it).
template <int kBits>
__device__ __forceinline__ unsigned peers_of(uint32_t d) {
  unsigned m = 0xFFFFFFFFu;
#pragma unroll
  for (int b = 0; b < kBits; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned v = __ballot_sync(0xFFFFFFFFu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_upsweep(const uint64_t *__restrict__ keys, uint32_t n,
                                                               int shift, uint32_t *__restrict__ hist,
                                                               uint32_t nblocks) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * kSortTile;
  int lane = threadIdx.x & 31;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    uint32_t i = base + it * kSortThreads + threadIdx.x;
    uint32_t d = i < n ? (uint32_t)(keys[i] >> shift) & 255u : 0xFFFFFFFFu;
    unsigned peers = peers_of<9>(d);  // nine bits: the out-of-range marker is a group of its own
    if (d != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's tile counts, in place.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t *__restrict__ hist, uint32_t nblocks,
                                                    uint32_t *__restrict__ digit_total) {
  __shared__ uint32_t sh[32];
  uint32_t *row = hist + (size_t)blockIdx.x * nblocks;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nblocks; base += blockDim.x) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < nblocks ? row[i] : 0u, tot;
    uint32_t p = block_excl_scan(v, &tot, sh);
    if (i < nblocks) row[i] = carry + p;
    carry += tot;
  }
  if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

// Scatter of one LSD radix pass.  kMode 0: the first pass over the codes
// (value = original index); 1: a later pass over (key, value) pairs.  The
// packed forms sort codes of at most 32 bits as one 64-bit word (code << 32
// | original index), so a pass moves 8 instead of 12 bytes per photon each
// way: 2 is the first pass (codes in, packed words out), 3 a middle pass,
// 4 the last pass (packed words in; the sorted codes and the permutation
// out).  `shift` selects the digit of the word the pass reads from smem
// (the packed word's for modes 2-4).
template <int kMode>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               uint64_t *__restrict__ kout,
                                                               uint32_t *__restrict__ vout, uint32_t n, int shift,
                                                               const uint32_t *__restrict__ hist,
                                                               const uint32_t *__restrict__ digit_total,
                                                               uint32_t nblocks) {
  constexpr bool kPacked = kMode >= 2, kVal = !kPacked;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kSortTile);
  uint32_t *whist = sval + kSortTile;       // [warp][digit]
  uint32_t *tstart = whist + kSortWarps * kRadix;  // tile-local start of each digit run
  uint32_t *gbase = tstart + kRadix;        // global position of this tile's run of each digit
  __shared__ uint32_t sh[32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile0 = blockIdx.x * kSortTile;
  const uint32_t nvalid = min((uint32_t)kSortTile, n - tile0);

  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) whist[i] = 0;
  {
    uint32_t tot;
    uint32_t dt = digit_total[tid];
    uint32_t base = block_excl_scan(dt, &tot, sh);
    gbase[tid] = base + hist[(size_t)tid * nblocks + blockIdx.x];
  }
  __syncthreads();

  uint64_t key[kSortItems];
  uint32_t val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    uint32_t li = warp * (32 * kSortItems) + r * 32 + lane;
    uint32_t gi = tile0 + li;
    bool ok = li < nvalid;
    key[r] = ok ? kin[gi] : ~0ull;
    if (kMode == 2 && ok) key[r] = (key[r] << 32) | gi;
    if (kVal) val[r] = ok ? (kMode == 0 ? gi : vin[gi]) : 0u;
    uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
    unsigned peers = peers_of<8>(d);
    uint32_t before = __popc(peers & ((1u << lane) - 1u));
    uint32_t b = whist[warp * kRadix + d];
    rank[r] = b + before;
    __syncwarp();
    if (before == 0) whist[warp * kRadix + d] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t t = whist[w * kRadix + tid];
      whist[w * kRadix + tid] = run;
      run += t;
    }
    uint32_t tot;
    tstart[tid] = block_excl_scan(run, &tot, sh);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
    uint32_t pos = tstart[d] + whist[warp * kRadix + d] + rank[r];
    skey[pos] = key[r];
    if (kVal) sval[pos] = val[r];
  }
  __syncthreads();
  for (uint32_t p = tid; p < nvalid; p += kSortThreads) {
    uint64_t k = skey[p];
    uint32_t d = (uint32_t)(k >> shift) & 255u;
    uint32_t g = gbase[d] + (p - tstart[d]);
    if (kMode == 4) {
      kout[g] = k >> 32;
      vout[g] = (uint32_t)k;
    } else {
      kout[g] = k;
      if (kVal) vout[g] = sval[p];
    }
  }
}

// The header of a one-scene grid (photon range {0, n}, geometry {lo,
// scale}) from kernel arguments: no host-to-device copy, which would queue
// behind the caller's large uploads on the same copy engine.
__global__ void k_grid_header(uint32_t *scene_begin, float *scene_geom, uint32_t n, float lo0, float lo1, float lo2,
                              float s0, float s1, float s2) {
  if (threadIdx.x == 0) {
    scene_begin[0] = 0u;
    scene_begin[1] = n;
    scene_geom[0] = lo0;
    scene_geom[1] = lo1;
    scene_geom[2] = lo2;
    scene_geom[3] = s0;
    scene_geom[4] = s1;
    scene_geom[5] = s2;
  }
}

__global__ void k_zero_words(uint32_t *p, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0u;
}

// Leaf count, active count, tree flags and the status word into the
// context's mapped host words (read after the stream synchronises).
__global__ void k_grid_readback(const uint32_t *counters, const uint32_t *status, uint32_t *out) {
  if (threadIdx.x == 0) {
    volatile uint32_t *o = out;
    o[0] = counters[0];
    o[1] = counters[1];
    o[2] = counters[2];
    o[3] = *status;
    __threadfence_system();
  }
}

__global__ void k_iota(uint32_t *v, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

// ---------------------------------------------------------------- a3: tree
struct Tree {
  uint64_t *code;    // cell prefix at its own depth
  uint32_t *begin, *end;
  int32_t *child;    // first of 8 children, or -1 for a leaf
  uint32_t *nleaf;   // leaves in the subtree
  uint32_t *off;     // Morton rank of the subtree's first leaf
  uint32_t *level_start, *level_count;  // [17]
  uint32_t *counters;  // [0] = L, [1] = A, [2] = barrier timeout of the single-launch form
  uint32_t cap;
};

// Loads of tree data.  The per-level kernels read what earlier launches
// wrote (plain loads); the single cooperative launch reads what other
// blocks of the same launch wrote, so it goes around the L1 (ld.global.cg).
struct PlainLoad {
  template <class T>
  __device__ static T ld(const T *p) { return *p; }
};
struct L2Load {
  __device__ static uint32_t ld(const uint32_t *p) { return __ldcg(p); }
  __device__ static int32_t ld(const int32_t *p) { return __ldcg(p); }
  __device__ static uint64_t ld(const uint64_t *p) {
    return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(p));
  }
};

__device__ __forceinline__ void tree_init_cell(const uint64_t *__restrict__ sorted, uint32_t n, int D, int min_depth,
                                               const Tree &t, uint32_t c) {
  const uint32_t ncell = 1u << (3 * min_depth);
  const int shift = 3 * (D - min_depth);
  t.code[c] = c;
  t.begin[c] = lower_bound_u64(sorted, n, (uint64_t)c << shift);
  t.end[c] = (c + 1 == ncell) ? n : lower_bound_u64(sorted, n, (uint64_t)(c + 1) << shift);
  t.child[c] = -1;
}

__global__ void k_tree_init(const uint64_t *__restrict__ sorted, uint32_t n, int D, int min_depth, Tree t) {
  uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t ncell = 1u << (3 * min_depth);
  if (c == 0) {
    t.level_start[min_depth] = 0;
    t.level_count[min_depth] = ncell;
  }
  if (c >= ncell) return;
  tree_init_cell(sorted, n, D, min_depth, t, c);
}

// Level d: a cell splits when count > thr and d < D.  Lanes 8j..8j+7 of a
// warp serve one cell: lane k finds the first photon of child k.  Called by
// whole warps (shuffles); gid is the lane's index over the level's 8 cnt
// lanes.
template <class Ld>
__device__ __forceinline__ void tree_split_lane(const uint64_t *__restrict__ sorted, int D, int d, uint32_t thr,
                                                const Tree &t, uint32_t *status, uint32_t gid, uint32_t cnt,
                                                uint32_t lstart) {
  uint32_t rel = gid >> 3;
  int k = gid & 7;
  if (gid == 0) t.level_start[d + 1] = lstart + cnt;
  bool in = rel < cnt;
  uint32_t c = lstart + rel;
  uint32_t b = 0, e = 0;
  bool split = false;
  uint64_t code = 0;
  if (in) {
    b = Ld::ld(t.begin + c);
    e = Ld::ld(t.end + c);
    code = Ld::ld(t.code + c);
    split = (e - b > thr) && d < D;
  }
  uint32_t base = 0xFFFFFFFFu;
  if (split && k == 0) {
    uint32_t slot = atomicAdd(&t.level_count[d + 1], 8u);
    base = lstart + cnt + slot;
    if (base + 8 > t.cap) {
      atomicOr(status, ST_CAPACITY);
      base = 0xFFFFFFFFu;
    }
  }
  int lane = threadIdx.x & 31, group0 = lane & ~7;
  base = __shfl_sync(0xFFFFFFFFu, base, group0);
  uint32_t cb = b;
  uint64_t ccode = code * 8 + (uint64_t)k;
  if (split && base != 0xFFFFFFFFu && k > 0)
    cb = b + lower_bound_u64(sorted + b, e - b, ccode << (3 * (D - d - 1)));
  uint32_t ce = __shfl_down_sync(0xFFFFFFFFu, cb, 1);
  if (k == 7) ce = e;
  if (!in) return;
  if (k == 0) t.child[c] = (split && base != 0xFFFFFFFFu) ? (int32_t)base : -1;
  if (split && base != 0xFFFFFFFFu) {
    t.code[base + k] = ccode;
    t.begin[base + k] = cb;
    t.end[base + k] = ce;
    t.child[base + k] = -1;
  }
}

__global__ void k_tree_split(const uint64_t *__restrict__ sorted, int D, int d, uint32_t thr, Tree t,
                             uint32_t *status) {
  tree_split_lane<PlainLoad>(sorted, D, d, thr, t, status, blockIdx.x * blockDim.x + threadIdx.x, t.level_count[d],
                             t.level_start[d]);
}

template <class Ld>
__device__ __forceinline__ void tree_count_cell(int d, const Tree &t, uint32_t rel) {
  uint32_t c = Ld::ld(t.level_start + d) + rel;
  int32_t ch = Ld::ld(t.child + c);
  uint32_t s = 1;
  if (ch >= 0) {
    s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += Ld::ld(t.nleaf + ch + k);
  }
  t.nleaf[c] = s;
}

__global__ void k_tree_count(int d, Tree t) {
  uint32_t rel = blockIdx.x * blockDim.x + threadIdx.x;
  if (rel >= t.level_count[d]) return;
  tree_count_cell<PlainLoad>(d, t, rel);
}

__global__ void __launch_bounds__(1024) k_tree_root_offsets(int min_depth, Tree t) {
  __shared__ uint32_t sh[32];
  uint32_t ncell = 1u << (3 * min_depth), carry = 0;
  for (uint32_t base = 0; base < ncell; base += blockDim.x) {
    uint32_t i = base + threadIdx.x, tot;
    uint32_t v = i < ncell ? t.nleaf[i] : 0u;
    uint32_t p = block_excl_scan(v, &tot, sh);
    if (i < ncell) t.off[i] = carry + p;
    carry += tot;
  }
  if (threadIdx.x == 0) t.counters[0] = carry;
}

template <class Ld>
__device__ __forceinline__ void tree_offsets_cell(int D, int d, const Tree &t, uint32_t rel,
                                                  uint64_t *__restrict__ leaf_code, int32_t *__restrict__ leaf_depth,
                                                  uint32_t *__restrict__ leaf_begin, uint32_t *__restrict__ leaf_end) {
  uint32_t c = Ld::ld(t.level_start + d) + rel;
  int32_t ch = Ld::ld(t.child + c);
  uint32_t o = Ld::ld(t.off + c);
  if (ch >= 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      t.off[ch + k] = o;
      o += Ld::ld(t.nleaf + ch + k);
    }
  } else {
    leaf_code[o] = Ld::ld(t.code + c) << (3 * (D - d));
    leaf_depth[o] = d;
    leaf_begin[o] = Ld::ld(t.begin + c);
    leaf_end[o] = Ld::ld(t.end + c);
  }
}

__global__ void k_tree_offsets(int D, int d, Tree t, uint64_t *__restrict__ leaf_code,
                               int32_t *__restrict__ leaf_depth, uint32_t *__restrict__ leaf_begin,
                               uint32_t *__restrict__ leaf_end) {
  uint32_t rel = blockIdx.x * blockDim.x + threadIdx.x;
  if (rel >= t.level_count[d]) return;
  tree_offsets_cell<PlainLoad>(D, d, t, rel, leaf_code, leaf_depth, leaf_begin, leaf_end);
}

// Active leaves (>= 1 photon) get consecutive map slots in leaf order.
__global__ void __launch_bounds__(1024) k_active(Tree t, const uint32_t *__restrict__ leaf_begin,
                                                 const uint32_t *__restrict__ leaf_end, uint32_t *__restrict__ active,
                                                 int32_t *__restrict__ slot_of_leaf) {
  __shared__ uint32_t sh[32];
  uint32_t L = t.counters[0], carry = 0;
  for (uint32_t base = 0; base < L; base += blockDim.x) {
    uint32_t l = base + threadIdx.x, tot;
    uint32_t f = (l < L && leaf_end[l] > leaf_begin[l]) ? 1u : 0u;
    uint32_t p = block_excl_scan(f, &tot, sh);
    if (l < L) {
      slot_of_leaf[l] = f ? (int32_t)(carry + p) : -1;
      if (f) active[carry + p] = l;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) t.counters[1] = carry;
}

// Coarse lookup table for query-side leaf location: for every cell of depth
// lut_depth, the leaf containing its first code.
__global__ void k_leaf_lut(const uint64_t *__restrict__ leaf_code, const uint32_t *__restrict__ counters, int shift,
                           uint32_t ncell, uint32_t *__restrict__ lut) {
  uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  lut[c] = find_leaf(leaf_code, counters[0], (uint64_t)c << shift);
}

// First leaf of every scene of a batch (leaves are ordered by scene), and L
// at index S: slot s starts at code s << shift.
__global__ void k_scene_leaves(const uint64_t *__restrict__ leaf_code, const uint32_t *__restrict__ counters,
                               int shift, uint32_t S, bool full, uint32_t *__restrict__ out) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > S) return;
  const uint32_t L = counters[0];
  out[s] = (s == S && full) ? L : find_leaf(leaf_code, L, (uint64_t)s << shift);
}

// ---------------------------------------------------------------- a3 in one launch
// The whole tree in one cooperative launch (every block resident): the
// levels and phases follow one another through grid-wide barriers instead
// of one launch per level and phase.
struct TreeAll {
  const uint64_t *sorted;
  uint32_t n;
  int D, dmin;
  uint32_t thr;
  Tree t;
  uint64_t *leaf_code;
  int32_t *leaf_depth;
  uint32_t *leaf_begin, *leaf_end;
  uint32_t *barrier;   // one zeroed arrival counter per barrier
  uint32_t *status;    // the context's status word (capacity, as the per-level launches)
  uint32_t *timeout;   // ST_TIMEOUT when a barrier gave up (read back by the host)
};

__device__ __forceinline__ unsigned long long grid_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier k: thread 0 of every block arrives and waits until all
// blocks have, at most about a second; then it sets ST_TIMEOUT and the
// block gives up (returns false).  The fences make the blocks' writes before
// the barrier visible to the loads after it.
__device__ bool grid_barrier(uint32_t *counters, int k, uint32_t *status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counters + k, 1u);
    ok = 1;
    const unsigned long long t0 = grid_globaltimer();
    for (uint32_t it = 0; *(volatile uint32_t *)(counters + k) < gridDim.x; ++it) {
      if ((it & 255u) == 255u && grid_globaltimer() - t0 > 1000000000ull) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) k_tree_all(TreeAll p) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const Tree &t = p.t;
  int bk = 0;
  const uint32_t ncell0 = 1u << (3 * p.dmin);
  if (tid == 0) {
    t.level_start[p.dmin] = 0;
    t.level_count[p.dmin] = ncell0;
  }
  for (uint32_t c = tid; c < ncell0; c += nth) tree_init_cell(p.sorted, p.n, p.D, p.dmin, t, c);
  if (!grid_barrier(p.barrier, bk++, p.timeout)) return;
  // Top-down splits, one level per barrier, until a level is empty or at
  // the maximum depth (whose cells never split).
  int dlast = p.dmin;
  for (int d = p.dmin; d < p.D; ++d) {
    const uint32_t cnt = L2Load::ld(t.level_count + d), lstart = L2Load::ld(t.level_start + d);
    if (cnt == 0) break;
    for (uint32_t base = blockIdx.x * blockDim.x; base < 8u * cnt; base += nth)
      tree_split_lane<L2Load>(p.sorted, p.D, d, p.thr, t, p.status, base + threadIdx.x, cnt, lstart);
    if (!grid_barrier(p.barrier, bk++, p.timeout)) return;
    if (L2Load::ld(t.level_count + d + 1) == 0) break;
    dlast = d + 1;
  }
  // Bottom-up leaf counts.
  for (int d = dlast; d >= p.dmin; --d) {
    const uint32_t cnt = L2Load::ld(t.level_count + d);
    for (uint32_t r = tid; r < cnt; r += nth) tree_count_cell<L2Load>(d, t, r);
    if (!grid_barrier(p.barrier, bk++, p.timeout)) return;
  }
  // Offsets of the initial cells (one block), then top-down.
  if (blockIdx.x == 0) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ncell0; base += blockDim.x) {
      uint32_t i = base + threadIdx.x, tot;
      uint32_t v = i < ncell0 ? L2Load::ld(t.nleaf + i) : 0u;
      uint32_t pre = block_excl_scan(v, &tot, sh);
      if (i < ncell0) t.off[i] = carry + pre;
      carry += tot;
    }
    if (threadIdx.x == 0) t.counters[0] = carry;
  }
  if (!grid_barrier(p.barrier, bk++, p.timeout)) return;
  for (int d = p.dmin; d <= dlast; ++d) {
    const uint32_t cnt = L2Load::ld(t.level_count + d);
    for (uint32_t r = tid; r < cnt; r += nth)
      tree_offsets_cell<L2Load>(p.D, d, t, r, p.leaf_code, p.leaf_depth, p.leaf_begin, p.leaf_end);
    if (!grid_barrier(p.barrier, bk++, p.timeout)) return;
  }
}

// ---------------------------------------------------------------- a4
// Leaf of every photon: the last leaf whose start code is at most the
// photon's, searched only among the leaves of its coarse cell (the table
// k_leaf_lut writes).
__global__ void k_leaf_assign(const uint64_t *__restrict__ sorted, const uint32_t *__restrict__ perm, uint32_t n,
                              const uint64_t *__restrict__ leaf_code, const uint32_t *__restrict__ counters,
                              const uint32_t *__restrict__ lut, uint32_t ncell, int shift,
                              uint32_t *__restrict__ leaf_of) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t L = counters[0];
  leaf_of[perm[i]] = find_leaf_lut(leaf_code, L, lut, ncell, shift, sorted[i]);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

pg_status build_grid(pg_ctx *ctx, const pg_photon *d_ph, uint64_t n64, const pg_grid_params *p, Grid *g,
                     const SceneBatch *sb) {
  cudaStream_t st = ctx->stream;
  const uint32_t n = (uint32_t)n64;
  // A scene batch adds scene_levels octree levels above every scene's root
  // (8^scene_levels >= S); those levels always split, so each scene keeps
  // exactly the tree it would have alone.
  const uint32_t S = sb ? sb->S : 1u;
  int SL = 0;
  while ((1ull << (3 * SL)) < S) ++SL;
  const int Dsp = p->max_depth;  // spatial depth of every scene
  const int D = Dsp + SL, dmin = p->min_depth + SL;
  if (D > 18 || dmin > 6) return PG_ERR_UNSUPPORTED;
  const uint32_t thr = p->split_threshold;
  g->n = n;
  g->D = Dsp;
  g->min_depth = p->min_depth;
  g->thr = thr;
  g->n_scenes = S;
  g->scene_levels = SL;
  for (int a = 0; a < 3; ++a) {
    g->lo[a] = p->lo[a];
    g->hi[a] = p->hi[a];
    g->scale[a] = (float)(ldexp(1.0, Dsp) / ((double)p->hi[a] - (double)p->lo[a]));
  }
  // Cell capacity: split cells of one level are disjoint and hold > thr
  // photons each, so each level below min_depth adds at most 8 n/(thr+1).
  uint64_t per_level = 8ull * (n / ((uint64_t)thr + 1ull));
  uint64_t cap = 1ull << (3 * dmin), lvl = cap;
  std::vector<uint64_t> bound(D + 2, 0);
  bound[dmin] = lvl;
  for (int d = dmin + 1; d <= D; ++d) {
    uint64_t full = lvl * 8;
    lvl = full < per_level ? full : per_level;
    bound[d] = lvl;
    cap += lvl;
  }
  if (cap >= (1ull << 31)) return PG_ERR_UNSUPPORTED;

  // Handle block.
  size_t b_codes = align256(8ull * n), b_perm = align256(4ull * n), b_lo = align256(4ull * n);
  size_t b_lc = align256(8 * cap), b_l4 = align256(4 * cap);
  g->lut_depth = D < 6 ? D : 6;
  const uint32_t lut_cells = 1u << (3 * g->lut_depth);
  size_t b_lut = align256(4ull * lut_cells);
  size_t b_sb = align256(4ull * (S + 1)), b_sg = align256(24ull * S);
  g->h.bytes = b_codes + b_perm + b_lo + b_lc + 5 * b_l4 + b_lut + 2 * b_sb + b_sg;
  PG_TRY(ctx_alloc(ctx, g->h.bytes, &g->block));
  uint8_t *q = (uint8_t *)g->block;
  g->codes = (uint64_t *)q; q += b_codes;
  g->perm = (uint32_t *)q; q += b_perm;
  g->leaf_of = (uint32_t *)q; q += b_lo;
  g->leaf_code = (uint64_t *)q; q += b_lc;
  g->leaf_depth = (int32_t *)q; q += b_l4;
  g->leaf_begin = (uint32_t *)q; q += b_l4;
  g->leaf_end = (uint32_t *)q; q += b_l4;
  g->active = (uint32_t *)q; q += b_l4;
  g->slot_of_leaf = (int32_t *)q; q += b_l4;
  g->lut = (uint32_t *)q; q += b_lut;
  g->scene_begin = (uint32_t *)q; q += b_sb;
  g->scene_leaf_begin = (uint32_t *)q; q += b_sb;
  g->scene_geom = (float *)q;
  if (sb) {
    PG_CUDA(cudaMemcpyAsync(g->scene_begin, sb->d_begin, 4ull * (S + 1), cudaMemcpyDefault, st));
    PG_CUDA(cudaMemcpyAsync(g->scene_geom, sb->h_geom, 24ull * S, cudaMemcpyHostToDevice, st));
  } else {
    k_grid_header<<<1, 32, 0, st>>>(g->scene_begin, g->scene_geom, (uint32_t)n, g->lo[0], g->lo[1], g->lo[2],
                                     g->scale[0], g->scale[1], g->scale[2]), PG_COUNT(ctx);
  }

  // Scratch: sort ping-pong, digit histograms, cells.
  const int passes = (3 * D + 7) / 8;
  const uint32_t nblocks = n ? ceil_div(n, kSortTile) : 0;
  size_t s_k = align256(8ull * n), s_v = align256(4ull * n), s_h = align256(4ull * kRadix * (nblocks + 1));
  size_t s_dt = align256(4 * kRadix), s_c8 = align256(8 * cap), s_c4 = align256(4 * cap), s_lv = align256(4 * 128);
  size_t scratch_bytes = 2 * s_k + s_v + s_h + s_dt + s_c8 + 5 * s_c4 + s_lv;
  void *scratch = nullptr;
  pg_status rs = ctx_alloc(ctx, scratch_bytes, &scratch);
  if (rs != PG_OK) return rs;
  struct Guard {
    pg_ctx *c; void *p; size_t b;
    ~Guard() { ctx_free(c, p, b); }
  } guard{ctx, scratch, scratch_bytes};
  q = (uint8_t *)scratch;
  uint64_t *kA = (uint64_t *)q; q += s_k;
  uint64_t *kB = (uint64_t *)q; q += s_k;
  uint32_t *vT = (uint32_t *)q; q += s_v;
  uint32_t *hist = (uint32_t *)q; q += s_h;
  uint32_t *dtot = (uint32_t *)q; q += s_dt;
  Tree t;
  t.code = (uint64_t *)q; q += s_c8;
  t.begin = (uint32_t *)q; q += s_c4;
  t.end = (uint32_t *)q; q += s_c4;
  t.child = (int32_t *)q; q += s_c4;
  t.nleaf = (uint32_t *)q; q += s_c4;
  t.off = (uint32_t *)q; q += s_c4;
  t.level_start = (uint32_t *)q;
  t.level_count = t.level_start + 20;
  t.counters = t.level_count + 20;
  t.cap = (uint32_t)cap;
  uint32_t *barriers = t.level_start + 64;  // arrival counters of the cooperative launch's barriers
  k_zero_words<<<1, 128, 0, st>>>(t.level_start, 128), PG_COUNT(ctx);

  GridGeom gg = geom_of(g);
  const int TB = 256;
  if (n && sb)
    k_morton_batched<<<ceil_div(n, TB), TB, 0, st>>>(d_ph, n, g->scene_begin, S, g->scene_geom, Dsp, g->codes,
                                                     ctx->d_status), PG_COUNT(ctx);
  else if (n)
    k_morton<<<ceil_div(n, TB), TB, 0, st>>>(d_ph, n, gg, g->codes, ctx->d_status), PG_COUNT(ctx);

  // a2: stable LSD radix sort; the final permutation lands in g->perm.
  const uint64_t *sorted = g->codes;
  if (n && passes == 0) {
    k_iota<<<ceil_div(n, TB), TB, 0, st>>>(g->perm, n), PG_COUNT(ctx);
  } else if (n) {
    PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
    PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
    // Codes of at most 32 bits sort as packed words (code << 32 | index):
    // one 8-byte word per photon through every pass but the last, which
    // writes the sorted codes and the permutation.
    const bool packed = passes >= 2 && 3 * D <= 32;
    if (packed) {
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
    }
    // Value buffers alternate so that the last pass writes g->perm.
    const uint64_t *kin = g->codes;
    const uint32_t *vin = nullptr;
    for (int ps = 0; ps < passes; ++ps) {
      uint64_t *kout = (ps & 1) ? kB : kA;
      uint32_t *vout = ((passes - 1 - ps) & 1) ? vT : g->perm;
      int shift = 8 * ps;
      if (packed) {
        // The first pass reads the codes themselves; the packed words carry
        // the code's digit 32 bits higher.
        k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, n, ps ? 32 + shift : shift, hist, nblocks),
            PG_COUNT(ctx);
        k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot), PG_COUNT(ctx);
        if (ps == 0)
          k_sort_scatter<2><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, nullptr, kout, nullptr, n, 32 + shift,
                                                                         hist, dtot, nblocks), PG_COUNT(ctx);
        else if (ps + 1 < passes)
          k_sort_scatter<3><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, nullptr, kout, nullptr, n, 32 + shift,
                                                                         hist, dtot, nblocks), PG_COUNT(ctx);
        else
          k_sort_scatter<4><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, nullptr, kout, g->perm, n, 32 + shift,
                                                                         hist, dtot, nblocks), PG_COUNT(ctx);
        kin = kout;
        continue;
      }
      k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, hist, nblocks), PG_COUNT(ctx);
      k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot), PG_COUNT(ctx);
      if (ps == 0)
        k_sort_scatter<0><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist, dtot,
                                                                          nblocks), PG_COUNT(ctx);
      else
        k_sort_scatter<1><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                           dtot, nblocks), PG_COUNT(ctx);
      kin = kout;
      vin = vout;
    }
    sorted = kin;
  }

  // a3: the tree in one cooperative launch where the device allows it
  // (PG_GRID_LEVEL_LAUNCHES=1 forces the per-level launches below).
  bool coop = false;
  {
    int dev = 0, can = 0, occ = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&can, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && can &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tree_all, 256, 0) == cudaSuccess && occ > 0 &&
        !getenv("PG_GRID_LEVEL_LAUNCHES")) {
      TreeAll pa;
      pa.sorted = sorted;
      pa.n = n;
      pa.D = D;
      pa.dmin = dmin;
      pa.thr = thr;
      pa.t = t;
      pa.leaf_code = g->leaf_code;
      pa.leaf_depth = g->leaf_depth;
      pa.leaf_begin = g->leaf_begin;
      pa.leaf_end = g->leaf_end;
      pa.barrier = barriers;
      pa.status = ctx->d_status;
      pa.timeout = t.counters + 2;
      void *args[] = {&pa};
      const int blocks = sms;  // one block per SM: the barriers wait for fewer arrivals
      if (cudaLaunchCooperativeKernel((const void *)k_tree_all, blocks, 256, args, 0, st) == cudaSuccess) {
        PG_COUNT(ctx);
        coop = true;
      }
    }
    cudaGetLastError();
  }
  if (!coop) {
    // a3: tree, level by level.
    uint32_t ncell0 = 1u << (3 * dmin);
    k_tree_init<<<ceil_div(ncell0, TB), TB, 0, st>>>(sorted, n, D, dmin, t), PG_COUNT(ctx);
    // Levels whose cell bound is zero cannot hold cells (no launch).
    for (int d = dmin; d <= D && bound[d]; ++d) {
      uint64_t threads = 8 * bound[d];
      k_tree_split<<<ceil_div(threads, TB), TB, 0, st>>>(sorted, D, d, thr, t, ctx->d_status), PG_COUNT(ctx);
    }
    for (int d = D; d >= dmin; --d)
      if (bound[d]) k_tree_count<<<ceil_div(bound[d], TB), TB, 0, st>>>(d, t), PG_COUNT(ctx);
    k_tree_root_offsets<<<1, 1024, 0, st>>>(dmin, t), PG_COUNT(ctx);
    for (int d = dmin; d <= D && bound[d]; ++d)
      k_tree_offsets<<<ceil_div(bound[d], TB), TB, 0, st>>>(D, d, t, g->leaf_code, g->leaf_depth, g->leaf_begin,
                                                             g->leaf_end), PG_COUNT(ctx);
  }
  k_active<<<1, 1024, 0, st>>>(t, g->leaf_begin, g->leaf_end, g->active, g->slot_of_leaf), PG_COUNT(ctx);
  k_leaf_lut<<<ceil_div(lut_cells, TB), TB, 0, st>>>(g->leaf_code, t.counters, 3 * (D - g->lut_depth), lut_cells,
                                                      g->lut), PG_COUNT(ctx);
  // a4: leaf of every photon.
  if (n)
    k_leaf_assign<<<ceil_div(n, TB), TB, 0, st>>>(sorted, g->perm, n, g->leaf_code, t.counters, g->lut, lut_cells,
                                                   3 * (D - g->lut_depth), g->leaf_of), PG_COUNT(ctx);
  k_scene_leaves<<<ceil_div(S + 1, TB), TB, 0, st>>>(g->leaf_code, t.counters, 3 * Dsp, S,
                                                     S == (1u << (3 * SL)), g->scene_leaf_begin), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());

  // Counts and status come back through mapped host words written by a
  // kernel, not a device-to-host copy (which would wait behind the caller's
  // large downloads on the copy engine).
  k_grid_readback<<<1, 32, 0, st>>>(t.counters, ctx->d_status, ctx->d_words), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaStreamSynchronize(st));
  const uint32_t hc[3] = {ctx->h_words[0], ctx->h_words[1], ctx->h_words[2]};
  const uint32_t status = ctx->h_words[3];
  if (status & ST_CAPACITY) return PG_ERR_UNSUPPORTED;
  if (hc[2] & ST_TIMEOUT) return PG_ERR_TIMEOUT;
  if (status & ST_INVALID_INPUT) {
    PG_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, st));
    PG_CUDA(cudaStreamSynchronize(st));
    return PG_ERR_INVALID_INPUT;
  }
  g->L = hc[0];
  g->A = hc[1];
  return PG_OK;
}

// ---------------------------------------------------------------- the paper's grid rule
// Regular R^3 voxels, each refined by a binary tree (Sec. 7.1, Sec. 8).
// Photons are sorted by voxel; the trees then grow level by level: a warp
// per node gathers the node's statistics (coordinate extent, fixed-point
// normal sums) and decides the split, and a CTA per splitting node finds the
// median by a four-pass radix select over order-preserving keys and
// partitions the node's slice of the permutation stably.  Leaves are
// numbered depth-first through bottom-up leaf counts and top-down offsets.
namespace {

constexpr int kKdNormalBits = 20;
constexpr int kKdSplitThreads = 256;

__device__ __forceinline__ uint32_t kd_key(float x) {
  const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));  // -0 -> +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float kd_unkey(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ float kd_coord(const pg_photon *__restrict__ ph, uint32_t p, int a) {
  return __ldg(reinterpret_cast<const float *>(ph + p) + a);
}

__global__ void k_kd_cells(const pg_photon *__restrict__ ph, uint32_t n, KdView kv, uint64_t *__restrict__ cells,
                           uint32_t *status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = __ldg(reinterpret_cast<const float4 *>(ph + i));
  uint32_t bad = 0;
  const uint32_t qx = quantise(a.x, kv.lo[0], kv.scale[0], kv.R - 1, bad);
  const uint32_t qy = quantise(a.y, kv.lo[1], kv.scale[1], kv.R - 1, bad);
  const uint32_t qz = quantise(a.z, kv.lo[2], kv.scale[2], kv.R - 1, bad);
  cells[i] = (uint64_t)qx + (uint64_t)kv.R * ((uint64_t)qy + (uint64_t)kv.R * qz);
  if (bad) atomicOr(status, ST_INVALID_INPUT);
}

__global__ void k_kd_roots(const uint64_t *__restrict__ sorted, uint32_t n, uint32_t C, uint32_t *__restrict__ nb,
                           uint32_t *__restrict__ ne) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  nb[c] = lower_bound_u64(sorted, n, c);
  ne[c] = c + 1 == C ? n : lower_bound_u64(sorted, n, (uint64_t)c + 1);
}

// One warp per node of a level: extent and normal sums, then the decision.
__global__ void k_kd_stats(const pg_photon *__restrict__ ph, const float *__restrict__ nrm,
                           const uint32_t *__restrict__ perm, uint32_t N, const uint32_t *__restrict__ nb,
                           const uint32_t *__restrict__ ne, int depth, int max_depth, uint32_t thr, double vthr,
                           uint32_t *__restrict__ flag, uint8_t *__restrict__ axis, uint32_t *status) {
  const uint32_t v = (uint32_t)((((uint64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= N) return;
  const uint32_t b = nb[v], e = ne[v], m = e - b;
  if (depth >= max_depth || m < 2) {
    if (lane == 0) {
      flag[v] = 0;
      axis[v] = 0;
    }
    return;
  }
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  long long sn[3] = {0, 0, 0};
  for (uint32_t i = b + lane; i < e; i += 32) {
    const uint32_t p = __ldg(perm + i);
    const float4 r = __ldg(reinterpret_cast<const float4 *>(ph + p));
    lo[0] = fminf(lo[0], r.x); hi[0] = fmaxf(hi[0], r.x);
    lo[1] = fminf(lo[1], r.y); hi[1] = fmaxf(hi[1], r.y);
    lo[2] = fminf(lo[2], r.z); hi[2] = fmaxf(hi[2], r.z);
    if (nrm) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float c = __ldg(nrm + 3 * (size_t)p + a);
        if (!(fabsf(c) <= 1.0f)) atomicOr(status, ST_INVALID_INPUT);  // unit normals only
        else sn[a] += __float2ll_rn(__fmul_rn(c, (float)(1 << kKdNormalBits)));
      }
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xFFFFFFFFu, lo[a], off));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xFFFFFFFFu, hi[a], off));
      sn[a] += __shfl_xor_sync(0xFFFFFFFFu, sn[a], off);
    }
  }
  if (lane) return;
  int a = 0;
  float best = __fsub_rn(hi[0], lo[0]);
  for (int k = 1; k < 3; ++k) {
    const float sp = __fsub_rn(hi[k], lo[k]);
    if (sp > best) {
      best = sp;
      a = k;
    }
  }
  bool split = false;
  if (best > 0.0f) {
    double V = 0.0;
    if (nrm) {
      const double x = (double)sn[0], y = (double)sn[1], z = (double)sn[2];
      const double r = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
      const double mm = __dmul_rn(__dmul_rn((double)m, (double)m), 1099511627776.0);  // 2^40
      V = __dsub_rn(1.0, __ddiv_rn(r, mm));
    }
    split = m > thr || V > vthr;
  }
  flag[v] = split ? 1u : 0u;
  axis[v] = (uint8_t)a;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t x, uint32_t *sh) {
  uint32_t tot;
  block_excl_scan(x, &tot, sh);
  return tot;
}

// One CTA per splitting node: median by radix select, then a stable partition.
__global__ void __launch_bounds__(kKdSplitThreads) k_kd_split(
    const pg_photon *__restrict__ ph, uint32_t *__restrict__ perm, uint32_t *__restrict__ tmp,
    const uint32_t *__restrict__ list, const uint32_t *__restrict__ nb, const uint32_t *__restrict__ ne,
    const uint8_t *__restrict__ axis, const uint32_t *__restrict__ rank, uint32_t next_base,
    float *__restrict__ tau, int32_t *__restrict__ link, uint32_t *__restrict__ cnb, uint32_t *__restrict__ cne) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t sh[32];
  __shared__ uint32_t s_prefix, s_mask, s_k;
  const uint32_t v = list[blockIdx.x];
  const uint32_t b = nb[v], e = ne[v], m = e - b;
  const int a = axis[v];
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_k = m / 2;
  }
  __syncthreads();
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    hist[tid] = 0;  // 256 threads, 256 bins
    __syncthreads();
    const uint32_t prefix = s_prefix, mask = s_mask;
    for (uint32_t i = b + tid; i < e; i += kKdSplitThreads) {
      const uint32_t key = kd_key(kd_coord(ph, perm[i], a));
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t k = s_k, cum = 0;
      int dg = 0;
      for (; dg < 255; ++dg) {
        if (k < cum + hist[dg]) break;
        cum += hist[dg];
      }
      s_k = k - cum;
      s_prefix = prefix | ((uint32_t)dg << shift);
      s_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  const float sv = kd_unkey(s_prefix);
  uint32_t below = 0;
  for (uint32_t i = b + tid; i < e; i += kKdSplitThreads) below += kd_coord(ph, perm[i], a) < sv ? 1u : 0u;
  below = block_sum(below, sh);
  const float t = below ? sv : nextafterf(sv, INFINITY);
  uint32_t nl = below;
  if (!below) {
    uint32_t c = 0;
    for (uint32_t i = b + tid; i < e; i += kKdSplitThreads) c += kd_coord(ph, perm[i], a) < t ? 1u : 0u;
    nl = block_sum(c, sh);
  }
  // Stable partition into tmp[b, e), then back into perm.
  uint32_t carry_l = 0, carry_r = 0;
  for (uint32_t base = b; base < e; base += kKdSplitThreads) {
    const uint32_t i = base + tid;
    const bool live = i < e;
    uint32_t p = 0;
    uint32_t f = 0;
    if (live) {
      p = perm[i];
      f = kd_coord(ph, p, a) < t ? 1u : 0u;
    }
    uint32_t tot_l;
    const uint32_t pl = block_excl_scan(f, &tot_l, sh);
    if (live) {
      const uint32_t pr = (uint32_t)tid - pl;  // live lanes are a prefix of the chunk
      tmp[f ? b + carry_l + pl : b + nl + carry_r + pr] = p;
    }
    const uint32_t nlive = min((uint32_t)kKdSplitThreads, e - base);
    carry_l += tot_l;
    carry_r += nlive - tot_l;
  }
  __syncthreads();
  for (uint32_t i = b + tid; i < e; i += kKdSplitThreads) perm[i] = tmp[i];
  if (tid == 0) {
    const uint32_t c = 2 * rank[v];
    tau[v] = t;
    link[v] = (int32_t)(next_base + c);
    cnb[c] = b;
    cne[c] = b + nl;
    cnb[c + 1] = b + nl;
    cne[c + 1] = e;
  }
}

// Bottom-up leaf counts of one level (children of level d are level d + 1).
__global__ void k_kd_nleaf(uint32_t N, const uint32_t *__restrict__ flag, const uint32_t *__restrict__ rank,
                           const uint32_t *__restrict__ child_nleaf, uint32_t *__restrict__ nleaf) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  nleaf[v] = flag[v] ? child_nleaf[2 * rank[v]] + child_nleaf[2 * rank[v] + 1] : 1u;
}

// Top-down: children inherit offsets and voxels; leaves get their ids.
__global__ void k_kd_offsets(uint32_t N, int depth, const uint32_t *__restrict__ flag,
                             const uint32_t *__restrict__ rank, const uint32_t *__restrict__ nb,
                             const uint32_t *__restrict__ ne, const uint32_t *__restrict__ off,
                             const uint32_t *__restrict__ cell, const uint32_t *__restrict__ child_nleaf,
                             uint32_t *__restrict__ child_off, uint32_t *__restrict__ child_cell,
                             int32_t *__restrict__ link, uint64_t *__restrict__ leaf_cell,
                             int32_t *__restrict__ leaf_depth, uint32_t *__restrict__ leaf_begin,
                             uint32_t *__restrict__ leaf_end) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const uint32_t o = off[v], c = cell ? cell[v] : v;
  if (flag[v]) {
    const uint32_t k = 2 * rank[v];
    child_off[k] = o;
    child_off[k + 1] = o + child_nleaf[k];
    child_cell[k] = c;
    child_cell[k + 1] = c;
  } else {
    link[v] = ~(int32_t)o;
    leaf_cell[o] = c;
    leaf_depth[o] = depth;
    leaf_begin[o] = nb[v];
    leaf_end[o] = ne[v];
  }
}

// leaf_of per photon: the first leaf whose range ends beyond its slot.
__global__ void k_kd_leaf_of(const uint32_t *__restrict__ perm, uint32_t n, const uint32_t *__restrict__ leaf_end,
                             uint32_t L, uint32_t *__restrict__ leaf_of) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t lo = 0, hi = L;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (leaf_end[mid] > i) hi = mid;
    else lo = mid + 1;
  }
  leaf_of[perm[i]] = lo;
}

// Device-wide exclusive scans of the build: tile sums, one block over the
// tile sums, then each tile rescanned with its offset and the result handed
// to an emitter.  A tile is 4096 values (1024 threads x 4).
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

template <class Val>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint32_t N, Val f, uint32_t *__restrict__ partial) {
  __shared__ uint32_t sh[32];
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) s += base + j < N ? f(base + j) : 0u;
  uint32_t tot;
  block_excl_scan(s, &tot, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t nt, uint32_t *__restrict__ partial,
                                                        uint32_t *__restrict__ total) {
  __shared__ uint32_t sh[32];
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < nt; b0 += blockDim.x) {
    const uint32_t b = b0 + threadIdx.x;
    uint32_t tot;
    const uint32_t x = b < nt ? partial[b] : 0u;
    const uint32_t p = block_excl_scan(x, &tot, sh);
    if (b < nt) partial[b] = carry + p;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class Val, class Emit>
__global__ void __launch_bounds__(kScanThreads) k_scan_emit(uint32_t N, Val f, const uint32_t *__restrict__ partial,
                                                           Emit e) {
  __shared__ uint32_t sh[32];
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < N ? f(base + j) : 0u;
    s += v[j];
  }
  uint32_t tot;
  uint32_t p = partial[blockIdx.x] + block_excl_scan(s, &tot, sh);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < N) e(base + j, p, v[j]);
    p += v[j];
  }
}

struct FlagVal {
  const uint32_t *flag;
  __device__ uint32_t operator()(uint32_t i) const { return flag[i]; }
};
struct RankEmit {  // rank of every node, and the list of splitting nodes
  uint32_t *rank, *list;
  __device__ void operator()(uint32_t i, uint32_t p, uint32_t v) const {
    rank[i] = p;
    if (v) list[p] = i;
  }
};
struct OffEmit {
  uint32_t *off;
  __device__ void operator()(uint32_t i, uint32_t p, uint32_t) const { off[i] = p; }
};
struct NonEmptyVal {
  const uint32_t *b, *e;
  __device__ uint32_t operator()(uint32_t i) const { return e[i] > b[i] ? 1u : 0u; }
};
struct SlotEmit {  // map slots of the leaves with photons
  uint32_t *active;
  int32_t *slot;
  __device__ void operator()(uint32_t i, uint32_t p, uint32_t v) const {
    slot[i] = v ? (int32_t)p : -1;
    if (v) active[p] = i;
  }
};

// partial: ceil(N / kScanTile) words of scratch; *total gets the sum.
template <class Val, class Emit>
pg_status scan_emit(pg_ctx *ctx, uint32_t N, Val f, Emit e, uint32_t *partial, uint32_t *total) {
  cudaStream_t st = ctx->stream;
  if (N == 0) {
    PG_CUDA(cudaMemsetAsync(total, 0, 4, st));
    return PG_OK;
  }
  const uint32_t nt = ceil_div(N, kScanTile);
  k_scan_tiles<<<nt, kScanThreads, 0, st>>>(N, f, partial), PG_COUNT(ctx);
  k_scan_partials<<<1, 1024, 0, st>>>(nt, partial, total), PG_COUNT(ctx);
  k_scan_emit<<<nt, kScanThreads, 0, st>>>(N, f, partial, e), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

// Per-level node arrays of the build (device), freed at the end.
struct KdLevel {
  uint32_t N = 0, S = 0;
  uint32_t *nb = nullptr, *ne = nullptr, *flag = nullptr, *rank = nullptr, *list = nullptr;
  uint32_t *nleaf = nullptr, *off = nullptr, *cell = nullptr;
  uint8_t *axis = nullptr;
  float *tau = nullptr;
  int32_t *link = nullptr;
  void *block = nullptr;
  size_t bytes = 0;
};

pg_status kd_level_alloc(pg_ctx *ctx, KdLevel &lv, uint32_t N) {
  lv.N = N;
  const size_t b4 = align256(4ull * N), b1 = align256(N);
  lv.bytes = 10 * b4 + b1;
  PG_TRY(ctx_alloc(ctx, lv.bytes, &lv.block));
  uint8_t *q = (uint8_t *)lv.block;
  lv.nb = (uint32_t *)q; q += b4;
  lv.ne = (uint32_t *)q; q += b4;
  lv.flag = (uint32_t *)q; q += b4;
  lv.rank = (uint32_t *)q; q += b4;
  lv.list = (uint32_t *)q; q += b4;
  lv.nleaf = (uint32_t *)q; q += b4;
  lv.off = (uint32_t *)q; q += b4;
  lv.cell = (uint32_t *)q; q += b4;
  lv.tau = (float *)q; q += b4;
  lv.link = (int32_t *)q; q += b4;
  lv.axis = q;
  PG_CUDA(cudaMemsetAsync(lv.tau, 0, 4ull * N, ctx->stream));
  PG_CUDA(cudaMemsetAsync(lv.link, 0xFF, 4ull * N, ctx->stream));
  return PG_OK;
}

}  // namespace

pg_status build_grid_kd(pg_ctx *ctx, const pg_photon *d_ph, const float *d_nrm, uint64_t n64, const pg_kd_params *p,
                        Grid *g) {
  cudaStream_t st = ctx->stream;
  const uint32_t n = (uint32_t)n64, R = (uint32_t)p->resolution, C = R * R * R;
  const int maxd = p->max_depth;
  g->kd = 1;
  g->kd_R = R;
  g->n = n;
  g->D = maxd;
  g->min_depth = 0;
  g->thr = p->split_threshold;
  g->n_scenes = 1;
  g->scene_levels = 0;
  g->lut = nullptr;
  g->lut_depth = 0;
  for (int a = 0; a < 3; ++a) {
    g->lo[a] = p->lo[a];
    g->hi[a] = p->hi[a];
    g->scale[a] = (float)((double)R / ((double)p->hi[a] - (double)p->lo[a]));
  }
  KdView kv;
  memset(&kv, 0, sizeof(kv));
  for (int a = 0; a < 3; ++a) {
    kv.lo[a] = g->lo[a];
    kv.scale[a] = g->scale[a];
  }
  kv.R = R;

  // Scratch: voxel codes (ping-pong), sort values and histograms, the partition buffer.
  int bits = 0;
  while ((1ull << bits) < C) ++bits;
  const int passes = (bits + 7) / 8;
  const uint32_t nblocks = n ? ceil_div(n, kSortTile) : 0;
  const size_t s_k = align256(8ull * n), s_v = align256(4ull * n), s_h = align256(4ull * kRadix * (nblocks + 1));
  const size_t s_dt = align256(4 * kRadix), s_c = 256;
  // Scan tile sums: a scan covers at most 2^31 values (nodes or leaves).
  const size_t s_p = align256(4ull * ((1ull << 31) / kScanTile + 1));
  const size_t scratch_bytes = 3 * s_k + 3 * s_v + s_h + s_dt + s_c + s_p;
  void *scratch = nullptr;
  PG_TRY(ctx_alloc(ctx, scratch_bytes, &scratch));
  std::vector<KdLevel> levels;
  struct Guard {
    pg_ctx *c; void *p; size_t b; std::vector<KdLevel> *lv;
    ~Guard() {
      ctx_free(c, p, b);
      for (auto &l : *lv) ctx_free(c, l.block, l.bytes);
    }
  } guard{ctx, scratch, scratch_bytes, &levels};
  uint8_t *q = (uint8_t *)scratch;
  uint64_t *codes = (uint64_t *)q; q += s_k;
  uint64_t *kA = (uint64_t *)q; q += s_k;
  uint64_t *kB = (uint64_t *)q; q += s_k;
  uint32_t *perm = (uint32_t *)q; q += s_v;
  uint32_t *vT = (uint32_t *)q; q += s_v;
  uint32_t *tmp = (uint32_t *)q; q += s_v;
  uint32_t *hist = (uint32_t *)q; q += s_h;
  uint32_t *dtot = (uint32_t *)q; q += s_dt;
  uint32_t *partial = (uint32_t *)q; q += s_p;
  uint32_t *count = (uint32_t *)q;

  const int TB = 256;
  const uint64_t *sorted = codes;
  if (n) {
    k_kd_cells<<<ceil_div(n, TB), TB, 0, st>>>(d_ph, n, kv, codes, ctx->d_status), PG_COUNT(ctx);
    if (passes == 0) {
      k_iota<<<ceil_div(n, TB), TB, 0, st>>>(perm, n), PG_COUNT(ctx);
    } else {
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      const uint64_t *kin = codes;
      const uint32_t *vin = nullptr;
      for (int ps = 0; ps < passes; ++ps) {
        uint64_t *kout = (ps & 1) ? kB : kA;
        uint32_t *vout = ((passes - 1 - ps) & 1) ? vT : perm;
        const int shift = 8 * ps;
        k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, hist, nblocks), PG_COUNT(ctx);
        k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot), PG_COUNT(ctx);
        if (ps == 0)
          k_sort_scatter<0><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                            dtot, nblocks), PG_COUNT(ctx);
        else
          k_sort_scatter<1><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                             dtot, nblocks), PG_COUNT(ctx);
        kin = kout;
        vin = vout;
      }
      sorted = kin;
    }
  }

  // Level 0: the voxel roots.
  levels.emplace_back();
  PG_TRY(kd_level_alloc(ctx, levels[0], C));
  k_kd_roots<<<ceil_div(C, TB), TB, 0, st>>>(sorted, n, C, levels[0].nb, levels[0].ne), PG_COUNT(ctx);
  uint32_t node_total = C;
  for (int d = 0;; ++d) {
    KdLevel &lv = levels[d];
    k_kd_stats<<<ceil_div((uint64_t)lv.N * 32, TB), TB, 0, st>>>(d_ph, d_nrm, perm, lv.N, lv.nb, lv.ne, d, maxd,
                                                                 p->split_threshold,
                                                                 (double)p->normal_variance_threshold, lv.flag,
                                                                 lv.axis, ctx->d_status), PG_COUNT(ctx);
    PG_TRY(scan_emit(ctx, lv.N, FlagVal{lv.flag}, RankEmit{lv.rank, lv.list}, partial, count));
    uint32_t S = 0, status = 0;
    PG_TRY(read_words(ctx, st, count, &S, ctx->d_status, &status));
    if (status & ST_INVALID_INPUT) {
      PG_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, st));
      PG_CUDA(cudaStreamSynchronize(st));
      return PG_ERR_INVALID_INPUT;
    }
    lv.S = S;
    if (S == 0) break;
    if ((uint64_t)node_total + 2ull * S >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
    levels.emplace_back();
    KdLevel &nx = levels[d + 1];
    KdLevel &cur = levels[d];  // emplace_back may have moved the vector
    PG_TRY(kd_level_alloc(ctx, nx, 2 * S));
    k_kd_split<<<S, kKdSplitThreads, 0, st>>>(d_ph, perm, tmp, cur.list, cur.nb, cur.ne, cur.axis, cur.rank,
                                              node_total, cur.tau, cur.link, nx.nb, nx.ne), PG_COUNT(ctx);
    node_total += 2 * S;
  }
  const int nlev = (int)levels.size();
  // Bottom-up leaf counts, root offsets, top-down offsets.
  for (int d = nlev - 1; d >= 0; --d) {
    KdLevel &lv = levels[d];
    k_kd_nleaf<<<ceil_div(lv.N, TB), TB, 0, st>>>(lv.N, lv.flag, lv.rank, d + 1 < nlev ? levels[d + 1].nleaf : nullptr,
                                                  lv.nleaf), PG_COUNT(ctx);
  }
  PG_TRY(scan_emit(ctx, C, FlagVal{levels[0].nleaf}, OffEmit{levels[0].off}, partial, count));
  uint32_t L = 0;
  PG_TRY(read_words(ctx, st, count, &L));

  // The handle block.
  const size_t b_codes = align256(8ull * n), b_n4 = align256(4ull * n), b_l8 = align256(8ull * L),
               b_l4 = align256(4ull * L), b_t4 = align256(4ull * node_total), b_t1 = align256(node_total),
               b_sb = 256, b_sg = 256;
  g->h.bytes = b_codes + 2 * b_n4 + b_l8 + 5 * b_l4 + 2 * b_t4 + b_t1 + 2 * b_sb + b_sg;
  PG_TRY(ctx_alloc(ctx, g->h.bytes, &g->block));
  q = (uint8_t *)g->block;
  g->codes = (uint64_t *)q; q += b_codes;
  g->perm = (uint32_t *)q; q += b_n4;
  g->leaf_of = (uint32_t *)q; q += b_n4;
  g->leaf_code = (uint64_t *)q; q += b_l8;
  g->leaf_depth = (int32_t *)q; q += b_l4;
  g->leaf_begin = (uint32_t *)q; q += b_l4;
  g->leaf_end = (uint32_t *)q; q += b_l4;
  g->active = (uint32_t *)q; q += b_l4;
  g->slot_of_leaf = (int32_t *)q; q += b_l4;
  g->kd_link = (int32_t *)q; q += b_t4;
  g->kd_tau = (float *)q; q += b_t4;
  g->kd_axis = q; q += b_t1;
  g->scene_begin = (uint32_t *)q; q += b_sb;
  g->scene_leaf_begin = (uint32_t *)q; q += b_sb;
  g->scene_geom = (float *)q;
  g->kd_nodes = node_total;
  g->L = L;
  for (int d = 0; d < nlev; ++d) {
    KdLevel &lv = levels[d];
    uint32_t *coff = d + 1 < nlev ? levels[d + 1].off : nullptr;
    uint32_t *ccell = d + 1 < nlev ? levels[d + 1].cell : nullptr;
    const uint32_t *cnl = d + 1 < nlev ? levels[d + 1].nleaf : nullptr;
    k_kd_offsets<<<ceil_div(lv.N, TB), TB, 0, st>>>(lv.N, d, lv.flag, lv.rank, lv.nb, lv.ne, lv.off,
                                                    d ? lv.cell : nullptr, cnl, coff, ccell, lv.link, g->leaf_code,
                                                    g->leaf_depth, g->leaf_begin, g->leaf_end), PG_COUNT(ctx);
  }
  uint32_t base = 0;
  for (int d = 0; d < nlev; ++d) {
    KdLevel &lv = levels[d];
    PG_CUDA(cudaMemcpyAsync(g->kd_link + base, lv.link, 4ull * lv.N, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(g->kd_tau + base, lv.tau, 4ull * lv.N, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(g->kd_axis + base, lv.axis, lv.N, cudaMemcpyDeviceToDevice, st));
    base += lv.N;
  }
  if (n) {
    PG_CUDA(cudaMemcpyAsync(g->codes, codes, 8ull * n, cudaMemcpyDeviceToDevice, st));
    PG_CUDA(cudaMemcpyAsync(g->perm, perm, 4ull * n, cudaMemcpyDeviceToDevice, st));
    k_kd_leaf_of<<<ceil_div(n, TB), TB, 0, st>>>(g->perm, n, g->leaf_end, L, g->leaf_of), PG_COUNT(ctx);
  }
  PG_TRY(scan_emit(ctx, L, NonEmptyVal{g->leaf_begin, g->leaf_end}, SlotEmit{g->active, g->slot_of_leaf}, partial,
                   count));
  uint32_t hb[2] = {0u, n}, hl[2] = {0u, L};
  float hg[6] = {g->lo[0], g->lo[1], g->lo[2], g->scale[0], g->scale[1], g->scale[2]};
  PG_CUDA(cudaMemcpyAsync(g->scene_begin, hb, 8, cudaMemcpyHostToDevice, st));
  PG_CUDA(cudaMemcpyAsync(g->scene_leaf_begin, hl, 8, cudaMemcpyHostToDevice, st));
  PG_CUDA(cudaMemcpyAsync(g->scene_geom, hg, 24, cudaMemcpyHostToDevice, st));
  PG_CUDA(cudaGetLastError());
  uint32_t A = 0;
  PG_TRY(read_words(ctx, st, count, &A));
  g->A = A;
  return PG_OK;
}

// ---------------------------------------------------------------- fixed leaf table
// Progressive iterations bin later photon batches into a grid that no longer
// splits: the batch is sorted by code like the build does, and each leaf's
// range in it is found by binary search of its start code.
namespace {

__global__ void k_leaf_ranges(const uint64_t *__restrict__ sorted, uint32_t n, const uint64_t *__restrict__ leaf_code,
                              uint32_t L, uint32_t *__restrict__ leaf_begin, uint32_t *__restrict__ leaf_end) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  leaf_begin[l] = l == 0 ? 0u : lower_bound_u64(sorted, n, leaf_code[l]);
  leaf_end[l] = l + 1 == L ? n : lower_bound_u64(sorted, n, leaf_code[l + 1]);
}

// Leaves holding photons of the batch, ascending; count in *count.
__global__ void __launch_bounds__(1024) k_batch_active(uint32_t L, const uint32_t *__restrict__ leaf_begin,
                                                       const uint32_t *__restrict__ leaf_end,
                                                       uint32_t *__restrict__ active, uint32_t *__restrict__ count) {
  __shared__ uint32_t sh[32];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < L; base += blockDim.x) {
    const uint32_t l = base + threadIdx.x;
    uint32_t tot;
    const uint32_t f = (l < L && leaf_end[l] > leaf_begin[l]) ? 1u : 0u;
    const uint32_t p = block_excl_scan(f, &tot, sh);
    if (f) active[carry + p] = l;
    carry += tot;
  }
  if (threadIdx.x == 0) *count = carry;
}

}  // namespace

pg_status bin_into_grid(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n64, Grid *view, void **scratch,
                        size_t *scratch_bytes) {
  *scratch = nullptr;
  *scratch_bytes = 0;
  if (g->n_scenes != 1 || n64 >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
  cudaStream_t st = ctx->stream;
  const uint32_t n = (uint32_t)n64, L = g->L;
  const int passes = (3 * g->D + 7) / 8;
  const uint32_t nblocks = n ? ceil_div(n, kSortTile) : 0;
  const size_t s_k = align256(8ull * n), s_v = align256(4ull * n), s_h = align256(4ull * kRadix * (nblocks + 1));
  const size_t s_dt = align256(4 * kRadix), s_l = align256(4ull * L), s_c = 256;
  const size_t bytes = 3 * s_k + 2 * s_v + s_h + s_dt + 3 * s_l + s_c;
  void *blk;
  PG_TRY(ctx_alloc(ctx, bytes, &blk));
  *scratch = blk;
  *scratch_bytes = bytes;
  uint8_t *q = (uint8_t *)blk;
  uint64_t *codes = (uint64_t *)q; q += s_k;
  uint64_t *kA = (uint64_t *)q; q += s_k;
  uint64_t *kB = (uint64_t *)q; q += s_k;
  uint32_t *perm = (uint32_t *)q; q += s_v;
  uint32_t *vT = (uint32_t *)q; q += s_v;
  uint32_t *hist = (uint32_t *)q; q += s_h;
  uint32_t *dtot = (uint32_t *)q; q += s_dt;
  uint32_t *lb = (uint32_t *)q; q += s_l;
  uint32_t *le = (uint32_t *)q; q += s_l;
  uint32_t *act = (uint32_t *)q; q += s_l;
  uint32_t *count = (uint32_t *)q;

  const int TB = 256;
  const uint64_t *sorted = codes;
  if (n) {
    k_morton<<<ceil_div(n, TB), TB, 0, st>>>(d_ph, n, geom_of(g), codes, ctx->d_status), PG_COUNT(ctx);
    if (passes == 0) {
      k_iota<<<ceil_div(n, TB), TB, 0, st>>>(perm, n), PG_COUNT(ctx);
    } else {
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      const uint64_t *kin = codes;
      const uint32_t *vin = nullptr;
      for (int ps = 0; ps < passes; ++ps) {
        uint64_t *kout = (ps & 1) ? kB : kA;
        uint32_t *vout = ((passes - 1 - ps) & 1) ? vT : perm;
        const int shift = 8 * ps;
        k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, hist, nblocks), PG_COUNT(ctx);
        k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot), PG_COUNT(ctx);
        if (ps == 0)
          k_sort_scatter<0><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                            dtot, nblocks), PG_COUNT(ctx);
        else
          k_sort_scatter<1><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                             dtot, nblocks), PG_COUNT(ctx);
        kin = kout;
        vin = vout;
      }
      sorted = kin;
    }
  }
  if (L) {
    k_leaf_ranges<<<ceil_div(L, TB), TB, 0, st>>>(sorted, n, g->leaf_code, L, lb, le), PG_COUNT(ctx);
    k_batch_active<<<1, 1024, 0, st>>>(L, lb, le, act, count), PG_COUNT(ctx);
  } else {
    PG_CUDA(cudaMemsetAsync(count, 0, 4, st));
  }
  PG_CUDA(cudaGetLastError());
  uint32_t A = 0, status = 0;
  PG_TRY(read_words(ctx, st, count, &A, ctx->d_status, &status));
  if (status & ST_INVALID_INPUT) {
    PG_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, st));
    PG_CUDA(cudaStreamSynchronize(st));
    return PG_ERR_INVALID_INPUT;
  }
  *view = *g;
  view->h.kind = 0;
  view->n = n;
  view->A = A;
  view->codes = codes;
  view->perm = perm;
  view->leaf_of = nullptr;
  view->leaf_begin = lb;
  view->leaf_end = le;
  view->active = act;
  view->block = nullptr;
  return PG_OK;
}

// A batch binned into a grid of the paper's form: each photon walks its
// voxel's tree to its leaf, the batch is sorted by leaf id, and each leaf's
// range is found by binary search of its id.
namespace {

__global__ void k_kd_batch_leaf(const pg_photon *__restrict__ ph, uint32_t n, KdView kv, uint64_t *__restrict__ keys,
                                uint32_t *status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = __ldg(reinterpret_cast<const float4 *>(ph + i));
  uint32_t bad = 0;
  keys[i] = kd_locate(kv, a.x, a.y, a.z, bad);
  if (bad) atomicOr(status, ST_INVALID_INPUT);
}

__global__ void k_leaf_ranges_ids(const uint64_t *__restrict__ sorted, uint32_t n, uint32_t L,
                                  uint32_t *__restrict__ leaf_begin, uint32_t *__restrict__ leaf_end) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  leaf_begin[l] = lower_bound_u64(sorted, n, l);
  leaf_end[l] = lower_bound_u64(sorted, n, (uint64_t)l + 1);
}

}  // namespace

pg_status bin_into_grid_kd(pg_ctx *ctx, const Grid *g, const pg_photon *d_ph, uint64_t n64, Grid *view,
                           void **scratch, size_t *scratch_bytes) {
  *scratch = nullptr;
  *scratch_bytes = 0;
  if (!g->kd || n64 >= (1ull << 31)) return PG_ERR_UNSUPPORTED;
  cudaStream_t st = ctx->stream;
  const uint32_t n = (uint32_t)n64, L = g->L;
  int bits = 0;
  while ((1ull << bits) < (uint64_t)L) ++bits;
  const int passes = (bits + 7) / 8;
  const uint32_t nblocks = n ? ceil_div(n, kSortTile) : 0;
  const size_t s_k = align256(8ull * n), s_v = align256(4ull * n), s_h = align256(4ull * kRadix * (nblocks + 1));
  const size_t s_dt = align256(4 * kRadix), s_l = align256(4ull * L), s_c = 256;
  const size_t bytes = 3 * s_k + 2 * s_v + s_h + s_dt + 3 * s_l + s_c;
  void *blk;
  PG_TRY(ctx_alloc(ctx, bytes, &blk));
  *scratch = blk;
  *scratch_bytes = bytes;
  uint8_t *q = (uint8_t *)blk;
  uint64_t *keys = (uint64_t *)q; q += s_k;
  uint64_t *kA = (uint64_t *)q; q += s_k;
  uint64_t *kB = (uint64_t *)q; q += s_k;
  uint32_t *perm = (uint32_t *)q; q += s_v;
  uint32_t *vT = (uint32_t *)q; q += s_v;
  uint32_t *hist = (uint32_t *)q; q += s_h;
  uint32_t *dtot = (uint32_t *)q; q += s_dt;
  uint32_t *lb = (uint32_t *)q; q += s_l;
  uint32_t *le = (uint32_t *)q; q += s_l;
  uint32_t *act = (uint32_t *)q; q += s_l;
  uint32_t *count = (uint32_t *)q;

  const int TB = 256;
  const uint64_t *sorted = keys;
  if (n) {
    k_kd_batch_leaf<<<ceil_div(n, TB), TB, 0, st>>>(d_ph, n, kd_view_of(g), keys, ctx->d_status), PG_COUNT(ctx);
    if (passes == 0) {
      k_iota<<<ceil_div(n, TB), TB, 0, st>>>(perm, n), PG_COUNT(ctx);
    } else {
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kScatterSmem));
      const uint64_t *kin = keys;
      const uint32_t *vin = nullptr;
      for (int ps = 0; ps < passes; ++ps) {
        uint64_t *kout = (ps & 1) ? kB : kA;
        uint32_t *vout = ((passes - 1 - ps) & 1) ? vT : perm;
        const int shift = 8 * ps;
        k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, hist, nblocks), PG_COUNT(ctx);
        k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot), PG_COUNT(ctx);
        if (ps == 0)
          k_sort_scatter<0><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                            dtot, nblocks), PG_COUNT(ctx);
        else
          k_sort_scatter<1><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, n, shift, hist,
                                                                             dtot, nblocks), PG_COUNT(ctx);
        kin = kout;
        vin = vout;
      }
      sorted = kin;
    }
  }
  if (L) {
    k_leaf_ranges_ids<<<ceil_div(L, TB), TB, 0, st>>>(sorted, n, L, lb, le), PG_COUNT(ctx);
    k_batch_active<<<1, 1024, 0, st>>>(L, lb, le, act, count), PG_COUNT(ctx);
  } else {
    PG_CUDA(cudaMemsetAsync(count, 0, 4, st));
  }
  PG_CUDA(cudaGetLastError());
  uint32_t A = 0, status = 0;
  PG_TRY(read_words(ctx, st, count, &A, ctx->d_status, &status));
  if (status & ST_INVALID_INPUT) {
    PG_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, st));
    PG_CUDA(cudaStreamSynchronize(st));
    return PG_ERR_INVALID_INPUT;
  }
  *view = *g;
  view->h.kind = 0;
  view->n = n;
  view->A = A;
  view->codes = keys;
  view->perm = perm;
  view->leaf_of = nullptr;
  view->leaf_begin = lb;
  view->leaf_end = le;
  view->active = act;
  view->block = nullptr;
  return PG_OK;
}

}  // namespace pgi

// ---------------------------------------------------------------- allocation-free sort
// Morton codes + stable radix sort with all scratch in one static device
// array (no allocation by this library, the CUDA runtime or torch), for
// callers that own every device allocation themselves.
namespace pgi {
namespace {

constexpr uint64_t kNoAllocMax = PG_NOALLOC_MAX_PHOTONS;
constexpr uint64_t kNoAllocTiles = (kNoAllocMax + kSortTile - 1) / kSortTile;
constexpr size_t kNaKeys = 8 * kNoAllocMax;              // one ping-pong key buffer
constexpr size_t kNaVals = 4 * kNoAllocMax;              // the spare value buffer
constexpr size_t kNaHist = 4 * kRadix * (kNoAllocTiles + 1);
constexpr size_t kNaBytes = 2 * kNaKeys + kNaVals + kNaHist + 4 * kRadix + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
static void *g_noalloc_ptr[kMaxDevices];
static unsigned long long g_noalloc_ctx[kMaxDevices];  // context the address belongs to (0: none yet)

// The unique id of the calling thread's current CUDA context (0 if none),
// through the driver entry points the runtime exposes (no link to libcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

pg_status current_context_id(unsigned long long *id) {
  static const CtxGetCurrentFn get_current = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? (CtxGetCurrentFn)f
               : (CtxGetCurrentFn) nullptr;
  }();
  static const CtxGetIdFn get_id = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? (CtxGetIdFn)f
               : (CtxGetIdFn) nullptr;
  }();
  *id = 0;
  if (!get_current || !get_id) return PG_ERR_UNSUPPORTED;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS) return PG_ERR_CUDA;
  if (c && get_id(c, id) != CUDA_SUCCESS) return PG_ERR_CUDA;
  return PG_OK;
}

std::mutex &noalloc_mutex() {
  static std::mutex mu;
  return mu;
}

}  // namespace
}  // namespace pgi

extern "C" pg_status pg_sort_photons_noalloc(const pg_photon *d_photons, uint64_t n, const pg_grid_params *p,
                                             uint64_t *d_codes, uint32_t *d_perm, void *cuda_stream) {
  using namespace pgi;
  if (n > kNoAllocMax) return PG_ERR_UNSUPPORTED;
  if (!p || (n && (!d_photons || !d_codes || !d_perm))) return PG_ERR_INVALID_ARG;
  if (p->max_depth < 0 || p->max_depth > 16) return PG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->lo[a]) || !isfinite(p->hi[a]) || !(p->hi[a] > p->lo[a])) return PG_ERR_INVALID_ARG;
  int dev = 0;
  PG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return PG_ERR_UNSUPPORTED;
  // Set-up, once per device and context: the device address of the static
  // scratch (the symbol itself is only a host-side stand-in).  The address
  // is kept with the id of the context it was looked up in; a call from
  // another context (a new primary context after cudaDeviceReset, say)
  // looks it up again instead of using a dead address.
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(noalloc_mutex());
    unsigned long long cid = 0;
    PG_TRY(current_context_id(&cid));
    if (!g_noalloc_ptr[dev] || cid == 0 || g_noalloc_ctx[dev] != cid) {
      void *ptr = nullptr;
      PG_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));  // makes the device's context current if none was
      PG_TRY(current_context_id(&cid));
      if (cid == 0) return PG_ERR_CUDA;
      g_noalloc_ptr[dev] = ptr;
      g_noalloc_ctx[dev] = cid;
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const uint32_t nn = (uint32_t)n;
  uint8_t *q = (uint8_t *)base;
  uint64_t *kA = (uint64_t *)q; q += kNaKeys;
  uint64_t *kB = (uint64_t *)q; q += kNaKeys;
  uint32_t *vT = (uint32_t *)q; q += kNaVals;
  uint32_t *hist = (uint32_t *)q; q += kNaHist;
  uint32_t *dtot = (uint32_t *)q; q += 4 * kRadix;
  uint32_t *status = (uint32_t *)q;
  PG_CUDA(cudaMemsetAsync(status, 0, 4, st));
  if (n == 0) return PG_OK;
  GridGeom gg;
  for (int a = 0; a < 3; ++a) {
    gg.lo[a] = p->lo[a];
    gg.scale[a] = (float)(ldexp(1.0, p->max_depth) / ((double)p->hi[a] - (double)p->lo[a]));
  }
  gg.D = p->max_depth;
  gg.top = (uint32_t)((1u << p->max_depth) - 1u);
  const int TB = 256;
  k_morton<<<ceil_div(nn, TB), TB, 0, st>>>(d_photons, nn, gg, d_codes, status);
  const int passes = (3 * p->max_depth + 7) / 8;
  if (passes == 0) {
    k_iota<<<ceil_div(nn, TB), TB, 0, st>>>(d_perm, nn);
  } else {
    PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
    PG_CUDA(cudaFuncSetAttribute(k_sort_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem));
    const uint32_t nblocks = ceil_div(nn, kSortTile);
    const uint64_t *kin = d_codes;
    const uint32_t *vin = nullptr;
    for (int ps = 0; ps < passes; ++ps) {
      uint64_t *kout = (ps & 1) ? kB : kA;
      uint32_t *vout = ((passes - 1 - ps) & 1) ? vT : d_perm;
      int shift = 8 * ps;
      k_sort_upsweep<<<nblocks, kSortThreads, 0, st>>>(kin, nn, shift, hist, nblocks);
      k_sort_scan<<<kRadix, 1024, 0, st>>>(hist, nblocks, dtot);
      if (ps == 0)
        k_sort_scatter<0><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, nn, shift, hist, dtot,
                                                                          nblocks);
      else
        k_sort_scatter<1><<<nblocks, kSortThreads, kScatterSmem, st>>>(kin, vin, kout, vout, nn, shift, hist,
                                                                           dtot, nblocks);
      kin = kout;
      vin = vout;
    }
  }
  PG_CUDA(cudaGetLastError());
  uint32_t hs = 0;
  PG_CUDA(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st));
  PG_CUDA(cudaStreamSynchronize(st));
  return (hs & ST_INVALID_INPUT) ? PG_ERR_INVALID_INPUT : PG_OK;
}
