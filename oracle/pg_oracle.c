/*
 * pg_oracle.c -- plain, slow CPU oracle of the guiding-distribution hot path
 * of Photon-Driven Neural Path Guiding (Zhu et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this file.  It shares no code, header
 * or table generator with the CUDA library; the two meet only through the
 * seeded inputs they are both given.
 *
 * Floating point is FP64 except where a floating-point value decides an
 * integer (a grid cell, a direction bin, a sampled bin): there the decision is
 * taken in the precision the GPU kernel takes it (FP32, IEEE round-to-nearest,
 * no contraction; this file is compiled with -ffp-contract=off).
 *
 * Every function cites the passage of the paper it follows.
 *
 * The convolution loops (one (leaf, output row) per iteration) and the
 * per-query sampling and evaluation loops are spread over host threads with
 * OpenMP: every output value is still the same sequential computation in the
 * same order, so results do not depend on the thread count (or_set_threads;
 * default: all cores).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_OVERFLOW = 4, OR_ERR_INVALID_INPUT = 8, OR_ERR_CAPACITY = 9 };

/* Host threads of the parallel loops (n <= 0: all cores); returns the
 * count the next parallel loop will use. */
int or_set_threads(int n) {
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
  return omp_get_max_threads();
}

/* ------------------------------------------------------------------------ */
/* a1. Voxel location (Algorithm 1, Sec. 7.1 grid).                          */
/* Per-axis cell index at depth D: t = x - lo, u = t * s in FP32 with        */
/* s = float(2^D / (hi - lo)), q = clamp(floor(u), 0, 2^D - 1).              */
/* ------------------------------------------------------------------------ */
void or_axis_scale(const float lo[3], const float hi[3], int D, float s[3]) {
  for (int a = 0; a < 3; ++a) s[a] = (float)(ldexp(1.0, D) / ((double)hi[a] - (double)lo[a]));
}

static int quantise(float x, float lo, float s, int D, uint32_t *q) {
  if (!isfinite(x)) { *q = 0; return OR_ERR_INVALID_INPUT; }
  float t = x - lo;
  float u = t * s;
  float f = floorf(u);
  double top = ldexp(1.0, D) - 1.0;
  if (f < 0.0f) f = 0.0f;
  if ((double)f > top) f = (float)top;
  *q = (uint32_t)f;
  return OR_OK;
}

/* Interleave bit b of (qx, qy, qz) to bits (3b, 3b+1, 3b+2). */
uint64_t or_morton3(uint32_t qx, uint32_t qy, uint32_t qz, int D) {
  uint64_t code = 0;
  for (int b = 0; b < D; ++b) {
    code |= (uint64_t)((qx >> b) & 1u) << (3 * b);
    code |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
    code |= (uint64_t)((qz >> b) & 1u) << (3 * b + 2);
  }
  return code;
}

int or_morton_codes(const float *pos, int64_t stride, int64_t n, const float lo[3], const float hi[3],
                    int D, uint64_t *codes) {
  float s[3];
  or_axis_scale(lo, hi, D, s);
  int st = OR_OK;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) st |= quantise(pos[i * stride + a], lo[a], s[a], D, &q[a]);
    codes[i] = or_morton3(q[0], q[1], q[2], D);
  }
  return st;
}

/* ------------------------------------------------------------------------ */
/* a2-a4. Adaptive hierarchical grid (Sec. 7.1 "Voxel subdivision";          */
/* Algorithm 1, subdivide when the photon count exceeds the threshold).      */
/* Reading: octree form -- a cell whose photon count is strictly above the   */
/* threshold and whose depth is below D splits into its 8 children, every    */
/* child is kept (empty ones too) so the leaves partition the domain.  The   */
/* topology is decided from all photons of the call, then every photon is    */
/* binned in its final leaf.  Leaves are listed in Morton order.             */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t code; uint32_t idx; } keyed;

static int cmp_keyed(const void *a, const void *b) {
  const keyed *x = (const keyed *)a, *y = (const keyed *)b;
  if (x->code != y->code) return x->code < y->code ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0); /* stable by original index */
}

typedef struct {
  const uint64_t *sorted; int D; uint32_t thr;
  int64_t cap, L;
  uint64_t *leaf_code; int32_t *leaf_depth; uint32_t *leaf_begin, *leaf_end;
} grid_ctx;

static void subdivide(grid_ctx *g, uint64_t prefix, int depth, uint32_t begin, uint32_t end) {
  uint32_t count = end - begin;
  if (count > g->thr && depth < g->D) {
    int shift = 3 * (g->D - depth - 1);
    uint32_t b = begin;
    for (uint64_t k = 0; k < 8; ++k) {
      uint64_t child = prefix * 8 + k;
      uint32_t e = b;
      while (e < end && (g->sorted[e] >> shift) == child) ++e;
      subdivide(g, child, depth + 1, b, e);
      b = e;
    }
    return;
  }
  if (g->L < g->cap) {
    g->leaf_code[g->L] = prefix << (3 * (g->D - depth));
    g->leaf_depth[g->L] = depth;
    g->leaf_begin[g->L] = begin;
    g->leaf_end[g->L] = end;
  }
  g->L++;
}

/* Returns the number of leaves L (or a negative status).  If L > cap only
 * the first cap leaves were written and the caller retries with cap >= L. */
int64_t or_build_grid(const float *ph, int64_t n, const float lo[3], const float hi[3], int D,
                      int min_depth, uint32_t thr, uint64_t *codes, uint32_t *perm, uint32_t *leaf_of,
                      int64_t cap, uint64_t *leaf_code, int32_t *leaf_depth, uint32_t *leaf_begin,
                      uint32_t *leaf_end) {
  int st = or_morton_codes(ph, 8, n, lo, hi, D, codes);
  if (st) return -st;
  keyed *k = (keyed *)malloc(sizeof(keyed) * (size_t)(n > 0 ? n : 1));
  uint64_t *sorted = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) { k[i].code = codes[i]; k[i].idx = (uint32_t)i; }
  qsort(k, (size_t)n, sizeof(keyed), cmp_keyed);
  for (int64_t i = 0; i < n; ++i) { sorted[i] = k[i].code; perm[i] = k[i].idx; }
  grid_ctx g = {sorted, D, thr, cap, 0, leaf_code, leaf_depth, leaf_begin, leaf_end};
  /* Initial regular grid (Sec. 7.1 "An initial regular grid"): all 8^min_depth
   * cells at depth min_depth, in Morton order, then recursive subdivision. */
  uint64_t ncell = (uint64_t)1 << (3 * min_depth);
  int shift = 3 * (D - min_depth);
  uint32_t b = 0;
  for (uint64_t c = 0; c < ncell; ++c) {
    uint32_t e = b;
    while (e < (uint32_t)n && (sorted[e] >> shift) == c) ++e;
    subdivide(&g, c, min_depth, b, e);
    b = e;
  }
  if (g.L <= cap) {
    for (int64_t l = 0; l < g.L; ++l)
      for (uint32_t i = leaf_begin[l]; i < leaf_end[l]; ++i) leaf_of[perm[i]] = (uint32_t)l;
  }
  free(k);
  free(sorted);
  return g.L;
}

/* ------------------------------------------------------------------------ */
/* Direction bins on the cylindrical map (Sec. 4 "Spherical function         */
/* representation": (u, v) = (z, phi)).  Rows split z in [-1, 1] into H     */
/* equal bands, columns split phi in [0, 2pi) into W equal sectors; equal    */
/* z-bands times equal phi-sectors are equal solid angles (Archimedes).      */
/* phi is measured from +x toward +y (the atan2 reading of phi=arctan(y/x)). */
/* Column boundaries are the rays (c_j, s_j) = (float cos, float sin) of     */
/* 2 pi j / W, exact at quarter turns; the column is the last boundary the    */
/* direction is not clockwise of, within its half plane.  The sign of        */
/* c_j y - s_j x is exact in FP64 (products of two floats are exact).        */
/* ------------------------------------------------------------------------ */
void or_phi_table(int W, float *c, float *s) {
  for (int j = 0; j < W; ++j) {
    if ((4 * j) % W == 0) {
      int quarter = (4 * j) / W;
      const float cc[4] = {1.0f, 0.0f, -1.0f, 0.0f}, ss[4] = {0.0f, 1.0f, 0.0f, -1.0f};
      c[j] = cc[quarter];
      s[j] = ss[quarter];
    } else {
      double th = 2.0 * M_PI * (double)j / (double)W;
      c[j] = (float)cos(th);
      s[j] = (float)sin(th);
    }
  }
}

static int not_clockwise(float c, float s, float x, float y) {
  double d = (double)c * (double)y - (double)s * (double)x;
  return d >= 0.0;
}

int or_dir_bin(float dx, float dy, float dz, int H, int W, const float *c, const float *s, int *row,
               int *col) {
  if (!isfinite(dx) || !isfinite(dy) || !isfinite(dz)) { *row = 0; *col = 0; return OR_ERR_INVALID_INPUT; }
  int i = (int)floorf(dz * (float)(H / 2)) + H / 2;
  if (i < 0) i = 0;
  if (i > H - 1) i = H - 1;
  int j = 0;
  if (!(dx == 0.0f && dy == 0.0f)) {
    int upper = dy > 0.0f || (dy == 0.0f && dx >= 0.0f);
    int j0 = upper ? 0 : W / 2, j1 = upper ? W / 2 : W;
    j = j0;
    for (int t = j0; t < j1; ++t)
      if (not_clockwise(c[t], s[t], dx, dy)) j = t;
  }
  *row = i;
  *col = j;
  return OR_OK;
}

int or_dir_bins(const float *dirs, int64_t stride, int64_t n, int H, int W, int32_t *rows, int32_t *cols) {
  float *c = (float *)malloc(sizeof(float) * W), *s = (float *)malloc(sizeof(float) * W);
  or_phi_table(W, c, s);
  int st = OR_OK;
  for (int64_t i = 0; i < n; ++i)
    st |= or_dir_bin(dirs[i * stride], dirs[i * stride + 1], dirs[i * stride + 2], H, W, c, s, &rows[i], &cols[i]);
  free(c);
  free(s);
  return st;
}

/* ------------------------------------------------------------------------ */
/* a5. Photon energy binning, Eq. (photon): Phi_{j,k} = sum of the power of  */
/* the photons in voxel j whose direction falls in bin k; the photon count  */
/* maps P_{e,t}, P_{e,t-1} and the previous-iteration map (Sec. 5 inputs).   */
/* Power is accumulated in fixed point, round(power * 2^F) (IEEE round half  */
/* to even), so every sum is exact.  "Previous iteration" photons are those  */
/* with original index < n_prev.  Each photon must satisfy                   */
/* round(power * 2^F) <= (2^63 - 1) / n, which keeps every sum below 2^63.    */
/* Outputs are dense [L][H*W] planes for all L leaves.                       */
/* ------------------------------------------------------------------------ */
int or_splat(const float *ph, int64_t n, int64_t n_prev, const uint32_t *perm, int64_t L,
             const uint32_t *leaf_begin, const uint32_t *leaf_end, int H, int W, int F,
             uint64_t *pow_cur, uint32_t *cnt_cur, uint64_t *pow_prev, uint32_t *cnt_prev) {
  int64_t HW = (int64_t)H * W;
  memset(pow_cur, 0, sizeof(uint64_t) * L * HW);
  memset(pow_prev, 0, sizeof(uint64_t) * L * HW);
  memset(cnt_cur, 0, sizeof(uint32_t) * L * HW);
  memset(cnt_prev, 0, sizeof(uint32_t) * L * HW);
  float *c = (float *)malloc(sizeof(float) * W), *s = (float *)malloc(sizeof(float) * W);
  or_phi_table(W, c, s);
  uint64_t limit = n > 0 ? (uint64_t)INT64_MAX / (uint64_t)n : 0;
  int st = OR_OK;
  for (int64_t l = 0; l < L; ++l) {
    for (uint32_t t = leaf_begin[l]; t < leaf_end[l]; ++t) {
      uint32_t p = perm[t];
      const float *r = ph + 8 * (int64_t)p;
      int row, col;
      st |= or_dir_bin(r[3], r[4], r[5], H, W, c, s, &row, &col);
      float power = r[6];
      uint64_t pfx = 0;
      if (!isfinite(power) || power < 0.0f) {
        st |= OR_ERR_INVALID_INPUT;
      } else {
        double v = ldexp((double)power, F);
        if (v >= ldexp(1.0, 63)) st |= OR_ERR_OVERFLOW;
        else {
          pfx = (uint64_t)nearbyint(v);
          if (pfx > limit) { st |= OR_ERR_OVERFLOW; pfx = 0; }
        }
      }
      int64_t k = l * HW + (int64_t)row * W + col;
      pow_cur[k] += pfx;
      cnt_cur[k] += 1;
      if ((int64_t)p < n_prev) {
        pow_prev[k] += pfx;
        cnt_prev[k] += 1;
      }
    }
  }
  free(c);
  free(s);
  return st;
}

/* ------------------------------------------------------------------------ */
/* a6. Network input (Sec. 5, F(S_{e,t}, S_{e,t-1}, P_{e,t}, P_{e,t-1},      */
/* B_{e,t}); Sec. 7.2 "normalized" raw maps).  Reading: S = Phi * HW / sum   */
/* Phi (a mean-one density; zero when the leaf has no energy), P =           */
/* log(1 + count), B = (count > 0).  Channel-last [A][H][W][5], FP64.        */
/* ------------------------------------------------------------------------ */
void or_assemble_inputs(int64_t A, int64_t HW, const uint64_t *pow_cur, const uint32_t *cnt_cur,
                        const uint64_t *pow_prev, const uint32_t *cnt_prev, double *x) {
  for (int64_t a = 0; a < A; ++a) {
    uint64_t tc = 0, tp = 0;
    for (int64_t k = 0; k < HW; ++k) { tc += pow_cur[a * HW + k]; tp += pow_prev[a * HW + k]; }
    for (int64_t k = 0; k < HW; ++k) {
      double *o = x + 5 * (a * HW + k);
      o[0] = tc ? (double)pow_cur[a * HW + k] * (double)HW / (double)tc : 0.0;
      o[1] = tp ? (double)pow_prev[a * HW + k] * (double)HW / (double)tp : 0.0;
      o[2] = log1p((double)cnt_cur[a * HW + k]);
      o[3] = log1p((double)cnt_prev[a * HW + k]);
      o[4] = cnt_cur[a * HW + k] > 0 ? 1.0 : 0.0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* a7. One convolution layer of the reconstruction CNN (Sec. 5.1), written   */
/* as the definition: out[l,y,x,o] = b[o] + sum_{ky,kx,i} w[o,ky,kx,i] *     */
/* in[l, y*stride + ky - k/2, x*stride + kx - k/2, i], zero outside the map. */
/* Channel-last activations, weights [Cout][k][k][Cin].                       */
/* ------------------------------------------------------------------------ */
/* A convolution with its taps spread `dil` pixels apart (dilated, Sec. 5.1's
 * bottleneck): output (y, x) reads input (y*stride + (ky - k/2)*dil,
 * x*stride + (kx - k/2)*dil), zero outside the map. */
void or_conv2d_dilated(const double *in, int64_t L, int Hin, int Win, int Cin, const float *w, const float *b,
                       int Cout, int k, int stride, int dil, double *out) {
  int Hout = Hin / stride, Wout = Win / stride, r = k / 2;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t l = 0; l < L; ++l)
    for (int y = 0; y < Hout; ++y)
      for (int x = 0; x < Wout; ++x)
        for (int o = 0; o < Cout; ++o) {
          double acc = (double)b[o];
          for (int ky = 0; ky < k; ++ky) {
            int iy = y * stride + (ky - r) * dil;
            if (iy < 0 || iy >= Hin) continue;
            for (int kx = 0; kx < k; ++kx) {
              int ix = x * stride + (kx - r) * dil;
              if (ix < 0 || ix >= Win) continue;
              const double *src = in + (((l * Hin + iy) * Win + ix) * (int64_t)Cin);
              const float *wk = w + (((int64_t)o * k + ky) * k + kx) * Cin;
              for (int i = 0; i < Cin; ++i) acc += (double)wk[i] * src[i];
            }
          }
          out[((l * Hout + y) * Wout + x) * (int64_t)Cout + o] = acc;
        }
}

void or_conv2d(const double *in, int64_t L, int Hin, int Win, int Cin, const float *w, const float *b,
               int Cout, int k, int stride, double *out) {
  int Hout = Hin / stride, Wout = Win / stride, pad = k / 2;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t l = 0; l < L; ++l)
    for (int y = 0; y < Hout; ++y)
      for (int x = 0; x < Wout; ++x)
        for (int o = 0; o < Cout; ++o) {
          double acc = (double)b[o];
          for (int ky = 0; ky < k; ++ky) {
            int iy = y * stride + ky - pad;
            if (iy < 0 || iy >= Hin) continue;
            for (int kx = 0; kx < k; ++kx) {
              int ix = x * stride + kx - pad;
              if (ix < 0 || ix >= Win) continue;
              const double *src = in + (((l * Hin + iy) * Win + ix) * (int64_t)Cin);
              const float *wk = w + (((int64_t)o * k + ky) * k + kx) * Cin;
              for (int i = 0; i < Cin; ++i) acc += (double)wk[i] * src[i];
            }
          }
          out[((l * Hout + y) * Wout + x) * (int64_t)Cout + o] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, written from its definition in     */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" */
/* (SC'11): ten rounds of two 32x32->64 multiplies, with the key bumped by   */
/* the Weyl constants between rounds.                                        */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* a10-a12. Guided sampling by inverse CDFs over the map, as for an         */
/* environment map (Sec. 7.3), and pdf evaluation p_guide (Eq. target_mis / */
/* mis_coef terms).                                                         */
/* For query q: leaf = last leaf whose start code <= code(position); the     */
/* four uniforms are (philox(ctr=(q_lo, q_hi, stream, 0), key=seed) >> 8) *  */
/* 2^-24.  Row i = first i with u0 < Fz[i], column j = first j with          */
/* u1 < Fphi[i][j] (FP32 tables, the precision the kernel decides in);       */
/* z = -1 + 2 (i + u2) / H, phi = 2 pi (j + u3) / W, pdf = P_ij * HW / 4pi   */
/* (p proportional to Phi / dOmega, Eq. energy_target, with dOmega = 4pi/HW). */
/* A query whose leaf has no map falls back to uniform sphere sampling       */
/* (z = 1 - 2 u0, phi = 2 pi u1, pdf 1/4pi) and its leaf id has bit 31 set.  */
/* ------------------------------------------------------------------------ */
static int64_t leaf_of_code(const uint64_t *leaf_code, int64_t L, uint64_t code) {
  int64_t lo = 0, hi = L; /* first index with leaf_code > code */
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (leaf_code[mid] <= code) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

/* Query t in leaf `leaf`: the guided sample of its map, or the uniform
 * fallback when the leaf has no valid map. */
static void sample_one(int64_t t, int64_t leaf, const int32_t *slot_of_leaf, int H, int W, const double *P,
                       const float *Fz, const float *Fphi, const uint8_t *valid, uint64_t seed, uint32_t stream,
                       double *dir, double *pdf, uint32_t *leaf_out, uint32_t *bin_out) {
  const double inv24 = ldexp(1.0, -24);
  int64_t HW = (int64_t)H * W;
  int32_t slot = slot_of_leaf[leaf];
  uint32_t ctr[4] = {(uint32_t)t, (uint32_t)((uint64_t)t >> 32), stream, 0};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  double u[4];
  for (int k = 0; k < 4; ++k) u[k] = (double)(r[k] >> 8) * inv24;
  double z, phi;
  if (slot < 0 || !valid[slot]) {
    z = 1.0 - 2.0 * u[0];
    phi = 2.0 * M_PI * u[1];
    pdf[t] = 1.0 / (4.0 * M_PI);
    leaf_out[t] = (uint32_t)leaf | 0x80000000u;
    bin_out[t] = 0xFFFFFFFFu;
  } else {
    const float *fz = Fz + (int64_t)slot * H;
    int i = 0;
    while (i < H - 1 && !((float)u[0] < fz[i])) ++i;
    const float *fp = Fphi + (int64_t)slot * HW + (int64_t)i * W;
    int j = 0;
    while (j < W - 1 && !((float)u[1] < fp[j])) ++j;
    z = -1.0 + 2.0 * ((double)i + u[2]) / (double)H;
    phi = 2.0 * M_PI * ((double)j + u[3]) / (double)W;
    pdf[t] = P[(int64_t)slot * HW + (int64_t)i * W + j] * (double)HW / (4.0 * M_PI);
    leaf_out[t] = (uint32_t)leaf;
    bin_out[t] = (uint32_t)(i * W + j);
  }
  double st = sqrt(fmax(0.0, 1.0 - z * z));
  dir[3 * t + 0] = st * cos(phi);
  dir[3 * t + 1] = st * sin(phi);
  dir[3 * t + 2] = z;
}

void or_sample(const float *pos, int64_t q, const float lo[3], const float hi[3], int D,
               const uint64_t *leaf_code, int64_t L, const int32_t *slot_of_leaf, int H, int W,
               const double *P, const float *Fz, const float *Fphi, const uint8_t *valid, uint64_t seed,
               uint32_t stream, double *dir, double *pdf, uint32_t *leaf_out, uint32_t *bin_out) {
  float s[3];
  or_axis_scale(lo, hi, D, s);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < q; ++t) {
    uint32_t qq[3];
    for (int a = 0; a < 3; ++a) quantise(pos[3 * t + a], lo[a], s[a], D, &qq[a]);
    int64_t leaf = leaf_of_code(leaf_code, L, or_morton3(qq[0], qq[1], qq[2], D));
    sample_one(t, leaf, slot_of_leaf, H, W, P, Fz, Fphi, valid, seed, stream, dir, pdf, leaf_out, bin_out);
  }
}

/* The same for queries whose leaves are given (any grid form). */
void or_sample_leaves(const int64_t *leaf, int64_t q, const int32_t *slot_of_leaf, int H, int W, const double *P,
                      const float *Fz, const float *Fphi, const uint8_t *valid, uint64_t seed, uint32_t stream,
                      double *dir, double *pdf, uint32_t *leaf_out, uint32_t *bin_out) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < q; ++t)
    sample_one(t, leaf[t], slot_of_leaf, H, W, P, Fz, Fphi, valid, seed, stream, dir, pdf, leaf_out, bin_out);
}

/* p_guide of direction t in leaf `leaf` (1/4pi without a valid map). */
static double eval_one(int64_t leaf, const float *d, const int32_t *slot_of_leaf, int H, int W, const double *P,
                       const uint8_t *valid, const float *c, const float *sn) {
  int32_t slot = slot_of_leaf[leaf];
  if (slot < 0 || !valid[slot]) return 1.0 / (4.0 * M_PI);
  int row, col;
  or_dir_bin(d[0], d[1], d[2], H, W, c, sn, &row, &col);
  return P[(int64_t)slot * H * W + (int64_t)row * W + col] * (double)H * W / (4.0 * M_PI);
}

void or_eval_pdf(const float *pos, const float *dirs, int64_t q, const float lo[3], const float hi[3],
                 int D, const uint64_t *leaf_code, int64_t L, const int32_t *slot_of_leaf, int H, int W,
                 const double *P, const uint8_t *valid, double *pdf) {
  float s[3];
  or_axis_scale(lo, hi, D, s);
  float *c = (float *)malloc(sizeof(float) * W), *sn = (float *)malloc(sizeof(float) * W);
  or_phi_table(W, c, sn);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < q; ++t) {
    uint32_t qq[3];
    for (int a = 0; a < 3; ++a) quantise(pos[3 * t + a], lo[a], s[a], D, &qq[a]);
    int64_t leaf = leaf_of_code(leaf_code, L, or_morton3(qq[0], qq[1], qq[2], D));
    pdf[t] = eval_one(leaf, dirs + 3 * t, slot_of_leaf, H, W, P, valid, c, sn);
  }
  free(c);
  free(sn);
}

void or_eval_pdf_leaves(const int64_t *leaf, const float *dirs, int64_t q, const int32_t *slot_of_leaf, int H,
                        int W, const double *P, const uint8_t *valid, double *pdf) {
  float *c = (float *)malloc(sizeof(float) * W), *sn = (float *)malloc(sizeof(float) * W);
  or_phi_table(W, c, sn);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < q; ++t) pdf[t] = eval_one(leaf[t], dirs + 3 * t, slot_of_leaf, H, W, P, valid, c, sn);
  free(c);
  free(sn);
}
