// a10-a12: guided direction sampling and pdf evaluation at path vertices
// (Sec. 7.3; the p_guide term of Eq. target_mis / mis_coef).
//
// One thread per query: voxel location (the a1 rule), binary search of the
// leaf start codes (or, for a grid of the paper's form, a walk down the
// voxel's binary tree), Philox4x32-10 uniforms, then an inverse-CDF search of the
// marginal (rows) and the conditional (columns) tables, each in two rounds
// (the 8-entry segment from the table's segment summary, then the entry
// within it); the direction is
// uniform in (z, phi) inside the chosen bin, i.e. uniform in solid angle on
// the equal-area cylindrical map, and its pdf is P_ij * HW / (4 pi).
#include "pg_internal.cuh"

namespace pgi {

namespace {

struct Tab {
  const uint64_t *leaf_code;
  const uint32_t *lut;
  uint32_t lut_cells;
  int lut_shift;
  const int32_t *slot_of_leaf;
  const float *P, *Fphi, *Fz;
  const float *Sphi, *Sz;  // segment summaries (null for rows under 16 bins)
  const uint8_t *valid;
  uint32_t L;
  int H, W;
  float pdf_scale;    // HW / (4 pi)
  float pdf_uniform;  // 1 / (4 pi)
};

// Scene of query t in a batched call: the range of qbegin holding t; its
// local index restarts at 0 and its Philox stream is that scene's id, so a
// scene's samples do not depend on the batch around it.
struct QueryCtx {
  GridGeom g0;            // single-scene geometry
  const uint32_t *qbegin; // [S+1] or null
  const uint32_t *streams;
  const float *geom;      // [S][6]
  uint32_t S;
  int shift;              // 3 * spatial depth
  KdView kd;              // grid of the paper's form (link null otherwise)
};

__device__ __forceinline__ uint64_t query_code(const QueryCtx &qc, const float *pos, uint64_t t, uint64_t &local,
                                               uint32_t &stream, uint32_t &bad) {
  if (!qc.qbegin) {
    local = t;
    return position_code(qc.g0, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  }
  uint32_t lo = 0, hi = qc.S;  // last s with qbegin[s] <= t
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(qc.qbegin + mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  local = t - __ldg(qc.qbegin + lo);
  if (qc.streams) stream = __ldg(qc.streams + lo);
  GridGeom g = qc.g0;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = __ldg(qc.geom + 6 * lo + a);
    g.scale[a] = __ldg(qc.geom + 6 * lo + 3 + a);
  }
  return ((uint64_t)lo << qc.shift) | position_code(g, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
}

__global__ void k_sample(const float *__restrict__ pos, uint64_t q, QueryCtx qc, Tab tb, uint2 key, uint32_t stream,
                         float *__restrict__ dir, float *__restrict__ pdf, uint32_t *__restrict__ leaf_out,
                         uint32_t *__restrict__ bin_out, uint32_t *status) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q) return;
  uint32_t bad = 0;
  uint64_t local = t;
  uint32_t l;
  if (qc.kd.link) {
    l = kd_locate(qc.kd, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  } else {
    const uint64_t code = query_code(qc, pos, t, local, stream, bad);
    l = find_leaf_lut(tb.leaf_code, tb.L, tb.lut, tb.lut_cells, tb.lut_shift, code);
  }
  if (bad) atomicOr(status, ST_INVALID_INPUT);
  int32_t s = __ldg(tb.slot_of_leaf + l);
  uint4 r = philox4x32_10(make_uint4((uint32_t)local, (uint32_t)(local >> 32), stream, 0u), key);
  const float k24 = 5.9604644775390625e-08f;  // 2^-24
  float u0 = (float)(r.x >> 8) * k24, u1 = (float)(r.y >> 8) * k24;
  float u2 = (float)(r.z >> 8) * k24, u3 = (float)(r.w >> 8) * k24;
  float z, phi, p;
  float zp, zm;  // 1 + z and 1 - z, each formed without cancellation
  uint32_t lo, bo;
  if (s < 0 || !__ldg(tb.valid + s)) {
    z = 1.0f - 2.0f * u0;
    zp = 2.0f * (1.0f - u0);
    zm = 2.0f * u0;
    phi = 2.0f * u1;
    p = tb.pdf_uniform;
    lo = l | 0x80000000u;
    bo = 0xFFFFFFFFu;
  } else {
    const size_t HW = (size_t)tb.H * tb.W;
    const int i = first_above_seg(tb.Fz + (size_t)s * tb.H, tb.Sz ? tb.Sz + (size_t)s * (tb.H >> 3) : nullptr,
                                  tb.H, u0);
    const size_t row = (size_t)s * tb.H + i;
    const int j = first_above_seg(tb.Fphi + row * tb.W, tb.Sphi ? tb.Sphi + row * (tb.W >> 3) : nullptr, tb.W, u1);
    z = -1.0f + ((float)i + u2) * (2.0f / (float)tb.H);
    zp = ((float)i + u2) * (2.0f / (float)tb.H);
    zm = ((float)(tb.H - i) - u2) * (2.0f / (float)tb.H);
    phi = ((float)j + u3) * (2.0f / (float)tb.W);  // in half turns: the angle is pi * phi
    p = __ldg(tb.P + (size_t)s * HW + (size_t)i * tb.W + j) * tb.pdf_scale;
    lo = l;
    bo = (uint32_t)(i * tb.W + j);
  }
  // sin(theta) = sqrt((1 + z)(1 - z)) from factors each accurate to a few
  // ulps relative, so the in-plane part keeps its relative accuracy near the
  // poles (1 - z * z would lose it to cancellation); sin and cos of pi * phi
  // (the argument reduction of sincospif is exact, cheaper and more accurate
  // than reducing 2 pi-scaled radians).
  float st = sqrtf(fmaxf(0.0f, zp * zm)), sn, cs;
  sincospif(phi, &sn, &cs);
  dir[3 * t] = st * cs;
  dir[3 * t + 1] = st * sn;
  dir[3 * t + 2] = z;
  pdf[t] = p;
  leaf_out[t] = lo;
  if (bin_out) bin_out[t] = bo;
}

__global__ void k_eval(const float *__restrict__ pos, const float *__restrict__ dirs, uint64_t q, QueryCtx qc, Tab tb,
                       const float *__restrict__ phi_tab, float *__restrict__ pdf, uint32_t *status) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q) return;
  uint32_t bad = 0, stream = 0;
  uint64_t local;
  uint32_t l;
  if (qc.kd.link) {
    l = kd_locate(qc.kd, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  } else {
    const uint64_t code = query_code(qc, pos, t, local, stream, bad);
    l = find_leaf_lut(tb.leaf_code, tb.L, tb.lut, tb.lut_cells, tb.lut_shift, code);
  }
  int32_t s = __ldg(tb.slot_of_leaf + l);
  float p = tb.pdf_uniform;
  if (s >= 0 && __ldg(tb.valid + s)) {
    float dx = dirs[3 * t], dy = dirs[3 * t + 1], dz = dirs[3 * t + 2];
    int row = 0, col = 0;
    if (isfinite(dx) && isfinite(dy) && isfinite(dz)) {
      row = dir_row(dz, tb.H);
      col = dir_col(dx, dy, tb.W, phi_tab);
    } else {
      bad = 1;
    }
    p = __ldg(tb.P + (size_t)s * tb.H * tb.W + (size_t)row * tb.W + col) * tb.pdf_scale;
  }
  if (bad) atomicOr(status, ST_INVALID_INPUT);
  pdf[t] = p;
}

QueryCtx make_qc(const Grid *g, const QueryScenes &qs) {
  QueryCtx qc;
  qc.g0 = geom_of(g);
  qc.qbegin = qs.d_qbegin;
  qc.streams = qs.d_streams;
  qc.geom = g->scene_geom;
  qc.S = g->n_scenes;
  qc.shift = 3 * g->D;
  qc.kd = kd_view_of(g);
  return qc;
}

Tab make_tab(const Grid *g, const Tables *t) {
  Tab tb;
  tb.leaf_code = g->leaf_code;
  tb.lut = g->lut;
  tb.lut_cells = 1u << (3 * g->lut_depth);
  tb.lut_shift = 3 * (g->D + g->scene_levels - g->lut_depth);
  tb.slot_of_leaf = g->slot_of_leaf;
  tb.P = t->P;
  tb.Fphi = t->cdf_phi;
  tb.Fz = t->cdf_z;
  tb.Sphi = t->sum_phi;
  tb.Sz = t->sum_z;
  tb.valid = t->valid;
  tb.L = g->L;
  tb.H = t->H;
  tb.W = t->W;
  tb.pdf_scale = (float)((double)t->H * t->W / (4.0 * 3.14159265358979323846));
  tb.pdf_uniform = (float)(1.0 / (4.0 * 3.14159265358979323846));
  return tb;
}

}  // namespace

pg_status sample(pg_ctx *ctx, const Grid *g, const Tables *t, const float *d_pos, uint64_t q, uint64_t seed,
                 uint32_t stream_id, float *d_dir, float *d_pdf, uint32_t *d_leaf, uint32_t *d_bin, QueryScenes qs) {
  uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  k_sample<<<ceil_div(q, 256), 256, 0, ctx->stream>>>(d_pos, q, make_qc(g, qs), make_tab(g, t), key, stream_id, d_dir,
                                                      d_pdf, d_leaf, d_bin, ctx->d_status), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status eval_pdf(pg_ctx *ctx, const Grid *g, const Tables *t, const float *d_pos, const float *d_dir, uint64_t q,
                   float *d_pdf, QueryScenes qs) {
  const float *tab;
  PG_TRY(phi_table(ctx, t->W, &tab));
  k_eval<<<ceil_div(q, 256), 256, 0, ctx->stream>>>(d_pos, d_dir, q, make_qc(g, qs), make_tab(g, t), tab, d_pdf,
                                                    ctx->d_status), PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
