// One-sample multiple importance sampling of the BSDF and the guide (Sec.
// 7.3, Eq. target_mis, mis_alpha and mis_coef; Algorithm 1, the MIS blocks).
//
// Per leaf j the library keeps the sums nu_{j,B}, nu_{j,G} of the bounce
// contributions whose direction came from BSDF or from guided sampling, their
// counts Q_{j,B}, Q_{j,G}, and alpha_j, the probability of choosing BSDF
// sampling (0.5 until both counts reach the update threshold, then
// nu_B_avg / (nu_B_avg + nu_G_avg) clamped to [lo, hi]).  A path vertex
// samples p_MIS = alpha p_BSDF + (1 - alpha) p_guide; its pdf is evaluated
// under the whole mixture.  The BSDF is a stand-in (no renderer here): a
// Lambertian lobe around the vertex normal, p_BSDF = max(0, n.w) / pi,
// sampled by projecting a uniform disk sample onto the hemisphere.  Vertices
// in a leaf without a valid map use BSDF sampling alone.
#include "pg_internal.cuh"

namespace pgi {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// Tangent frame of a unit normal (Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin, "Building an Orthonormal Basis, Revisited", JCGT 2017).
__device__ __forceinline__ void tangent_frame(float nx, float ny, float nz, float3 &b1, float3 &b2) {
  const float sgn = copysignf(1.0f, nz);
  const float a = -1.0f / (sgn + nz);
  const float b = nx * ny * a;
  b1 = make_float3(1.0f + sgn * nx * nx * a, sgn * b, -sgn * nx);
  b2 = make_float3(b, sgn + ny * ny * a, -ny);
}

struct MisTab {
  GridGeom geom;
  const uint64_t *leaf_code;
  const uint32_t *lut;
  uint32_t lut_cells, L;
  int lut_shift;
  const int32_t *slot_of_leaf;
  const float *P, *Fphi, *Fz, *phi_tab;
  const float *Sphi, *Sz;  // segment summaries of the CDFs (null for rows under 16 bins)
  const uint8_t *valid;
  const float *alpha;
  int H, W;
  float pdf_scale;  // HW / (4 pi)
  KdView kd;        // grid of the paper's form (link null otherwise)
};

__device__ __forceinline__ uint32_t leaf_of(const MisTab &tb, float x, float y, float z, uint32_t &bad) {
  if (tb.kd.link) return kd_locate(tb.kd, x, y, z, bad);
  const uint64_t code = position_code(tb.geom, x, y, z, bad);
  return find_leaf_lut(tb.leaf_code, tb.L, tb.lut, tb.lut_cells, tb.lut_shift, code);
}

// Guide pdf of direction d in map slot s (the a12 bin rule).
__device__ __forceinline__ float guide_pdf(const MisTab &tb, int s, float dx, float dy, float dz) {
  const int row = dir_row(dz, tb.H), col = dir_col(dx, dy, tb.W, tb.phi_tab);
  return __ldg(tb.P + (size_t)s * tb.H * tb.W + (size_t)row * tb.W + col) * tb.pdf_scale;
}

__global__ void k_mis_init(double *nu_b, double *nu_g, uint32_t *q_b, uint32_t *q_g, float *alpha, uint32_t L) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  nu_b[l] = 0.0;
  nu_g[l] = 0.0;
  q_b[l] = 0u;
  q_g[l] = 0u;
  alpha[l] = 0.5f;
}

__global__ void k_mis_accumulate(const float *__restrict__ pos, const uint8_t *__restrict__ strategy,
                                 const float *__restrict__ contrib, uint64_t q, MisTab tb, double *nu_b,
                                 double *nu_g, uint32_t *q_b, uint32_t *q_g, uint32_t *status) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q) return;
  uint32_t bad = 0;
  const uint32_t l = leaf_of(tb, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  const float c = contrib[t];
  if (bad || !(c >= 0.0f) || !isfinite(c)) {
    atomicOr(status, ST_INVALID_INPUT);
    return;
  }
  if (strategy[t]) {
    atomicAdd(nu_g + l, (double)c);
    atomicAdd(q_g + l, 1u);
  } else {
    atomicAdd(nu_b + l, (double)c);
    atomicAdd(q_b + l, 1u);
  }
}

__global__ void k_mis_update(const double *__restrict__ nu_b, const double *__restrict__ nu_g,
                             const uint32_t *__restrict__ q_b, const uint32_t *__restrict__ q_g, uint32_t L,
                             uint32_t min_count, double lo, double hi, float *__restrict__ alpha) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const uint32_t nb = q_b[l], ng = q_g[l];
  if (nb < min_count || ng < min_count || nb == 0 || ng == 0) return;
  const double mb = nu_b[l] / (double)nb, mg = nu_g[l] / (double)ng;
  if (!(mb + mg > 0.0)) return;
  alpha[l] = (float)fmin(fmax(mb / (mb + mg), lo), hi);
}

__global__ void k_mis_sample(const float *__restrict__ pos, const float *__restrict__ normal, uint64_t q, MisTab tb,
                             uint2 key, uint32_t stream, float *__restrict__ dir, float *__restrict__ pdf,
                             uint8_t *__restrict__ strategy, uint32_t *status) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q) return;
  uint32_t bad = 0;
  const uint32_t l = leaf_of(tb, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  const float nx = normal[3 * t], ny = normal[3 * t + 1], nz = normal[3 * t + 2];
  if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) bad = 1;
  if (bad) atomicOr(status, ST_INVALID_INPUT);
  const int32_t s = __ldg(tb.slot_of_leaf + l);
  const bool guided = s >= 0 && __ldg(tb.valid + s);
  const float a = guided ? __ldg(tb.alpha + l) : 1.0f;
  const float k24 = 5.9604644775390625e-08f;  // 2^-24
  // Counter word 3 = 1: the selection and BSDF uniforms; word 3 = 0 gives the
  // guide's uniforms, the ones pg_sample_dirs draws for the same query.
  const uint4 rm = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), stream, 1u), key);
  const float v0 = (float)(rm.x >> 8) * k24, v1 = (float)(rm.y >> 8) * k24, v2 = (float)(rm.z >> 8) * k24;
  float dx, dy, dz;
  uint8_t st;
  if (v0 < a) {
    float3 b1, b2;
    tangent_frame(nx, ny, nz, b1, b2);
    const float r = sqrtf(v1), phi = 2.0f * v2, lz = sqrtf(fmaxf(0.0f, 1.0f - v1));  // angle pi * phi
    float sn, cs;
    sincospif(phi, &sn, &cs);
    const float lx = r * cs, ly = r * sn;
    dx = b1.x * lx + b2.x * ly + nx * lz;
    dy = b1.y * lx + b2.y * ly + ny * lz;
    dz = b1.z * lx + b2.z * ly + nz * lz;
    st = 0;
  } else {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), stream, 0u), key);
    const float u0 = (float)(r.x >> 8) * k24, u1 = (float)(r.y >> 8) * k24;
    const float u2 = (float)(r.z >> 8) * k24, u3 = (float)(r.w >> 8) * k24;
    const int i = first_above_seg(tb.Fz + (size_t)s * tb.H, tb.Sz ? tb.Sz + (size_t)s * (tb.H >> 3) : nullptr,
                                  tb.H, u0);
    const size_t row = (size_t)s * tb.H + i;
    const int j = first_above_seg(tb.Fphi + row * tb.W, tb.Sphi ? tb.Sphi + row * (tb.W >> 3) : nullptr, tb.W, u1);
    const float z = -1.0f + ((float)i + u2) * (2.0f / (float)tb.H);
    const float ph = ((float)j + u3) * (2.0f / (float)tb.W);  // angle pi * ph
    // sin(theta) from (1 + z)(1 - z), each factor formed without cancellation.
    const float zp = ((float)i + u2) * (2.0f / (float)tb.H), zm = ((float)(tb.H - i) - u2) * (2.0f / (float)tb.H);
    const float stz = sqrtf(fmaxf(0.0f, zp * zm));
    float sn, cs;
    sincospif(ph, &sn, &cs);
    dx = stz * cs;
    dy = stz * sn;
    dz = z;
    st = 1;
  }
  const float pb = fmaxf(0.0f, nx * dx + ny * dy + nz * dz) / kPi;
  const float pg = guided ? guide_pdf(tb, s, dx, dy, dz) : 0.0f;
  dir[3 * t] = dx;
  dir[3 * t + 1] = dy;
  dir[3 * t + 2] = dz;
  pdf[t] = a * pb + (1.0f - a) * pg;
  strategy[t] = st;
}

__global__ void k_mis_eval(const float *__restrict__ pos, const float *__restrict__ normal,
                           const float *__restrict__ dirs, uint64_t q, MisTab tb, float *__restrict__ pdf,
                           uint32_t *status) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q) return;
  uint32_t bad = 0;
  const uint32_t l = leaf_of(tb, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], bad);
  const float nx = normal[3 * t], ny = normal[3 * t + 1], nz = normal[3 * t + 2];
  const float dx = dirs[3 * t], dy = dirs[3 * t + 1], dz = dirs[3 * t + 2];
  if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz)) bad = 1;
  if (bad) {
    atomicOr(status, ST_INVALID_INPUT);
    pdf[t] = 0.0f;
    return;
  }
  const int32_t s = __ldg(tb.slot_of_leaf + l);
  const bool guided = s >= 0 && __ldg(tb.valid + s);
  const float a = guided ? __ldg(tb.alpha + l) : 1.0f;
  const float pb = fmaxf(0.0f, nx * dx + ny * dy + nz * dz) / kPi;
  const float pg = guided ? guide_pdf(tb, s, dx, dy, dz) : 0.0f;
  pdf[t] = a * pb + (1.0f - a) * pg;
}

MisTab make_mis_tab(const Grid *g, const Tables *t, const Mis *m, const float *phi_tab) {
  MisTab tb;
  tb.geom = geom_of(g);
  tb.leaf_code = g->leaf_code;
  tb.lut = g->lut;
  tb.lut_cells = 1u << (3 * g->lut_depth);
  tb.lut_shift = 3 * (g->D + g->scene_levels - g->lut_depth);
  tb.L = g->L;
  tb.slot_of_leaf = g->slot_of_leaf;
  tb.P = t ? t->P : nullptr;
  tb.Fphi = t ? t->cdf_phi : nullptr;
  tb.Fz = t ? t->cdf_z : nullptr;
  tb.Sphi = t ? t->sum_phi : nullptr;
  tb.Sz = t ? t->sum_z : nullptr;
  tb.valid = t ? t->valid : nullptr;
  tb.phi_tab = phi_tab;
  tb.alpha = m->alpha;
  tb.H = t ? t->H : 0;
  tb.W = t ? t->W : 0;
  tb.pdf_scale = t ? (float)((double)t->H * t->W / (4.0 * 3.14159265358979323846)) : 0.0f;
  tb.kd = kd_view_of(g);
  return tb;
}

}  // namespace

pg_status mis_init(pg_ctx *ctx, Mis *m) {
  if (m->L == 0) return PG_OK;
  k_mis_init<<<ceil_div(m->L, 256), 256, 0, ctx->stream>>>(m->nu_b, m->nu_g, m->q_b, m->q_g, m->alpha, m->L),
      PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status mis_accumulate(pg_ctx *ctx, Mis *m, const Grid *g, const float *d_pos, const uint8_t *d_strategy,
                         const float *d_contrib, uint64_t q) {
  if (q == 0) return PG_OK;
  k_mis_accumulate<<<ceil_div(q, 256), 256, 0, ctx->stream>>>(d_pos, d_strategy, d_contrib, q,
                                                              make_mis_tab(g, nullptr, m, nullptr), m->nu_b,
                                                              m->nu_g, m->q_b, m->q_g, ctx->d_status),
      PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status mis_update(pg_ctx *ctx, Mis *m, uint32_t min_count, float alpha_lo, float alpha_hi) {
  if (m->L == 0) return PG_OK;
  k_mis_update<<<ceil_div(m->L, 256), 256, 0, ctx->stream>>>(m->nu_b, m->nu_g, m->q_b, m->q_g, m->L, min_count,
                                                             (double)alpha_lo, (double)alpha_hi, m->alpha),
      PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status mis_sample(pg_ctx *ctx, const Grid *g, const Tables *t, const Mis *m, const float *d_pos,
                     const float *d_normal, uint64_t q, uint64_t seed, uint32_t stream_id, float *d_dir,
                     float *d_pdf, uint8_t *d_strategy) {
  if (q == 0) return PG_OK;
  const float *tab;
  PG_TRY(phi_table(ctx, t->W, &tab));
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  k_mis_sample<<<ceil_div(q, 256), 256, 0, ctx->stream>>>(d_pos, d_normal, q, make_mis_tab(g, t, m, tab), key,
                                                          stream_id, d_dir, d_pdf, d_strategy, ctx->d_status),
      PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

pg_status mis_eval(pg_ctx *ctx, const Grid *g, const Tables *t, const Mis *m, const float *d_pos,
                   const float *d_normal, const float *d_dir, uint64_t q, float *d_pdf) {
  if (q == 0) return PG_OK;
  const float *tab;
  PG_TRY(phi_table(ctx, t->W, &tab));
  k_mis_eval<<<ceil_div(q, 256), 256, 0, ctx->stream>>>(d_pos, d_normal, d_dir, q, make_mis_tab(g, t, m, tab), d_pdf,
                                                        ctx->d_status),
      PG_COUNT(ctx);
  PG_CUDA(cudaGetLastError());
  return PG_OK;
}

}  // namespace pgi
