/*
 * pg.h -- C ABI of the GB300 guiding-distribution library (libpg.so).
 *
 * The library computes the guiding hot path of Photon-Driven Neural Path
 * Guiding (Zhu et al., ACM TOG 2021): photons -> adaptive hierarchical grid ->
 * per-leaf cylindrical direction histograms -> CNN reconstruction -> per-leaf
 * CDFs -> guided direction sampling and pdf evaluation at path vertices.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a pg_status; nothing throws across the ABI.
 *  - A NULL context, handle or required pointer gives PG_ERR_INVALID_ARG
 *    before any CUDA call, so argument errors cost no device work.
 *    pg_destroy(NULL), pg_budget_destroy(NULL) and pg_free(NULL) are no-ops
 *    (PG_OK).
 *  - Work is asynchronous on the context's CUDA stream (pg_create).  A call
 *    returns once its work is enqueued; results are ready after pg_sync() or
 *    any later stream-ordered operation.  The exceptions are pg_build_grid
 *    (it reads the leaf counts back, see there) and pg_export/pg_info.
 *  - Array arguments named d_* may be DEVICE pointers (used in place) or HOST
 *    pointers (pinned or pageable; the library stages them through device
 *    memory on the context stream, copies inside the call).  They are owned
 *    by the caller and must stay valid until the call's work has finished.
 *  - Handles (pg_grid, pg_hist, pg_net, pg_map, pg_tables) are owned by the
 *    library, live in device memory until pg_free(), and may be reused by
 *    any number of later calls on the same context.
 *  - Data-dependent errors found by kernels (non-finite input, fixed-point
 *    overflow) are posted to a per-context status word; pg_sync() returns and
 *    clears it.
 *  - Allocations are charged to the context's HBM budget; a call that would
 *    exceed it fails with PG_ERR_OOM and allocates nothing.
 */
#ifndef PG_H
#define PG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PG_OK = 0,
  PG_ERR_INVALID_ARG = 1,    /* null pointer, bad size or inconsistent handles */
  PG_ERR_NOT_DEVICE_PTR = 2, /* a pointer the CUDA runtime cannot classify */
  PG_ERR_OOM = 3,            /* device allocation failed or HBM budget exceeded */
  PG_ERR_OVERFLOW = 4,       /* a photon's fixed-point power exceeds (2^63-1)/n */
  PG_ERR_NOT_POW2 = 5,       /* histogram H or W not a supported power of two */
  PG_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  PG_ERR_CUDA = 7,           /* a CUDA runtime call failed */
  PG_ERR_INVALID_INPUT = 8,  /* non-finite position/direction or negative power */
  PG_ERR_UNSUPPORTED = 9     /* configuration outside what the kernels support */
} pg_status;

/* Arithmetic of the reconstruction CNN's convolutions (accumulation is FP32
 * in every case). */
/* PG_FP8_MIXED (U-Net only): E4M3 operands inside the network (the layers
 * below full resolution), BF16 at the full-resolution level, its skip
 * concatenation and the head; activation scales as for PG_FP8_E4M3. */
typedef enum { PG_FP32 = 0, PG_BF16 = 1, PG_FP8_E4M3 = 2, PG_FP8_MIXED = 3 } pg_precision;

/* One photon record, 32 bytes: hit position, unit incident direction, power
 * (the flux Delta Phi_p carried by the photon, Eq. "photon" of Sec. 4). */
typedef struct {
  float px, py, pz;
  float dx, dy, dz;
  float power;
  float pad;
} pg_photon;

/* Spatial grid parameters (Sec. 7.1).  The domain [lo, hi) is cut into a
 * regular 2^min_depth grid per axis (the paper's initial regular grid); a cell
 * holding more than split_threshold photons is split into its 8 children
 * until max_depth.  0 <= min_depth <= max_depth <= 16, min_depth <= 6. */
typedef struct {
  float lo[3], hi[3];
  int32_t max_depth;
  int32_t min_depth;
  uint32_t split_threshold;
} pg_grid_params;

typedef struct pg_ctx pg_ctx;
typedef struct pg_grid pg_grid;
typedef struct pg_hist pg_hist;
typedef struct pg_net pg_net;
typedef struct pg_map pg_map;
typedef struct pg_tables pg_tables;
typedef struct pg_mis pg_mis;
typedef struct pg_progress pg_progress;

/* ---- context ----------------------------------------------------------- */

/* Creates a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; 0 = the legacy default stream).  hbm_budget caps the
 * bytes of all live handles and call scratch (0 = no cap). */
pg_status pg_create(pg_ctx **ctx, void *cuda_stream, size_t hbm_budget);
pg_status pg_destroy(pg_ctx *ctx);
/* Rebinds the context to another stream (later calls enqueue there). */
pg_status pg_set_stream(pg_ctx *ctx, void *cuda_stream);
/* Waits for the context stream, then returns (and clears) the first error
 * any kernel posted since the last pg_sync. */
pg_status pg_sync(pg_ctx *ctx);
/* Bytes currently charged to the context's budget. */
pg_status pg_bytes_in_use(const pg_ctx *ctx, uint64_t *bytes);
/* Kernels the library has launched for this context so far (autotuning
 * candidates excluded); the difference across a region is the number of
 * kernel launches that region made. */
pg_status pg_launch_count(const pg_ctx *ctx, uint64_t *launches);

/* ---- shared HBM budget (serving) ----------------------------------------
 * One byte budget shared by several contexts, e.g. one context per serving
 * stream on the same device.  The paper has no counterpart (it renders one
 * scene at a time); this is the admission signal of a multi-request server.
 * Every handle and call scratch of an attached context is charged to the
 * shared budget as well as to the context's own hbm_budget; a call whose
 * allocation would pass either cap fails with PG_ERR_OOM having allocated
 * nothing (calls are all-or-nothing), so the caller can wait for a release
 * and retry the same call.  Caller-owned device buffers (inputs, outputs)
 * may be charged with pg_budget_charge / pg_budget_release.  All budget
 * functions are thread-safe. */
typedef struct pg_budget pg_budget;
pg_status pg_budget_create(uint64_t capacity, pg_budget **out);
/* PG_ERR_INVALID_ARG while a context is still attached. */
pg_status pg_budget_destroy(pg_budget *b);
/* Attaches ctx to b (NULL detaches).  The bytes ctx already holds move to
 * the new budget (PG_ERR_OOM, and nothing changes, if they do not fit). */
pg_status pg_ctx_attach_budget(pg_ctx *ctx, pg_budget *b);
/* Charges `bytes` if they fit (PG_ERR_OOM otherwise, nothing charged). */
pg_status pg_budget_charge(pg_budget *b, uint64_t bytes);
pg_status pg_budget_release(pg_budget *b, uint64_t bytes);
/* Blocks until `bytes` would fit or a release has happened after the
 * release count *generation (as returned by pg_budget_query or by a
 * previous wait), at most timeout_ms; PG_ERR_TIMEOUT if neither.  Updates
 * *generation to the current release count. */
pg_status pg_budget_wait(pg_budget *b, uint64_t bytes, uint64_t *generation, uint32_t timeout_ms);
pg_status pg_budget_query(const pg_budget *b, uint64_t *in_use, uint64_t *capacity, uint64_t *generation);

/* ---- a1-a4: grid ------------------------------------------------------- */

/* Voxel location and adaptive subdivision (Algorithm 1; Sec. 7.1, voxel
 * subdivision), octree form:
 *   cell index per axis  q = clamp(floor(fl32(fl32(x - lo) * s)), 0, 2^D-1),
 *                        s = fl32(2^D / (hi - lo)) computed in double;
 *   Morton code          bits (3b, 3b+1, 3b+2) = bit b of (qx, qy, qz);
 *   photons are stably sorted by code; from depth min_depth down, a cell
 *   with count > split_threshold and depth < max_depth is replaced by its 8
 *   children (empty ones kept), so the leaves partition [lo, hi).
 * d_photons: n records (device or host).  On success *out holds, in device
 * memory: the Morton-ordered leaf table (start code at depth max_depth,
 * depth, photon range in sorted order), the sort permutation (sorted slot ->
 * original index), leaf_of (original index -> leaf) and the active-leaf list
 * (leaves with >= 1 photon, in leaf order) that owns a map slot.  The call
 * synchronises the stream once to learn the leaf count.  n < 2^31. */
pg_status pg_build_grid(pg_ctx *ctx, const pg_photon *d_photons, uint64_t n,
                        const pg_grid_params *params, pg_grid **out);

/* The paper's own grid rule (Sec. 7.1 "An initial regular grid" and "Voxel
 * subdivision"; Sec. 8: R = 100, trees of depth <= 8, V_thr = 0.5).  The
 * domain is cut into R^3 voxels (cell index per axis by the rule above with
 * R cells, voxel = qx + R (qy + R qz)), and every voxel holds a binary tree:
 * a node of m photons at depth d < max_depth splits when m >= 2, its photons
 * do not all share one coordinate along the axis of largest spread (max - min
 * in FP32, first axis on ties), and m > split_threshold or the normal
 * variance V = 1 - |mean n|^2 exceeds normal_variance_threshold.  V is
 * formed in double, as 1 - ((Sx^2 + Sy^2) + Sz^2) / ((m^2) 2^40), from the
 * integer sums S of round_half_even(n * 2^20) over the node's unit normals;
 * without normals (d_normals NULL) V = 0.  The split value is the
 * floor(m/2)-th smallest coordinate s (0-based) along that axis: the left
 * child takes x < tau, tau = s, or tau = the next float above s when no
 * coordinate is below s; children keep the photons' order.  Nodes are
 * numbered level by level (voxel roots first, then two children per
 * splitting node in parent order) and leaves depth-first, left first, voxel
 * by voxel, so leaf photon ranges ascend.  d_normals: n x 3 float (device or
 * host) or NULL.  The grid serves pg_splat_photons, pg_sample_dirs,
 * pg_eval_pdf and pg_mis_*; queries find their leaf by walking their voxel's
 * tree.  For such a grid PG_GRID_CODES and PG_GRID_LEAF_CODE give voxel
 * indices, and the tree is exported by PG_GRID_KD_*.  Batched scenes and
 * progressive states use the octree form only. */
typedef struct {
  float lo[3], hi[3];
  int32_t resolution;               /* R voxels per axis, R^3 <= 2^27 */
  int32_t max_depth;                /* deepest split inside a voxel, <= 16 */
  uint32_t split_threshold;         /* M_thr */
  float normal_variance_threshold;  /* V_thr */
} pg_kd_params;

pg_status pg_build_grid_kd(pg_ctx *ctx, const pg_photon *d_photons, const float *d_normals, uint64_t n,
                           const pg_kd_params *params, pg_grid **out);

/* ---- a5: splat --------------------------------------------------------- */

/* Photon energy and count maps, Eq. (photon) and the input buffers of
 * Sec. 5: for every active leaf and bin k = row*W + col,
 *   pow_cur[k]  = sum of round_half_even(power * 2^frac_bits) (uint64),
 *   cnt_cur[k]  = number of photons,
 *   pow_prev/cnt_prev = the same over photons with original index < n_prev.
 * The direction bin: row = clamp(floor(dz * H/2) + H/2, 0, H-1); column =
 * the sector of phi = atan2(dy, dx) in [0, 2 pi) in W equal sectors, decided
 * exactly against boundary rays (float(cos 2 pi j/W), float(sin 2 pi j/W)),
 * exact on the axes; dx = dy = 0 gives column 0.  H, W powers of two,
 * 4 <= H, W <= 256, H*W <= 16384.  d_photons must be the array the grid was
 * built from.  Each photon's fixed-point power must be <= (2^63-1)/n
 * (else PG_ERR_OVERFLOW via pg_sync), so no sum can overflow. */
pg_status pg_splat_photons(pg_ctx *ctx, const pg_grid *grid, const pg_photon *d_photons,
                           uint64_t n, uint64_t n_prev, int H, int W, int frac_bits,
                           pg_hist **out);

/* ---- a6-a7: reconstruction CNN ----------------------------------------- */

/* Loads a network from a host blob (little endian): u32 magic 0x314E4750,
 * u32 arch (0 = three 3x3 convs ELU/ELU/softplus, 1 = 4-level U-Net),
 * u32 in_channels (5), u32 n_layers, u32 widths[4], u64 seed; then per layer
 * u32 {cout, cin, k, stride, act, 0}, float32 weights [cout][k][k][cin],
 * float32 bias[cout].  The blob is copied; the caller keeps ownership. */
pg_status pg_net_load(pg_ctx *ctx, const void *host_blob, size_t bytes, pg_net **out);

/* Sampling-map reconstruction (Sec. 5, Sec. 7.2): for every active leaf the
 * 5-channel input (S_t = Phi HW / sum Phi, S_{t-1} likewise, log(1 + count),
 * log(1 + count_prev), count > 0) is run through the network; *out holds the
 * non-negative softplus output y [A][H][W] (float32).  Convolutions run in
 * `precision` with FP32 accumulation. */
pg_status pg_reconstruct(pg_ctx *ctx, const pg_hist *hist, const pg_net *net,
                         pg_precision precision, pg_map **out);
/* The mixture of experts of Sec. 8 (one network per range of voxel photon
 * counts, [0,100), [100,500), [500,1000), [1000,5000), [5000,inf) in the
 * paper): the map of every active leaf comes from nets[e], where e is the
 * number of count_bounds (n_experts - 1 ascending uint32 values, host
 * memory) that are <= the leaf's photon count (the sum of its current count
 * plane).  A leaf's map is the one pg_reconstruct gives it with its expert's
 * net alone.  In BF16 with 2 to 8 U-Net experts (arch 1, equal layer
 * shapes) the leaves are grouped by expert on the device and the network
 * runs as one launch per layer over every expert's leaves, with the first
 * net's tuned launch shapes; nothing is read back to the host.  Otherwise
 * each expert with leaves runs once over its leaves, and the call reads the
 * counts back to the host (it returns after a stream synchronisation).
 * 1 <= n_experts <= 16. */
pg_status pg_reconstruct_experts(pg_ctx *ctx, const pg_hist *hist, const pg_net *const *nets, int n_experts,
                                 const uint32_t *count_bounds, pg_precision precision, pg_map **out);

/* Picks the tensor-core launch shape (CTAs per SM, pipeline stages) of every
 * convolution of `net` for `precision` by timing each feasible shape on the
 * first chunk of `hist` with CUDA events, and stores the choice in the net
 * (used by later pg_reconstruct calls with maps of the same size).  A no-op
 * for PG_FP32.  Synchronous; results of the timing runs are discarded. */
pg_status pg_autotune(pg_ctx *ctx, const pg_hist *hist, pg_net *net, pg_precision precision);
/* The launch shapes pg_autotune chose for a net (7 int32 per layer and
 * precision: CTAs per SM, stages, 128-row subtiles, operand staging mode,
 * chunk bytes, map bins tuned for, staged output stores), so that another
 * process can load them with pg_net_set_tuning instead of tuning again.
 * pg_net_get_tuning writes *needed (the count) and, when out != NULL and
 * n >= *needed, the values; pg_net_set_tuning checks the count and ranges
 * (PG_ERR_INVALID_ARG). */
pg_status pg_net_get_tuning(const pg_net *net, int32_t *out, size_t n, size_t *needed);
pg_status pg_net_set_tuning(pg_net *net, const int32_t *in, size_t n);

/* Wraps caller-provided maps y [n_maps][H][W] (float32, >= 0) as a pg_map
 * (copied), so tables can be built from maps computed elsewhere. */
pg_status pg_map_import(pg_ctx *ctx, const float *d_y, uint64_t n_maps, int H, int W,
                        pg_map **out);

/* ---- a8-a9: normalisation and CDFs ------------------------------------- */

/* Sampling map and CDFs (Eq. energy_target; Sec. 7.3: CDFs over the map
 * pixels, sampled as an environment map is): P = y / sum y per map; marginal
 * CDF over rows Fz[i] = sum_{i'<=i} m_i' / sum m with m_i = sum_j y_ij;
 * conditional CDF Fphi[i][j] = sum_{j'<=j} y_ij' / m_i ((j+1)/W for an empty
 * row).  Sums, prefixes and quotients carry about 48 significant bits (pairs
 * of float32 joined by error-free transformations), stored float32 with the
 * last entry of every CDF exactly 1.  A map with sum 0 is marked invalid
 * (uniform fallback when sampled). */
pg_status pg_build_cdf(pg_ctx *ctx, const pg_map *map, pg_tables **out);

/* ---- a10-a12: guided sampling and pdf evaluation ----------------------- */

/* For each query t < q at position d_pos[3t..3t+2]: leaf = last leaf whose
 * start code <= Morton code of the position (the a1 rule); four uniforms
 * u_k = (r_k >> 8) 2^-24 from Philox4x32-10 (key = seed, counter =
 * (t mod 2^32, t >> 32, stream_id, 0)); row = first i with u0 < Fz[i],
 * column = first j with u1 < Fphi[i][j]; z = -1 + 2 (i + u2)/H,
 * phi = 2 pi (j + u3)/W; pdf = P_ij * H W / (4 pi).  A leaf without a
 * valid map falls back to uniform sphere sampling (z = 1 - 2 u0,
 * phi = 2 pi u1, pdf = 1/(4 pi)) and its d_leaf entry has bit 31 set.
 * Outputs (caller-owned): d_dir [q][3] float32, d_pdf [q] float32, d_leaf [q]
 * uint32, d_bin [q] uint32 (row*W + col, 0xFFFFFFFF for the fallback; may be
 * NULL). */
pg_status pg_sample_dirs(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables,
                         const float *d_pos, uint64_t q, uint64_t seed, uint32_t stream_id,
                         float *d_dir, float *d_pdf, uint32_t *d_leaf, uint32_t *d_bin);

/* p_guide of direction d_dir[t] at position d_pos[t] (the guide term of
 * Eq. target_mis / mis_coef): P_k * H W / (4 pi) for the bin k of the
 * direction (the pg_splat_photons bin rule) in the map of the position's
 * leaf, 1/(4 pi) for a leaf without a valid map.  d_pdf [q] float32. */
pg_status pg_eval_pdf(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables,
                      const float *d_pos, const float *d_dir, uint64_t q, float *d_pdf);

/* ---- scene batches ------------------------------------------------------ */

/* Many independent scenes in one call sequence (the batched form of the
 * calls above).  Photons are grouped by scene: scene s owns photons
 * [scene_begin[s], scene_begin[s+1]), scene_begin[0] = 0,
 * scene_begin[S] = n, 1 <= S <= 4096.  params[s] gives scene s's domain;
 * max_depth, min_depth and split_threshold must be equal across scenes
 * (max_depth + ceil(log8 S) <= 18, min_depth + ceil(log8 S) <= 6).  The
 * scene index becomes the top bits of every code (s << 3 max_depth), so one
 * sort and one subdivision build every scene's tree exactly as it would be
 * built alone; leaves are ordered by scene, then Morton order.  Leaf depths
 * exported from a batched grid include the ceil(log8 S) scene levels. */
pg_status pg_build_grid_batched(pg_ctx *ctx, const pg_photon *d_photons, uint64_t n,
                                const uint32_t *d_scene_begin, uint32_t S,
                                const pg_grid_params *params, pg_grid **out);
/* pg_splat_photons for a batched grid: a photon of scene s counts in the
 * previous-iteration planes when its index within the scene is below
 * n_prev[s] (d_n_prev: S uint32), and the overflow bound of scene s is the
 * one it has alone, (2^63-1) / (scene_begin[s+1] - scene_begin[s]). */
pg_status pg_splat_photons_batched(pg_ctx *ctx, const pg_grid *grid, const pg_photon *d_photons,
                                   uint64_t n, const uint32_t *d_n_prev, int H, int W,
                                   int frac_bits, pg_hist **out);
/* pg_sample_dirs over a batched grid: queries of scene s are
 * [query_begin[s], query_begin[s+1]) (S+1 uint32, non-decreasing, last = q);
 * a query's Philox counter uses its index within the scene and its stream is
 * stream_ids[s], so a scene's samples are the same alone or in any batch.
 * q < 2^32. */
pg_status pg_sample_dirs_batched(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables,
                                 const float *d_pos, const uint32_t *d_query_begin, uint64_t q,
                                 uint64_t seed, const uint32_t *d_stream_ids, float *d_dir,
                                 float *d_pdf, uint32_t *d_leaf, uint32_t *d_bin);
/* pg_eval_pdf over a batched grid, queries grouped as in
 * pg_sample_dirs_batched. */
pg_status pg_eval_pdf_batched(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables,
                              const float *d_pos, const float *d_dir,
                              const uint32_t *d_query_begin, uint64_t q, float *d_pdf);

/* ---- one-sample MIS of BSDF and guide (Sec. 7.3, Eq. target_mis, mis_alpha,
 * mis_coef; Algorithm 1) ---------------------------------------------------
 * Per leaf of a single-scene grid: the sums nu_B, nu_G of bounce
 * contributions whose direction came from BSDF resp. guided sampling, their
 * counts Q_B, Q_G, and alpha, the probability of choosing BSDF sampling
 * (starts at 0.5).  The BSDF is a stand-in: a Lambertian lobe around the
 * vertex normal n (unit), p_BSDF(w) = max(0, n.w) / pi, sampled as the
 * projection of a uniform disk sample (r = sqrt(v1), phi = 2 pi v2) onto the
 * hemisphere, in the tangent frame of Duff et al. (JCGT 2017).  A vertex in
 * a leaf without a valid map uses BSDF sampling alone (alpha = 1). */
pg_status pg_mis_create(pg_ctx *ctx, const pg_grid *grid, pg_mis **out);
/* Adds q bounce records: position (q x 3), strategy (q uint8: 0 BSDF,
 * 1 guide) and contribution nu_b = L cos f (q float, finite, >= 0; else
 * PG_ERR_INVALID_INPUT via pg_sync).  Sums are FP64 atomic additions, so
 * their last bits depend on the order of the additions; counts are exact. */
pg_status pg_mis_accumulate(pg_ctx *ctx, pg_mis *mis, const pg_grid *grid, const float *d_pos,
                            const uint8_t *d_strategy, const float *d_contrib, uint64_t q);
/* Eq. mis_alpha for every leaf with Q_B >= min_count and Q_G >= min_count
 * (the paper: 50): alpha = nu_B_avg / (nu_B_avg + nu_G_avg), clamped to
 * [alpha_lo, alpha_hi] (the paper: 0.2, 0.8); other leaves keep alpha. */
pg_status pg_mis_update(pg_ctx *ctx, pg_mis *mis, uint32_t min_count, float alpha_lo, float alpha_hi);
/* Samples p_MIS = alpha p_BSDF + (1 - alpha) p_guide at q vertices (positions
 * and unit normals q x 3).  Philox4x32-10 with key = seed: counter (query
 * index, stream_id, 1) gives the selection uniform v0 (BSDF when v0 < alpha)
 * and the BSDF uniforms v1, v2; a guided sample is the one pg_sample_dirs
 * draws for the same query (counter word 3 = 0).  Outputs: direction
 * (q x 3), the mixture pdf of that direction (the guide term by the
 * pg_eval_pdf bin rule), strategy (q uint8: 0 BSDF, 1 guide). */
pg_status pg_mis_sample(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables, const pg_mis *mis,
                        const float *d_pos, const float *d_normal, uint64_t q, uint64_t seed, uint32_t stream_id,
                        float *d_dir, float *d_pdf, uint8_t *d_strategy);
/* p_MIS of given directions (q x 3) at vertices (positions, normals). */
pg_status pg_mis_eval(pg_ctx *ctx, const pg_grid *grid, const pg_tables *tables, const pg_mis *mis,
                      const float *d_pos, const float *d_normal, const float *d_dir, uint64_t q, float *d_pdf);

/* ---- progressive iterations -------------------------------------------- */

/* Progressive photon iterations (Sec. 7.1, 7.2; Algorithm 1, the photon and
 * reconstruction blocks; Sec. 8 for the constants).  Iteration t brings a
 * batch of photons (the paper doubles the batch each iteration).
 *
 * Iterations t < refine_iterations (the paper: 2) refine the grid: their
 * photons (and normals) are kept, and the grid is rebuilt from all photons
 * so far with the split threshold floor(split_c * sqrt(2^t)) (the paper:
 * c = 500), so a voxel splits on its photon count through the iterations.
 * grid_rule 0 refines by the octree rule of pg_build_grid (max_depth,
 * min_depth); grid_rule 1 by the paper's rule of pg_build_grid_kd
 * (resolution R, trees of depth max_depth, normal_variance_threshold; the
 * normals come with the batches).  The grid is fixed from then on, and later
 * batches are binned into its leaves (the a1 rule or the voxel's tree walk)
 * and dropped.
 *
 * Every leaf with photons owns a map slot.  After a refinement the leaves
 * with photons take slots 0.. in leaf order; a leaf that first receives
 * photons later takes the next free slot (the newcomers of one batch in leaf
 * order).  Each slot keeps the leaf's energy and count maps summed over all
 * iterations so far (the current planes), and, as the previous planes,
 * those sums as they stood before the last iteration that brought the leaf
 * photons.  In a refining iteration every slot counts as updated, and its
 * previous planes are the sums over the earlier iterations' photons.  The
 * fixed-point bound of pg_splat_photons applies with n = max_photons, the
 * photon total over all iterations.
 *
 * With refine_iterations = 0 the grid is the unrefined grid from the start
 * (the regular grid of depth min_depth, or R^3 voxels).  The renderer's
 * valid-voxel marking is not modelled: every leaf accumulates. */
typedef struct {
  float lo[3], hi[3];
  int32_t max_depth;          /* deepest split (octree or tree), <= 16 */
  int32_t min_depth;          /* octree: the initial regular grid, <= 6 */
  double split_c;             /* split threshold floor(split_c * sqrt(2^t)) */
  int32_t refine_iterations;  /* iterations that rebuild the grid */
  int32_t H, W, frac_bits;    /* as for pg_splat_photons */
  uint64_t max_photons;       /* photons over all iterations, < 2^31 */
  int32_t grid_rule;          /* 0 octree, 1 the paper's rule (pg_build_grid_kd) */
  int32_t resolution;         /* grid_rule 1: R voxels per axis, R^3 <= 2^27 */
  float normal_variance_threshold;  /* grid_rule 1: V_thr */
} pg_progress_params;

pg_status pg_progress_create(pg_ctx *ctx, const pg_progress_params *params, pg_progress **out);
/* Adds iteration t's batch (n records, device or host) and advances t.
 * PG_ERR_INVALID_ARG if the photon total would pass max_photons; invalid
 * positions or powers give PG_ERR_INVALID_INPUT or PG_ERR_OVERFLOW (now or
 * via pg_sync) as in pg_build_grid / pg_splat_photons.  The updated slots
 * can be read with pg_export(PG_PROGRESS_UPDATED). */
pg_status pg_progress_add_photons(pg_ctx *ctx, pg_progress *state, const pg_photon *d_photons, uint64_t n);
/* The same with the unit surface normals at the photons (n x 3 float,
 * device or host, or NULL), used by grid_rule 1 while the grid is refined:
 * either every refining batch brings normals or none does
 * (PG_ERR_INVALID_ARG otherwise). */
pg_status pg_progress_add_photons_normals(pg_ctx *ctx, pg_progress *state, const pg_photon *d_photons,
                                          const float *d_normals, uint64_t n);
/* Reconstructs the maps of the slots updated by the last add (Sec. 7.2:
 * only voxels that received photons in this batch), from their current and previous
 * planes as pg_reconstruct would; the other slots keep their maps.  Then
 * rebuilds the tables of every slot's map as pg_build_cdf does. */
pg_status pg_progress_reconstruct(pg_ctx *ctx, pg_progress *state, const pg_net *net, pg_precision precision);
/* Borrowed handles of the state (any pointer may be NULL), valid until the
 * state's next add or reconstruct call: the grid (its slot_of_leaf and
 * active list are the state's slots, so that the tables, one row per slot,
 * serve pg_sample_dirs, pg_eval_pdf and pg_mis_*; its photon arrays describe
 * the last refining iteration's photons), the slot planes ([slots][H*W];
 * pg_autotune and pg_reconstruct accept them), the maps and the tables (NULL
 * before the first reconstruct).  pg_free ignores borrowed handles. */
pg_status pg_progress_view(const pg_progress *state, const pg_grid **grid, const pg_hist **planes,
                           const pg_map **map, const pg_tables **tables);

/* ---- inspection -------------------------------------------------------- */

enum {
  PG_INFO_N_PHOTONS = 1, PG_INFO_N_LEAVES = 2, PG_INFO_N_ACTIVE = 3, PG_INFO_H = 4,
  PG_INFO_W = 5, PG_INFO_BYTES = 6, PG_INFO_MAX_DEPTH = 7, PG_INFO_N_SCENES = 8, PG_INFO_SCENE_LEVELS = 9,
  PG_INFO_ITERATION = 10,  /* progress: iterations added so far */
  PG_INFO_N_UPDATED = 11,  /* progress: slots updated by the last add */
  PG_INFO_KD_NODES = 12    /* grid of the paper's form: tree nodes, voxel roots included */
};
pg_status pg_info(const void *handle, int what, uint64_t *value);

/* Copies one array of a handle to dst (host or device), synchronously.
 * `bytes` must equal the array's size. */
enum {
  PG_GRID_CODES = 100,      /* uint64 [n]  Morton code per original photon */
  PG_GRID_PERM = 101,       /* uint32 [n]  sorted slot -> original index */
  PG_GRID_LEAF_OF = 102,    /* uint32 [n]  original index -> leaf */
  PG_GRID_LEAF_CODE = 103,  /* uint64 [L]  start code (depth max_depth) */
  PG_GRID_LEAF_DEPTH = 104, /* int32  [L] */
  PG_GRID_LEAF_BEGIN = 105, /* uint32 [L]  first sorted slot */
  PG_GRID_LEAF_END = 106,   /* uint32 [L]  one past the last sorted slot */
  PG_GRID_ACTIVE = 107,     /* uint32 [A]  active leaves, ascending */
  PG_GRID_SLOT_OF_LEAF = 108, /* int32 [L] map slot or -1 */
  PG_GRID_SCENE_LEAF_BEGIN = 109, /* uint32 [S+1] first leaf of each scene (leaves are
                                     ordered by scene), L at S; a leaf id returned by
                                     pg_sample_dirs_batched minus this is the id the
                                     scene's leaf has in its grid alone */
  PG_GRID_KD_AXIS = 110,    /* uint8 [nodes] split axis (0 x, 1 y, 2 z) */
  PG_GRID_KD_TAU = 111,     /* float [nodes] split value: left holds x[axis] < tau */
  PG_GRID_KD_LINK = 112,    /* int32 [nodes] left child, or ~leaf */
  PG_HIST_POW_CUR = 200,    /* uint64 [A][H*W] */
  PG_HIST_CNT_CUR = 201,    /* uint32 [A][H*W] */
  PG_HIST_POW_PREV = 202,   /* uint64 [A][H*W] */
  PG_HIST_CNT_PREV = 203,   /* uint32 [A][H*W] */
  PG_MAP_Y = 300,           /* float  [A][H][W] */
  PG_MIS_NU_B = 500,        /* double [L]  sum of BSDF-sampled contributions */
  PG_MIS_NU_G = 501,        /* double [L]  sum of guide-sampled contributions */
  PG_MIS_Q_B = 502,         /* uint32 [L]  BSDF-sampled bounces */
  PG_MIS_Q_G = 503,         /* uint32 [L]  guide-sampled bounces */
  PG_MIS_ALPHA = 504,       /* float  [L]  BSDF selection probability */
  PG_PROGRESS_UPDATED = 600, /* uint32 [N_UPDATED] slots updated by the last add (in leaf order) */
  PG_TAB_P = 400,           /* float  [A][H*W] */
  PG_TAB_CDF_PHI = 401,     /* float  [A][H][W] */
  PG_TAB_CDF_Z = 402,       /* float  [A][H] */
  PG_TAB_VALID = 403        /* uint8  [A] */
};
pg_status pg_export(pg_ctx *ctx, const void *handle, int what, void *dst, size_t bytes);

/* Releases any handle (grid, hist, net, map, tables, mis, progress); NULL and
 * handles borrowed from a progress state are no-ops.  The
 * memory is returned in stream order on the stream of the context that made
 * the handle, which must still exist. */
void pg_free(void *handle);

const char *pg_status_string(pg_status status);

/* ---- allocation-free variant ------------------------------------------- */

/* Largest photon count pg_sort_photons_noalloc accepts. */
#define PG_NOALLOC_MAX_PHOTONS (1u << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code that must not call cudaMalloc
 * (for example a renderer plug-in whose host application owns every device
 * allocation, or a thread that must not block on the driver's allocator).
 * It computes the first two steps of pg_build_grid -- per-photon Morton codes
 * (the pg_build_grid quantisation rule) and the stable sort permutation --
 * without allocating anything: no cudaMalloc/cudaFree, no stream-ordered
 * allocation, no library routine that allocates.  Its scratch is one static
 * device array of about 20.3 MB compiled into libpg.so, present on every GPU
 * that loads the library until the process exits.
 *   d_photons  n photon records (device memory)
 *   d_codes    [n] uint64 out, Morton code per original photon (device)
 *   d_perm     [n] uint32 out, sorted slot -> original index (device)
 *   cuda_stream  the cudaStream_t the work runs on (0 = legacy default)
 * Results equal pg_export(PG_GRID_CODES / PG_GRID_PERM) of pg_build_grid on
 * the same photons and parameters.  n > PG_NOALLOC_MAX_PHOTONS returns
 * PG_ERR_UNSUPPORTED without touching the GPU.  The call waits for its work
 * and returns PG_ERR_INVALID_INPUT if a position was not finite.
 * The first call on a device looks up the scratch's device address (with
 * that device current) and keeps it with the id of the current CUDA context;
 * the first call from any other context on that device (for example a new
 * primary context after cudaDeviceReset) looks it up again.  Make such a
 * first call before any stream capture.
 * Every call uses the same scratch array, which keeps the previous call's
 * contents (the status word is cleared at the start of each call): calls
 * that overlap on the GPU -- from several host threads or streams -- race
 * and must be serialised by the caller. */
pg_status pg_sort_photons_noalloc(const pg_photon *d_photons, uint64_t n, const pg_grid_params *params,
                                  uint64_t *d_codes, uint32_t *d_perm, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PG_H */
