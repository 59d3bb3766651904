/*
 * packuv.h -- C ABI of the PackUV-GS render step on one GB300 (sm_103a).
 *
 * The library renders Gaussians stored as texels of packed multi-scale UV
 * atlases (PackUV, arXiv 2602.23040, Sec. 4.1 "Pyramid UV Mapping" and "UV
 * Atlas Layout"; Sec. 4.2 "Fitting UV Maps Directly") with the tile-based
 * splatting rasteriser of 3DGS (Sec. 3), and returns gradients to the
 * texels (Sec. 4.2 "Objective", "Gradient Freezing", "Low Precision
 * Optimization").  One fitting iteration is the chain
 *
 *   pk_atlas_gather -> pk_project_and_sh -> pk_bin_and_sort ->
 *   pk_rasterize_fwd -> [loss] -> pk_rasterize_bwd -> pk_atlas_scatter_grad
 *
 * over every view (camera x frame) of the plan in one sequence of launches.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array arguments are raw DEVICE pointers owned by the caller; the
 *    library never frees them and never allocates device memory after
 *    pk_plan_create (which allocates none either), so every call can be
 *    captured in a CUDA graph.  Scratch lives in the caller-owned
 *    `workspace` of pk_sizes.workspace_bytes, initialised once by
 *    pk_workspace_init.
 *  - Every call only enqueues work on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream) and returns without synchronising.  Host-side
 *    argument errors return a non-zero pk_status before anything is
 *    enqueued.  Errors found on the device (capacity overflow, a mismatch of
 *    the live-texel count, non-finite splats) are recorded in the status
 *    block inside the workspace; read it with pk_read_status.  No kernel
 *    traps, asserts or spins without bound.
 *  - Pointers must be 16-byte aligned (256-byte for the workspace).
 *  - Texel channels (D = 11 + 3 (L+1)^2): 0..2 position, 3..5 log-scale,
 *    6..9 quaternion (w, x, y, z), 10 opacity logit, 11 + 3 j + c the SH
 *    coefficient j = l^2 + l + m of colour c (real SH, Condon-Shortley
 *    phase, degree L <= 3).
 *  - Gaussian g of frame f is the g-th live texel of the occupancy mask in
 *    row-major atlas order; its global index is f * N + g.
 *  - A "pair" is (view v, Gaussian g of v's frame), index v * N + g.
 *  - Images are planar per view, views concatenated: channel c of pixel
 *    (x, y) of view v is at 3 * pix_off(v) + c * W_v * H_v + y * W_v + x,
 *    with pix_off(v) = sum_{u<v} W_u H_u; per-pixel scalars at
 *    pix_off(v) + y * W_v + x.
 *  - Constants: opacity alpha = min(0.99, o exp(-q/2)); a splat is skipped
 *    at a pixel if q > 9 (the 3-sigma footprint of Alg. 1 step 5) or alpha
 *    < 1/255; compositing stops before the splat that would bring the
 *    transmittance below 1e-4.
 */
#ifndef PACKUV_H
#define PACKUV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PK_VERSION 1
#define PK_MAX_LEVELS 16
#define PK_MAX_VIEWS 4096
#define PK_RECORD_FLOATS 12  /* projected record, 48 bytes */
#define PK_GRAD2D_FLOATS 12  /* per-pair 2D gradient record, 48 bytes (9 used) */
#define PK_MAX_CHANNELS 59   /* D at SH degree 3 */

typedef struct CUstream_st *pk_stream_t; /* identical to cudaStream_t */

typedef enum pk_status {
  PK_OK = 0,
  PK_ERR_ARG = 1,         /* null/misaligned pointer, size out of range */
  PK_ERR_DESC = 2,        /* invalid atlas descriptor or view table */
  PK_ERR_CAPACITY = 3,    /* a device capacity was exceeded (device status) */
  PK_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (device status) */
  PK_ERR_CUDA = 5,        /* a CUDA runtime call failed */
  PK_ERR_UNSUPPORTED = 6, /* option not supported by this build */
  PK_ERR_TOO_LARGE = 7    /* problem larger than pk_bin_and_sort_noalloc's fixed scratch */
} pk_status;

typedef enum pk_texel_type { PK_TEXEL_F32 = 0, PK_TEXEL_F16 = 1 } pk_texel_type;

/* One pyramid level inside the atlas: stored size and origin; a rotated
 * level is stored turned 90 degrees counter-clockwise (Sec. 4.1). */
typedef struct pk_level {
  int32_t w, h, x0, y0, rotated;
} pk_level;

typedef struct pk_atlas_desc {
  int32_t atlas_w, atlas_h;        /* W_A, H_A in texels */
  int32_t num_levels;              /* 1 .. PK_MAX_LEVELS */
  pk_level level[PK_MAX_LEVELS];
  int32_t sh_degree;               /* L in 0..3 */
  int32_t frames;                  /* F atlases per launch (Sec. 4.1: one atlas per frame) */
  int32_t texel_type;              /* pk_texel_type */
} pk_atlas_desc;

/* Pinhole view: X_cam = R X + t, camera looks along +z, x right, y down
 * (Supp. "Viewer"); pixel (i, j) has centre (i + 0.5, j + 0.5). */
typedef struct pk_view {
  float R[9];                      /* row-major world->camera rotation */
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  int32_t frame;                   /* atlas frame rendered by this view */
} pk_view;

/* Which tiles of a splat's r-square (r = ceil(3 sqrt(lambda_max))) receive
 * it: every one (PK_BIN_RECT), or those its footprint q <= 9 reaches
 * (PK_BIN_ELLIPSE, the default).  Images are the same in both modes. */
typedef enum pk_bin_mode { PK_BIN_RECT = 0, PK_BIN_ELLIPSE = 1 } pk_bin_mode;

/* How the compositing kernels stage a batch of a tile's splats into shared
 * memory: every thread loads its splats' records (PK_STAGE_LOADS), or the
 * next batch's records are fetched by bulk copies on the TMA unit while the
 * current batch is composited (PK_STAGE_BULK).  Same results either way. */
typedef enum pk_stage_mode { PK_STAGE_LOADS = 0, PK_STAGE_BULK = 1 } pk_stage_mode;

typedef struct pk_options {
  int32_t tile;                    /* side of the binning tiles: 32 (0 = 32) or 16; images do not
                                      depend on it, 32 halves the entries to sort at C3 */
  float znear;                     /* cull z <= znear; default 0.01 */
  float bg[3];                     /* background colour; default 0 */
  uint64_t max_dups;               /* capacity of (pair, tile) entries; 0 = 32 * pairs; at most
                                      2^35 (a larger value is lowered to it) */
  int32_t bin_mode;                /* pk_bin_mode; default PK_BIN_ELLIPSE */
  int32_t batch;                   /* splats staged per batch by pk_rasterize_fwd: 64, 128 or
                                      256 (0 = 128); pk_autotune picks it */
  int32_t stage_fwd;               /* pk_stage_mode of pk_rasterize_fwd; default PK_STAGE_LOADS */
  int32_t stage_bwd;               /* pk_stage_mode of pk_rasterize_bwd; default PK_STAGE_LOADS */
  int32_t batch_bwd;               /* the same for pk_rasterize_bwd (0 = 128) */
  int32_t sort_bits_tile;          /* digit width of the radix passes of pk_bin_and_sort's tile sort:
                                      8 or 11 (0 = 8); pk_autotune picks it */
  int32_t sort_bits_depth;         /* ... and of its depth sort of the pairs: 8 or 11 (0 = 8) */
  int32_t count_evals;             /* 1: the compositing kernels count their (pixel, splat)
                                      evaluations into the status block (evals_fwd, evals_bwd), a
                                      measurement; 0 (default): no counter in their loops, the
                                      status fields are left at 0 */
  int32_t first_wait_polls;        /* polls of the first bounded wait on each bulk-copied batch
                                      (radix sort, and the compositing kernels in PK_STAGE_BULK):
                                      0 = the default (about 2^22); -1 = give up without polling,
                                      a hook for testing the timeout path.  Waits that drain
                                      copies already issued always keep the default. */
} pk_options;

typedef struct pk_plan pk_plan;

typedef struct pk_sizes {
  int64_t n_live;                  /* N: live texels = Gaussians per frame */
  int64_t n_gauss;                 /* F * N */
  int32_t channels;                /* D */
  int32_t n_views;                 /* V */
  int64_t n_pairs;                 /* V * N */
  int64_t n_pixels;                /* P = sum_v W_v H_v */
  int64_t n_tiles;                 /* sum_v ceil(W_v/T) ceil(H_v/T) */
  uint64_t max_dups;               /* capacity of sorted_vals */
  uint64_t workspace_bytes;
  int64_t mask_words;              /* sum_v H_v ceil(W_v/32): uint32 words of the motion masks */
  int32_t bin_kernels;             /* kernels one pk_bin_and_sort call launches on this device */
} pk_sizes;

/* Device status block (in the workspace).  flags is a bit set of
 * PK_DEV_* bits; counters describe the last call that set them. */
#define PK_DEV_CAPACITY 1u       /* bin_and_sort: entries > max_dups, emitted none */
#define PK_DEV_LIVE_MISMATCH 2u  /* gather: occupancy holds != N live texels */
#define PK_DEV_TIMEOUT 4u        /* a bounded device wait gave up */
#define PK_DEV_BOUNDS 8u         /* a data-dependent index failed its check; the access was skipped */
/* After PK_DEV_TIMEOUT or PK_DEV_BOUNDS inside pk_bin_and_sort the call
 * emits nothing: every tile range is empty, so no later call reads a
 * partly sorted list.  Flags stay set until pk_workspace_init. */
typedef struct pk_device_status {
  uint32_t flags;
  uint32_t live_seen;              /* live texels counted by the last gather (saturating) */
  uint64_t dups;                   /* entries emitted by the last bin_and_sort */
  uint64_t dups_needed;            /* entries the last bin_and_sort needed */
  uint64_t valid_pairs;            /* pairs touching at least one tile */
  uint64_t evals_fwd;              /* (pixel, splat) evaluations of the last forward (count_evals) */
  uint64_t evals_bwd;              /* ... of the last backward (count_evals) */
  double loss;                     /* last pk_l1_loss_grad / pk_photo_loss_grad value */
  double ssim;                     /* mean SSIM of the last pk_photo_loss_grad (0 after L1) */
  uint64_t nonfinite;              /* Gaussians (over all frames) with a non-finite texel value,
                                      counted by the last pk_atlas_gather; pk_project_and_sh culls
                                      every pair of such a Gaussian and pk_atlas_scatter_grad
                                      gives it a zero gradient */
} pk_device_status;

/* ------------------------------------------------------------------------ */
/* Plan and workspace                                                        */
/* ------------------------------------------------------------------------ */

/* Packed layout of K pyramid levels of an S x S base, per Sec. 4.1: the
 * level sizes follow the "Pyramid UV Mapping" equation (odd k halves N,
 * even k halves M); L0 sits at the right, L1 (rotated) and L2 on the left,
 * deeper levels rightward of L2 alternating rotated/horizontal.  Fills
 * desc->atlas_w/h, num_levels and level[]; other fields are untouched.
 * Returns PK_ERR_ARG for S < 2, K outside 1..16 or a level of size 0. */
pk_status pk_atlas_layout(int32_t S, int32_t K, pk_atlas_desc *desc);

/* Validate the descriptor (levels inside the atlas, not overlapping), the
 * views (positive sizes, frame < F, finite parameters) and n_live (the
 * pairs V * n_live must stay below 2^32: pair indices are 32-bit), and
 * build the host-side plan.  Copies everything it needs.  Allocates no
 * device memory.  On error *out is NULL. */
pk_status pk_plan_create(const pk_atlas_desc *desc, const pk_view *views, int32_t n_views,
                         int64_t n_live, const pk_options *opts, pk_plan **out);
pk_status pk_plan_sizes(const pk_plan *plan, pk_sizes *out);
/* The plan's current options (after defaults and pk_autotune). */
pk_status pk_plan_options(const pk_plan *plan, pk_options *out);
void pk_plan_destroy(pk_plan *plan);

/* Autotuning (the batching pattern of the render step): times, on the
 * caller's current inputs and on `stream`, pk_rasterize_fwd and then
 * pk_rasterize_bwd for every staging batch (64, 128, 256 splats) and keeps
 * the fastest of each, then times each kernel with both staging modes and
 * keeps the faster one per kernel, then times pk_bin_and_sort with 8- and
 * 11-bit radix digits for its depth sort and then for its tile sort and
 * keeps the faster width of each (two timed runs after one warm-up each; a
 * choice other than the defaults -- 128, plain loads, 8 bits -- must be
 * more than 2 % faster).  The choices are stored in the plan's options
 * (pk_plan_options reads them); *chosen_batch receives the forward's batch
 * (may be NULL).  The tile side changes the plan's tiles and buffers, so it
 * is not tuned here: a caller times plans of both sides and keeps one.  The
 * arguments are those of the calls; afterwards sorted_vals and tile_ranges
 * hold the records' lists (the same for every width), and image, T_final,
 * n_contrib and grad2d a forward and backward with the chosen options.
 * Synchronises `stream`; do not call it during graph capture. */
pk_status pk_autotune(pk_plan *plan, const float *records, uint32_t *sorted_vals, uint64_t *tile_ranges,
                      float *image, float *T_final, uint32_t *n_contrib, const float *dL_dimage, float *grad2d,
                      void *workspace, pk_stream_t stream, int32_t *chosen_batch);

/* Upload the plan's view tables into the workspace and clear its status
 * block.  Call once per workspace (and again after reusing the memory
 * for another plan), before any other call and outside graph capture. */
pk_status pk_workspace_init(const pk_plan *plan, void *workspace, pk_stream_t stream);

/* Copy the device status block to *out: one small kernel on `stream`
 * writes it into a small pinned, device-mapped host buffer of the plan
 * (allocated on first use, freed by pk_plan_destroy; no copy engine, so the
 * read never waits behind the caller's copies on other streams), then the
 * call synchronises `stream`.  One plan's status is read by one thread at
 * a time.  Returns PK_ERR_CAPACITY / PK_ERR_TIMEOUT when those flags are
 * set (the block is copied either way). */
pk_status pk_read_status(const pk_plan *plan, const void *workspace, pk_stream_t stream,
                         pk_device_status *out);

/* ------------------------------------------------------------------------ */
/* The render step                                                           */
/* ------------------------------------------------------------------------ */

/* a1 -- Sec. 4.2 "Fitting UV Maps Directly" (U[u,v,k] = g_i) and "Low
 * Precision Optimization" (the renderer reads the low-precision proxy).
 * atlas:   [F][D][H_A][W_A] texels of desc.texel_type (FP16 decoded to FP32).
 * occ:     [H_A][ceil(W_A/32)] uint32 occupancy bits (texel x in bit x & 31
 *          of word x >> 5); the same mask for every frame.
 * dyn:     same layout, dynamic-texel mask D_i; NULL = all dynamic.
 * soa:     out [D][F*N] float32, channel-major.
 * texel:   out [N] uint32, y * W_A + x of Gaussian g.
 * dynflag: out [N] uint8, 1 = dynamic.
 * If the mask holds a number of live texels other than N the device sets
 * PK_DEV_LIVE_MISMATCH and writes only Gaussians with index < N. */
pk_status pk_atlas_gather(const pk_plan *plan, const void *atlas, const uint32_t *occ,
                          const uint32_t *dyn, float *soa, uint32_t *texel, uint8_t *dynflag,
                          void *workspace, pk_stream_t stream);

/* a2 -- Sec. 4.2 "Covariance-Aware Gaussian Masking" and Alg. 1 steps 1-4
 * (Sigma3D = R diag(s^2) R^T, Sigma2D = J W Sigma3D W^T J^T + 0.3 I, det
 * check, lambda_max, r = ceil(3 sqrt(lambda_max))), Supp. "Viewer" for the
 * pinhole mean, Sec. 3 for opacity and SH colour.  Per pair writes the
 * 12-float record {m_x, m_y, conic_a, conic_b, conic_c, opacity, z,
 * radius, red, green, blue, 0}, conic = Sigma2D^-1 = [[a, b], [b, c]],
 * s = exp(log-scale), opacity = sigmoid(logit), colour =
 * max(0, sum_j k_j Y_j(normalize(mu - camera centre)) + 0.5).  A culled
 * pair (z <= znear, det <= 1e-7, a non-finite texel value of the Gaussian
 * -- any of its D channels -- or a non-finite result) has radius 0.
 * soa: [D][F*N] float32 from pk_atlas_gather.  records: out [V*N][12]. */
pk_status pk_project_and_sh(const pk_plan *plan, const float *soa, float *records,
                            void *workspace, pk_stream_t stream);

/* a3 -- Sec. 3 (tile-based rasteriser), Supp. "Viewer" (per-camera depth
 * order).  For each pair with radius > 0 the candidate tiles are, in FP32
 * and this order without fused multiply-add: lo = max(ceil((m - 0.5) - r),
 * 0), hi = min(floor((m - 0.5) + r), size - 1) per axis, empty if lo > hi;
 * tiles lo/T .. hi/T.  In PK_BIN_ELLIPSE mode a candidate tile receives the
 * splat only if the minimum of q = d^T conic d over the rectangle of the
 * tile's pixel centres is <= 9 (1 + 2^-12) (the 3-sigma footprint of Sec.
 * 4.2 / Alg. 1 step 5), evaluated in FP32 as: inside -> yes, else the
 * least q over the four edges with the 1-D minimiser -(b d)/c (resp. /a)
 * clamped to the edge.  Every receiving (pair, tile) becomes one entry.
 * A tile's entries are contiguous and ordered by (bits(z), pair index),
 * i.e. as a stable sort of the keys (tile << 32 | bits(z)) in emission
 * order (view, Gaussian, tile row-major) leaves them; each tile's list is
 * bit-exact by contract.  The tiles' lists follow one another in an order
 * of the library's choosing (not necessarily by tile id): read a tile's
 * list through tile_ranges.
 * records:     [V*N][12] (reads m, conic, z, radius).
 * sorted_vals: out [max_dups] uint32 pair index of each entry.
 * tile_ranges: out [n_tiles][2] uint64 [start, end) into sorted_vals (entry
 *              positions are 64-bit: a plan may hold up to 2^35 entries),
 *              8-byte aligned;
 *              global tile id = tile_off(v) + ty * ceil(W_v/T) + tx.
 * If the entries exceed max_dups the device sets PK_DEV_CAPACITY, records
 * dups_needed and emits nothing (all ranges empty). */
pk_status pk_bin_and_sort(const pk_plan *plan, const float *records, uint32_t *sorted_vals,
                          uint64_t *tile_ranges, void *workspace, pk_stream_t stream);

/* pk_bin_and_sort without a workspace.  The paper has no counterpart: this
 * is a convenience for callers that cannot give the library device memory
 * -- e.g. a renderer driven from inside another framework's frame callback,
 * where that framework owns every device allocation and allocating would
 * stall the frame, or a small tool without a device allocator.  Same
 * inputs, outputs and bit-exact result as pk_bin_and_sort; the scratch is a
 * 64 MiB array inside the library (reserved on every GPU that loads it, for
 * the life of the process), so the plan must satisfy 44 * V * N + 12 *
 * max_dups + 164 * V + about 1.7 MB <= 64 MiB (with 8-bit radix digits;
 * about 12.7 MB in place of 1.7 MB with 11-bit ones), else PK_ERR_TOO_LARGE is
 * returned and nothing is enqueued.  n_entries: out, one device uint32 --
 * the entries written; 0xFFFFFFFF if they exceeded max_dups (then nothing
 * was emitted); 0xFFFFFFFE if a bounded device wait gave up or an index
 * check failed inside the call (PK_DEV_TIMEOUT / PK_DEV_BOUNDS: nothing was
 * emitted either, every tile range is empty).  The first call on a device
 * looks up the array's address; make it before any stream capture.  Every
 * call shares the one array and leaves its contents behind (each call
 * clears its status and counters and uploads its own plan's tables before
 * use): calls whose work can overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The call hands the
 * plan's view and tile tables to the device as kernel arguments (a few
 * small launches, no host-to-device copy) and never allocates. */
pk_status pk_bin_and_sort_noalloc(const pk_plan *plan, const float *records, uint32_t *sorted_vals,
                                  uint64_t *tile_ranges, uint32_t *n_entries, pk_stream_t stream);

/* a4 -- Supp. "Viewer": C = sum_i T_i alpha_i c_i, T_i = prod_{j<i}
 * (1 - alpha_j), front to back in the order of pk_bin_and_sort, plus
 * T_final * bg.  One persistent launch over the tiles of every view.
 * image:     out [3 * P] float32 (planar per view).
 * T_final:   out [P] float32 transmittance after the last blended splat.
 * n_contrib: out [P] uint32, 1-based position within the list of the
 *            pixel's binning tile (pk_options.tile) of the last blended
 *            entry (0 = none).
 * Each CTA composites a 16 x 16 block: a 32 px tile's list is walked by the
 * four CTAs of its quadrants. */
pk_status pk_rasterize_fwd(const pk_plan *plan, const float *records, const uint32_t *sorted_vals,
                           const uint64_t *tile_ranges, float *image, float *T_final,
                           uint32_t *n_contrib, void *workspace, pk_stream_t stream);

/* a5 -- adjoint of pk_rasterize_fwd (Sec. 4.2 "Objective").  Walks each
 * pixel's list backwards from n_contrib, recovering T_i = T_{i+1} /
 * (1 - alpha_i) from T_final.  grad2d: out [V*N][12] float32, zeroed by the
 * call then accumulated; fields 0..8 are dL/d(m_x, m_y, conic_a, conic_b,
 * conic_c, opacity, red, green, blue), conic_b being the off-diagonal
 * entry counted once.  dL_dimage has the layout of image. */
pk_status pk_rasterize_bwd(const pk_plan *plan, const float *records, const uint32_t *sorted_vals,
                           const uint64_t *tile_ranges, const float *T_final,
                           const uint32_t *n_contrib, const float *dL_dimage, float *grad2d,
                           void *workspace, pk_stream_t stream);

/* pk_rasterize_bwd without the clearing of grad2d: the gradients are added
 * to what grad2d holds ([V*N][12] float32, 16-byte aligned) -- zeros left by
 * pk_rasterize_fwd_l1_clear, or an earlier backward's sums to add to.  The
 * same arguments, layouts and errors as pk_rasterize_bwd. */
pk_status pk_rasterize_bwd_accumulate(const pk_plan *plan, const float *records, const uint32_t *sorted_vals,
                                      const uint64_t *tile_ranges, const float *T_final,
                                      const uint32_t *n_contrib, const float *dL_dimage, float *grad2d,
                                      void *workspace, pk_stream_t stream);

/* a6 -- chain rule from grad2d through the projection and SH colour back to
 * the texel attributes, summed over the views of each Gaussian's frame,
 * then multiplied by D_i (Sec. 4.2 "Gradient Freezing"); the FP16 proxy is
 * passed straight through (Sec. 4.2 "Low Precision Optimization").
 * grad_atlas: [F][D][H_A][W_A] float32; the live texels are overwritten
 * (accumulate = 0) or added to (accumulate = 1); other texels untouched.
 * dynflag may be NULL (all dynamic). */
pk_status pk_atlas_scatter_grad(const pk_plan *plan, const float *soa, const float *grad2d,
                                const uint8_t *dynflag, const uint32_t *texel, float *grad_atlas,
                                int32_t accumulate, void *workspace, pk_stream_t stream);

/* Convenience: the forward of one iteration, pk_atlas_gather ->
 * pk_project_and_sh -> pk_bin_and_sort -> pk_rasterize_fwd, with the
 * arguments (and errors) of those calls; stops at the first error. */
pk_status pk_render_fwd(const pk_plan *plan, const void *atlas, const uint32_t *occ, const uint32_t *dyn,
                        float *soa, uint32_t *texel, uint8_t *dynflag, float *records, uint32_t *sorted_vals,
                        uint64_t *tile_ranges, float *image, float *T_final, uint32_t *n_contrib,
                        void *workspace, pk_stream_t stream);

/* Convenience: the backward, pk_rasterize_bwd -> pk_atlas_scatter_grad. */
pk_status pk_render_bwd(const pk_plan *plan, const float *soa, const uint8_t *dynflag, const uint32_t *texel,
                        const float *records, const uint32_t *sorted_vals, const uint64_t *tile_ranges,
                        const float *T_final, const uint32_t *n_contrib, const float *dL_dimage,
                        float *grad2d, float *grad_atlas, int32_t accumulate, void *workspace,
                        pk_stream_t stream);

/* Photometric L1 term of Sec. 4.2 "Objective": loss = mean |image - target|
 * over 3 P values (stored in the status block), dL_dimage = sign(image -
 * target) / (3 P) (0 where equal). */
pk_status pk_l1_loss_grad(const pk_plan *plan, const float *image, const float *target,
                          float *dL_dimage, void *workspace, pk_stream_t stream);

/* pk_rasterize_fwd with pk_l1_loss_grad fused into its epilogue: the same
 * image, T_final and n_contrib, the same dL_dimage bit for bit, the loss
 * in the status block (summed in another order: equal to pk_l1_loss_grad's
 * up to rounding).  Saves writing the image out and reading it back.
 * target: [3 * P] float32, planar per view like the image. */
pk_status pk_rasterize_fwd_l1(const pk_plan *plan, const float *records, const uint32_t *sorted_vals,
                              const uint64_t *tile_ranges, const float *target, float *image,
                              float *T_final, uint32_t *n_contrib, float *dL_dimage, void *workspace,
                              pk_stream_t stream);

/* pk_rasterize_fwd_l1 that also sets grad2d ([V*N][12] float32, 16-byte
 * aligned) to zero, for a following pk_rasterize_bwd_accumulate: the
 * compositing kernel clears a share of it per work item, stores that ride
 * along with its arithmetic-bound work instead of a clearing pass in front
 * of the backward (the pair is one step's forward and backward of Sec. 4.2
 * "Objective" with the L1 term).  Outputs and errors otherwise as
 * pk_rasterize_fwd_l1. */
pk_status pk_rasterize_fwd_l1_clear(const pk_plan *plan, const float *records, const uint32_t *sorted_vals,
                                    const uint64_t *tile_ranges, const float *target, float *image,
                                    float *T_final, uint32_t *n_contrib, float *dL_dimage, float *grad2d,
                                    void *workspace, pk_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Motion masks and the dynamic mask D_i                                     */
/* ------------------------------------------------------------------------ */

/* Binary motion masks (Sec. 4.2 "Optical Flow and Binary Motion Masks"):
 * M_v(p) = 1 iff the flow vector at p has magnitude > tau, then M_v <-
 * dilate(M_v; dilate_r).  The magnitude and its comparison are taken in
 * FP32 as sqrt(fx * fx + fy * fy) > tau, IEEE-rounded, without fused
 * multiply-adds; the dilation uses the (2r+1) x (2r+1) square and treats
 * pixels outside the image as still.
 * flow:      [2 * P] float32, per view planar [2][H_v][W_v] (x component
 *            plane, then y), views concatenated: component k of pixel
 *            (x, y) of view v at 2 * pix_off(v) + k * W_v * H_v + y * W_v + x.
 * mask_bits: out [pk_sizes.mask_words] uint32; view v's rows start at word
 *            sum_{u<v} H_u ceil(W_u/32), row y at + y * ceil(W_v/32), pixel
 *            x in bit x & 31 of word x >> 5; bits past W_v are 0.
 * tau:       any value but NaN; dilate_r in [0, 4096], else PK_ERR_ARG.
 * Uses the workspace's mask scratch (one mask's worth of words). */
pk_status pk_motion_mask(const pk_plan *plan, const float *flow, float tau, int32_t dilate_r,
                         uint32_t *mask_bits, void *workspace, pk_stream_t stream);

/* Dynamic mask (Sec. 4.2 "Covariance-Aware Gaussian Masking", Alg. 1 step
 * 5, and D_i = OR over cameras): Gaussian g is dynamic iff, for some view
 * v, a pixel of v's image with M_v = 1 lies in g's ellipse d^2 = (p -
 * m)^T conic (p - m) <= 9, p being the pixel centre (x + 0.5, y + 0.5) and
 * the candidates the square |p - m|_inf <= r, r = min(r_max, radius) of the
 * pair's record (r_max <= 0: no clamp).  Square and d^2 are evaluated in
 * FP32 in the order
 *   x_lo = ceil((m_x - 0.5) - r), x_hi = floor((m_x - 0.5) + r) (same in
 *   y), clamped to the image;
 *   d^2 = ((a dx) dx + (c dy) dy) + ((2 b) dy) dx, dx = (x + 0.5) - m_x,
 * without fused multiply-adds, so the result is a function of the records.
 * records:   [V*N][12] from pk_project_and_sh (culled pairs have radius 0).
 * texel:     [N] from pk_atlas_gather.
 * mask_bits: [pk_sizes.mask_words] from pk_motion_mask (same layout).
 * dyn:       in/out [H_A][ceil(W_A/32)] uint32 texel bits, the layout of
 *            pk_atlas_gather's dyn input: bit of texel[g] set for every
 *            dynamic g.  accumulate = 0 clears it first; 1 ORs into it.
 * r_max must not be NaN.  Texels of non-live texels are left as they are.
 * Uses the workspace's block-mask scratch (one bit per 32 x 32 pixels). */
pk_status pk_dynamic_mask(const pk_plan *plan, const float *records, const uint32_t *texel,
                          const uint32_t *mask_bits, float r_max, uint32_t *dyn, int32_t accumulate,
                          void *workspace, pk_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Low-precision proxy (Sec. 4.2 "Low Precision Optimization", Supp. "Video  */
/* Coding")                                                                  */
/* ------------------------------------------------------------------------ */

/* Channel c of every texel is quantised uniformly to K_c bits over its
 * range [lo_c, hi_c]: K_c = 16 for the position channels 0..2, 8 for all
 * others; Delta_c = (hi_c - lo_c) / (2^K_c - 1); code
 * q = floor((x - lo_c) / Delta_c + 0.5) clamped to [0, 2^K_c - 1], 0 when
 * that is not a number (hi_c == lo_c, or x NaN); the renderer's proxy is
 * lo_c + q Delta_c.  Every step in FP32, IEEE-rounded, in that order, no
 * fused multiply-adds.  The 8-bit plane layout ("codes") is
 * [F][D + 3][H_A][W_A] bytes: plane 2c / 2c + 1 holds the high / low byte
 * of position channel c < 3, plane c + 3 the code of channel c >= 3;
 * texels that are not live hold 0.  Gradients pass the quantiser straight
 * through: pk_atlas_scatter_grad's texel gradients are those of the FP32
 * masters. */
#define PK_LPO_CODES 0    /* pk_atlas_gather_lpo reads 8-bit code planes */
#define PK_LPO_MASTERS 1  /* ... or fake-quantises the FP32 master atlas */

/* lohi: out [D][2] float32 {lo_c, hi_c}, min and max of channel c over the
 * live texels of all F frames of the FP32 atlas [F][D][H_A][W_A]; NaN
 * texels are skipped; 0, 0 for a channel without a live texel. */
pk_status pk_lpo_minmax(const pk_plan *plan, const float *atlas, const uint32_t *occ, float *lohi,
                        void *workspace, pk_stream_t stream);

/* codes: out [F][D + 3][H_A][W_A] uint8 from the FP32 atlas and lohi. */
pk_status pk_lpo_encode(const pk_plan *plan, const float *atlas, const uint32_t *occ, const float *lohi,
                        uint8_t *codes, void *workspace, pk_stream_t stream);

/* a1 on the proxy: as pk_atlas_gather (same occ, dyn, soa, texel, dynflag
 * and status), the SoA receiving the proxy values lo_c + q Delta_c.  src
 * is the codes (src_kind = PK_LPO_CODES) or the FP32 master atlas
 * (PK_LPO_MASTERS: quantised on the fly, nothing stored).  The plan's
 * texel_type is not used. */
pk_status pk_atlas_gather_lpo(const pk_plan *plan, const void *src, int32_t src_kind, const float *lohi,
                              const uint32_t *occ, const uint32_t *dyn, float *soa, uint32_t *texel,
                              uint8_t *dynflag, void *workspace, pk_stream_t stream);

/* ------------------------------------------------------------------------ */
/* UV cells and Max-K UV pruning                                             */
/* ------------------------------------------------------------------------ */

/* UV cell of a Gaussian by eq. uvgs2 (Sec. 3 "UV-based Point-to-Image
 * Transformation"): rho = |mu|, theta = atan2(y, x), phi = acos(z / rho),
 * u = floor((pi + theta) / (2 pi) M), v = floor(phi / pi N), computed in
 * FP64; cell id v M + u.  Valid UV projection (Sec. 4.2 "UV-Based
 * Pruning"): rho positive and finite, 0 <= u < M, 0 <= v < N, and the
 * opacity logit not NaN.  Max-K UV pruning: of the valid Gaussians of a
 * cell, the K of highest opacity are kept (opacity = sigmoid(logit) is
 * increasing, so logits are compared; ties go to the lower index).  The
 * Gaussians need no plan: the call takes n candidates, e.g. the children
 * of a densification step.
 * soa:   [D][stride] float32, Gaussian i in column i (position channels
 *        0..2, opacity logit channel 10), stride >= n.
 * cell:  out [n] uint32 cell id, 0xFFFFFFFF if not valid.
 * rank:  out [n] uint32 0-based position in its cell's order (0xFFFFFFFF
 *        if not valid); keep: out [n] uint8, rank < K.
 * count: out [M N] uint32 valid Gaussians per cell.
 * scratch: pk_uv_max_k_scratch_bytes(n, M, N) bytes of device memory,
 *        256-byte aligned.  M N and n must be below 2^32 - 1. */
uint64_t pk_uv_max_k_scratch_bytes(int64_t n, int32_t M, int32_t N);
pk_status pk_uv_max_k(const float *soa, int64_t n, int64_t stride, int32_t M, int32_t N, int32_t K,
                      uint32_t *cell, uint32_t *rank, uint8_t *keep, uint32_t *count, void *scratch,
                      pk_stream_t stream);

/* Photometric objective of Sec. 4.2 "Objective":
 *   loss = (1 - lambda) mean|image - target| + lambda (1 - SSIM),
 * SSIM being the mean over the 3 P values of the per-channel SSIM map with
 * the 11 x 11 Gaussian window (standard deviation 1.5, weights summing to
 * 1; pixels outside the image count as 0 in every window sum), C1 = 0.01^2,
 * C2 = 0.03^2.  dL_dimage: out, the exact gradient of that loss (FP32
 * arithmetic): sign(image - target) (1 - lambda) / (3 P) plus the adjoint
 * of the window sums.  loss and ssim are stored in the status block.
 * lambda in [0, 1], else PK_ERR_ARG; lambda = 0.2 is the usual choice. */
pk_status pk_photo_loss_grad(const pk_plan *plan, const float *image, const float *target, float lambda,
                             float *dL_dimage, void *workspace, pk_stream_t stream);

const char *pk_status_string(pk_status s);
int32_t pk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PACKUV_H */
