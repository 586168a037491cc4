/*
 * dbmp.h -- C ABI of libdbmp, a GB300 (sm_103a) differentiable rasterizer for
 * bitmap primitives (DiffBMP, "Differentiable Rendering with Bitmap Primitives").
 *
 * The library draws N transformed bitmap primitives onto an RGB canvas,
 * front-to-back, and differentiates the result w.r.t. every primitive's
 * parameters.  One primitive i has eight float32 parameters, stored as one row
 * of an N x 8 row-major array:
 *
 *     x_i, y_i, s_i, theta_i, nu_i, c_r, c_g, c_b
 *
 *   Eq. 1   [u v]^T = R(theta_i) [(x - x_i)/s_i, (y - y_i)/s_i]^T,
 *           R = [[cos, sin], [-sin, cos]]; pixel (px, py) is the canvas point
 *           x = px, y = py (row py, column px; y grows downwards)
 *   Eq. 2   U = (u + 1)/2 (W_b - 1), V = (v + 1)/2 (H_b - 1)
 *   Eqs. S1-S3 (Sec. S1.1)  M = bilinear sample of bitmap P at (U, V); taps
 *           outside the bitmap read 0
 *   Eq. 3   alpha_i = alpha_max sigmoid(nu_i) M_i           (nu: opacity logit)
 *   Eqs. 4-5 T_k = prod_{j<k} (1 - alpha_j); I = sum_k T_k alpha_k sigmoid(c_k)
 *           (index 0 is the front layer; c: colour logits)
 *   Eq. 8   I += T_N b  (background b: none, a constant RGB, or a per-pixel buffer)
 *
 * Conventions for every call:
 *   - Return value: DBMP_OK (0) or a negative DbmpStatus.  Argument errors are
 *     detected on the host before any work is queued; dbmp_last_error() then
 *     holds a one-line message (per thread).
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; they must
 *     stay valid until the queued work has finished.  Host pointers are read
 *     during the call only.
 *   - Every call that takes a cudaStream_t only queues work on that stream and
 *     never synchronises it, except where stated (dbmp_status_poll,
 *     dbmp_workspace_create/destroy, dbmp_atlas_create/destroy, dbmp_autotune).
 *     Some kernels are launched as programmatic dependents of the kernel before
 *     them in the stream and wait for its completion before their first memory
 *     access, so stream order holds whatever the caller queued before a call.
 *   - Errors found on the device (tile-list capacity exceeded, degenerate
 *     primitives) are recorded in the workspace's status block; read them with
 *     dbmp_status_poll.  A kernel that finds the capacity error set does nothing.
 *   - Images are planar float32: image[c][py][px], c = 0..2; per-pixel maps are
 *     [py][px].  Canvases are any H, W >= 1 (ragged last tiles are handled).
 */
#ifndef DBMP_H
#define DBMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *dbmp_stream_t; /* == cudaStream_t; NULL = legacy default stream */

typedef enum {
    DBMP_OK = 0,
    DBMP_ERR_INVALID_ARG = -1, /* bad pointer, size, tile size or value */
    DBMP_ERR_CAPACITY = -2,    /* tile lists exceed the workspace capacity */
    DBMP_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    DBMP_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    DBMP_ERR_NOT_READY = -5,   /* required state missing (e.g. no prior dbmp_bin) */
    DBMP_ERR_NO_MEMORY = -6    /* device allocation failed */
} DbmpStatus;

/* Background of Eq. 8 (Sec. 3.2.3). */
typedef enum { DBMP_BG_NONE = 0, DBMP_BG_CONST = 1, DBMP_BG_BUFFER = 2 } DbmpBgMode;

typedef struct {
    int32_t mode;           /* DbmpBgMode */
    float rgb[3];           /* DBMP_BG_CONST: b                          */
    const float *buf_dev;   /* DBMP_BG_BUFFER: 3 x H x W planar, in [0,1] */
} DbmpBackground;

/* One-line description of the last error on this thread ("" if none). */
const char *dbmp_last_error(void);

/* ABI version of this header: 1. */
int32_t dbmp_abi_version(void);

/* ------------------------------------------------------------------------- */
/* Bitmap atlas (the primitives P_i of Eq. 2 / Sec. S1.1)                     */
/* ------------------------------------------------------------------------- */
typedef struct DbmpAtlas DbmpAtlas;

/* Builds the device-side sampling layout of n_bmp bitmaps of H_b x W_b texels
 * (texels_dev: float32 [n_bmp][H_b][W_b], values in [0, 1]; H_b, W_b >= 2).
 * The library stacks the bitmaps in one pitch-linear float plane, each followed
 * by a zero row, and reads it through a 2-D texture object with a zero border,
 * so that one texture gather returns the four taps of a bilinear sample (zero
 * outside the bitmap).  It also builds a summed-area table of the non-zero
 * texels, with which the compositors skip primitives whose bitmap is empty over
 * a whole region of pixels.  The plane must fit the device's pitch-linear
 * texture limits (GB300: n_bmp (H_b + 1) <= 65000 rows, W_b <= 131072);
 * otherwise DBMP_ERR_INVALID_ARG.  Allocates about n_bmp (H_b+1)(W_b+1) 8 bytes,
 * creates one texture object and synchronises `stream`.  texels_dev is not
 * referenced after the call. */
int32_t dbmp_atlas_create(const float *texels_dev, int32_t n_bmp, int32_t H_b, int32_t W_b,
                          dbmp_stream_t stream, DbmpAtlas **out);
int32_t dbmp_atlas_destroy(DbmpAtlas *atlas);
/* Re-fills an existing atlas from new texels of the same shape (no allocation;
 * stream-ordered). */
int32_t dbmp_atlas_update(DbmpAtlas *atlas, const float *texels_dev, dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Workspace                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct DbmpWorkspace DbmpWorkspace;

typedef struct {
    int32_t max_prims;    /* largest N (summed over canvases in batched mode) */
    int32_t max_tiles;    /* largest tile count (summed over canvases)         */
    int64_t max_pairs;    /* capacity of the tile lists: sum_t d_t (Sec. S4)    */
    int32_t max_canvases; /* batched mode: largest number of canvases (>= 1)   */
} DbmpLimits;

/* Device bytes a workspace with these limits holds. */
int32_t dbmp_workspace_bytes(const DbmpLimits *limits, size_t *bytes);
/* Allocates a workspace (device memory: per-primitive records, tile lists,
 * per-chunk histograms, gradient accumulators, status block, and a record of the
 * forward's surviving (primitive, list position) pairs for the backward, max_pairs/8
 * entries of 8 bytes). */
int32_t dbmp_workspace_create(const DbmpLimits *limits, DbmpWorkspace **out);
int32_t dbmp_workspace_destroy(DbmpWorkspace *ws);
/* Testing aid, in place of a memory sanitizer: fills every scratch buffer of the
 * workspace (records, rectangles, tile offsets, order and lists, histograms,
 * canvas descriptors, statistics; not the status block, nor the per-primitive
 * gradient sums, which every backward leaves zero for the next) with 0xFF
 * bytes, i.e. NaN floats and -1 integers, stream-ordered.  A later call that read a
 * buffer before writing it would then return different results.  Call it before
 * dbmp_batch_plan / dbmp_bin: it also erases a stored plan. */
int32_t dbmp_workspace_poison(DbmpWorkspace *ws, dbmp_stream_t stream);
/* Measurement aid (the work unit of the compositors' rooflines): with on != 0 the
 * forwards of this workspace count the pairs they composite with alpha > 0 into
 * the status block's pairs_contributing; off (the default) they leave it 0.  The
 * count is a per-pixel increment in the forward's inner loop that costs about a
 * tenth of its time, so it is compiled into a second instance of the forward that
 * only this switch selects; images and maps are the same either way. */
int32_t dbmp_workspace_count_pairs(DbmpWorkspace *ws, int32_t on);

/* Device-side status block, read (and cleared) by dbmp_status_poll. */
typedef struct {
    int32_t code;           /* DBMP_OK or DBMP_ERR_CAPACITY / DBMP_ERR_TIMEOUT   */
    int32_t n_degenerate;   /* primitives with a bitmap id outside the atlas or a
                               transform that overflows float32 (drawn as empty) */
    int64_t pairs_required; /* sum_t d_t of the last binning                    */
    int64_t pairs_evaluated;/* (pixel, list entry) pairs the last fwd evaluated  */
    int64_t pairs_evaluated_bwd; /* same for the last bwd                       */
    /* (The forward's counters start from zero at each forward, the backward's at each
     * backward; they are cleared by the binning / the forward's region sort when those
     * come first, so that the pass can start as their programmatic dependent, and
     * otherwise by a memset queued with the pass.) */
    int64_t pairs_contributing;  /* pairs with alpha > 0 the last fwd composited,
                                    i.e. layers with M > 0 met while T >= T_stop;
                                    0 unless dbmp_workspace_count_pairs enabled it */
    int64_t warp_steps;          /* list entries walked by warps in the last fwd   */
    int64_t warp_steps_bwd;      /* same for the last bwd                          */
    int64_t survivors;           /* list entries that passed the region test (fwd) */
    int64_t survivors_bwd;       /* same for the last bwd                          */
    int32_t bad_kind;            /* index-checked build only (dbmp_index_checks):
                                    the first out-of-range index met since the last
                                    poll, a DbmpBadIndex; the access was skipped     */
    int32_t bad_pad;
    int64_t bad_index;           /* which one: tile id (TILE_RANGE), list position
                                    (LIST_ENTRY, LIST_WRITE) or primitive (BITMAP_ROW) */
} DbmpDeviceStatus;

typedef enum {
    DBMP_BAD_NONE = 0,
    DBMP_BAD_TILE_RANGE = 1,  /* a tile's list range outside [0, sum_t d_t]: the tile is
                                 clipped to it (empty if it starts outside)          */
    DBMP_BAD_LIST_ENTRY = 2,  /* a list entry that is no primitive of the plan: culled */
    DBMP_BAD_BITMAP_ROW = 3,  /* a record whose bitmap row is not a bitmap's first row:
                                 culled                                              */
    DBMP_BAD_LIST_WRITE = 4   /* a binning write outside the lists: dropped          */
} DbmpBadIndex;

/* 1 if this library was built with device-side index checks (the checked build,
 * libdbmp_checked.so: the compositors check every tile range, list entry and
 * bitmap row they read and the binning every list position it writes, record the
 * first bad one in the status block and skip the access), else 0.  The checks
 * stand in for a device-assert build, whose failing assert would trap the GPU. */
int32_t dbmp_index_checks(void);

/* Testing aid for the index checks: overwrites one value of a binned workspace,
 * stream-ordered, then synchronises `stream`.  what = 0: tile offset `index`
 * (0..max_tiles); 1: tile-list entry `index` (0..max_pairs-1); 2: the bitmap row of
 * primitive `index`'s record (0..max_prims-1).  Indices outside the workspace's
 * allocations are rejected (DBMP_ERR_INVALID_ARG), so the write itself stays inside
 * them; what a later render then reads is for the caller to keep inside them too. */
int32_t dbmp_workspace_debug_set(DbmpWorkspace *ws, int32_t what, int64_t index, int64_t value,
                                 dbmp_stream_t stream);

/* Synchronises `stream`, copies the status block to *out, clears the sticky
 * error code and returns out->code. */
int32_t dbmp_status_poll(DbmpWorkspace *ws, dbmp_stream_t stream, DbmpDeviceStatus *out);

/* Scaling statistics of the workspace's last binning (Sec. S4, "Additional scaling
 * statistics": normalised footprint A_i / (H W), tile-hit degree tau_i, per-tile
 * density d_t), summed over the plan's canvases.  A_i is the padded box area
 * (2 hx + 2)(2 hy + 2) of the bitmap's whole support rotated and scaled, with
 * e_u = 1 + 2/(W_b-1), e_v = 1 + 2/(H_b-1), hx = |s| (|cos| e_u + |sin| e_v),
 * hy = |s| (|sin| e_u + |cos| e_v) and the sine and cosine of the binning
 * specification below (FP64 from the fp32 half-extents), normalised by its own
 * canvas; it does not depend on which texels of the bitmap are non-zero.
 * Histograms have 32 bins:
 *   tau_hist[b]   listed primitives (tau_i >= 1) with floor(log2 tau_i) = b
 *   d_hist[b]     tiles with d_t >= 1 and floor(log2 d_t) = b
 *   foot_hist[b]  listed primitives with A_i / (H W) in [2^-(b+1), 2^-b) (b = 0
 *                 also takes ratios >= 1; smaller ratios go to b = 31)
 * pairs = sum_i tau_i = sum_t d_t.  Needs a binning in the workspace (else
 * DBMP_ERR_NOT_READY) with its params still valid; synchronises `stream`. */
typedef struct {
    int64_t n_listed, pairs, tau_max, d_max, n_tiles, empty_tiles;
    int64_t tau_hist[32];
    int64_t d_hist[32];
    int64_t foot_hist[32];
} DbmpBinStats;
int32_t dbmp_bin_stats(DbmpWorkspace *ws, dbmp_stream_t stream, DbmpBinStats *out);

/* ------------------------------------------------------------------------- */
/* Binning (Sec. 3.1.1 "Parallelization"; Sec. S1.3)                          */
/* ------------------------------------------------------------------------- */
/* Per-primitive preprocessing and tile lists for one canvas H x W split into
 * tile x tile pixel tiles (tile in {8, 16, 32}).  A primitive is listed in
 * every tile its bounding box overlaps; each tile's list holds primitive indices
 * in increasing (front-to-back) order.  The box holds every pixel where the
 * primitive's sample can be non-zero: with zero padding that needs bitmap
 * coordinates within one texel of the bitmap's non-zero texels, whose first and
 * last columns and rows [u0, u1] x [v0, v1] the atlas records per bitmap.  It is
 * the fp32 specification below, evaluated one IEEE operation at a time (no fused
 * multiply-add), so the lists are bit-exact and reproducible:
 *     (sin, cos) of theta by Cody-Waite reduction by pi/2, degree-9/8 Taylor
 *     polynomials and the quadrant's signs;
 *     kw = (W_b-1)/2, kv = (H_b-1)/2; uc = ((u0 + u1 - (W_b-1)) / 2) / kw,
 *     eu = ((u1 - u0 + 2) / 2) / kw, likewise vc, ev with v0, v1, kv;
 *     dx = s (cos uc - sin vc), dy = s (sin uc + cos vc),
 *     hx = |s| (|cos| eu + |sin| ev), hy = |s| (|sin| eu + |cos| ev)
 *     (|theta| > 65536: dx = dy = 0, hx = hy = |s| (((|uc| + eu) + |vc|) + ev));
 *     m = 1 + |s| 2^-19; cx = x + dx, cy = y + dy;
 *     tx0 = floor(((cx - hx) - m) / tile), tx1 = floor(((cx + hx) + m) / tile),
 *     likewise ty0, ty1, clipped to the canvas' tiles.
 * Primitives with a non-finite parameter, s == 0 or an all-zero bitmap are not
 * listed.
 *   params_dev     float32 [N][8] (x, y, s, theta, nu, c_r, c_g, c_b)
 *   bitmap_id_dev  int32 [N], each in [0, n_bmp); a primitive with an id
 *                  outside the atlas is not listed and is counted in the status
 *                  block's n_degenerate
 *   alpha_max      in (0, 1] (Eq. 3)
 * The tile lists are written by a stable counting sort keyed on the tile index
 * (the primitive index is already the order inside a tile), so the result is
 * identical to sorting (tile << 32 | index) keys.  If sum_t d_t exceeds
 * limits.max_pairs nothing is written past the capacity, the status block gets
 * DBMP_ERR_CAPACITY and pairs_required, and later fwd/bwd calls do nothing. */
int32_t dbmp_bin(DbmpWorkspace *ws, int32_t H, int32_t W, int32_t tile, const float *params_dev,
                 const int32_t *bitmap_id_dev, int32_t N, const DbmpAtlas *atlas, float alpha_max,
                 dbmp_stream_t stream);

/* Copies the tile lists of the last dbmp_bin to caller buffers:
 * offsets_dev int64 [n_tiles + 1] (row-major tiles), list_dev int32 [cap].
 * Writes min(K, cap) list entries; *n_tiles_out (host) gets the tile count. */
int32_t dbmp_get_tile_lists(DbmpWorkspace *ws, int64_t *offsets_dev, int32_t *list_dev, int64_t cap,
                            int32_t *n_tiles_out, dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Forward (Eqs. 1-5, 8; Algorithm 1)                                         */
/* ------------------------------------------------------------------------- */
/* Composites the binned primitives (requires a prior dbmp_bin on `ws`, with the
 * same atlas).  Each warp composites one region of a tile (32 ppt pixels) as an
 * independent worker: it stages batches of the tile's primitive records in its
 * own shared-memory slice and walks the list front to back until all of its
 * pixels are saturated.
 *   T_stop   early termination: a layer is composited only while the pixel's
 *            transmittance is >= max(T_stop, 2^-100); the image then differs from
 *            the full composite by at most T_stop.  0 = every layer.
 *   image_dev    out float32 [3][H][W]
 *   T_final_dev  out float32 [H][W]  transmittance after the last composited
 *                layer (I_alpha = 1 - T_final, Sec. 3.3.2)
 *   n_last_dev   out int32 [H][W]  position, in the pixel's tile list, of the
 *                last layer with alpha > 0 (-1: none); saved for the backward */
int32_t dbmp_render_fwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg,
                        float T_stop, float *image_dev, float *T_final_dev, int32_t *n_last_dev,
                        dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Backward (Eq. 6; Eqs. S4-S5, Sec. S1.2)                                    */
/* ------------------------------------------------------------------------- */
/* Gradient of a scalar loss L w.r.t. the raw parameters (logits for nu and c),
 * given dL/dI (3 x H x W) and optionally dL/dI_alpha (H x W, NULL = 0).
 * Requires the dbmp_bin + dbmp_render_fwd of the same inputs (T_final and n_last
 * are that forward's outputs).  Each tile is walked back to front from its
 * largest n_last, recovering T_k = T_{k+1} / (1 - alpha_k) (the forward stores
 * no per-layer state); the exact derivative is taken, including the background
 * term Eq. S5 omits.  Per-(pixel, layer) terms are reduced across each warp by
 * shuffles, then added with one atomic per primitive per warp, so dparams is
 * exact up to float32 summation order.  The chain rule to s and nu reads the
 * params_dev given to dbmp_bin: that buffer must still hold the same values.
 * When the workspace's last forward rendered the same lists with the same region
 * shape, the backward walks the records that forward kept per region (those that
 * passed its region test) instead of re-reading and re-testing the tile lists;
 * a region whose pixels' last layers lie beyond what that forward tested (maps from
 * another forward with a smaller T_stop) is walked from its list as before.
 *   dparams_dev  float32 [N][8], ACCUMULATED into (zero it first). */
int32_t dbmp_render_bwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg,
                        float T_stop, const float *dL_dimage_dev, const float *dL_dalpha_dev,
                        const float *T_final_dev, const int32_t *n_last_dev, float *dparams_dev,
                        dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Loss and optimiser (Tab. S1: MSE loss, Adam-like optimiser with per-group   */
/* learning-rate gains and exponential decay; compute_psnr)                   */
/* ------------------------------------------------------------------------- */
/* L = mean((I - I*)^2) over n elements; dL_dI_dev = 2 (I - I*) / n; loss_dev
 * (device double[1]) = L.  PSNR = 10 log10(1 / L) for images in [0, 1]. */
int32_t dbmp_mse_grad(const float *image_dev, const float *target_dev, int64_t n,
                      float *dL_dI_dev, double *loss_dev, dbmp_stream_t stream);

typedef struct {
    float lr;        /* base learning rate (Tab. S1: 0.1)                      */
    float gamma;     /* exponential decay per step: lr_t = lr gamma^(t-1)      */
    float beta1, beta2, eps;
    float gains[8];  /* per parameter column (Tab. S1: 10 10 10 1 1.5 1 1 1)  */
    int32_t zero_grad; /* non-zero: the step writes 0 to grad after reading it, so
                          the next backward can accumulate into it directly    */
} DbmpAdamConfig;

/* One bias-corrected Adam step on params/m/v (float32 [N][8]).  step_dev is a
 * device int32 counter of completed steps: this call uses t = *step_dev + 1 and
 * then increments it, so a captured CUDA graph replays correct steps. */
int32_t dbmp_adam_step(float *params_dev, float *grad_dev, float *m_dev, float *v_dev,
                       int32_t N, int32_t *step_dev, const DbmpAdamConfig *cfg,
                       dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Batched, persistent rendering of many canvases                             */
/* ------------------------------------------------------------------------- */
/* A batch plan fixes the canvases of a step: canvas c is H[c] x W[c], owns the
 * primitives [prim_offset[c], prim_offset[c+1]) of the concatenated parameter
 * array, and its image / T_final / n_last / gradient maps start at pixel
 * pix_offset[c] = sum_{c'<c} H[c'] W[c'] of concatenated per-canvas buffers
 * (image: 3 planar channels per canvas, i.e. canvas c's image starts at
 * 3 pix_offset[c]).  All host arrays have n_canvas (+1) entries.  The plan is
 * uploaded to the workspace (synchronises `stream`); dbmp_batch_render then
 * reads no host memory, so a whole optimisation step can be captured in a CUDA
 * graph. */
typedef struct {
    int32_t tile;   /* 8, 16 or 32 */
    int32_t batch;  /* records each warp stages per shared-memory batch: 32 or 64 */
    int32_t ppt;    /* pixels per lane of the forward: 1, 2 or 4 (4 needs tile >= 16);
                       a warp owns a region of 32 ppt pixels of a tile */
    int32_t ppt_bwd;/* pixels per lane of the backward, same values; 0 = ppt.  The
                       passes share only per-pixel maps, so their regions may differ */
} DbmpTuning;

int32_t dbmp_batch_plan(DbmpWorkspace *ws, int32_t n_canvas, const int32_t *H, const int32_t *W,
                        const int32_t *prim_offset, const DbmpTuning *tuning,
                        dbmp_stream_t stream);

/* Restricts the forward and backward of the current plan to canvas rows [y0, y1)
 * of every canvas (binning still lists every tile); y0 = y1 = 0 lifts the
 * restriction, and dbmp_batch_plan resets it.  Regions outside the window are
 * skipped: their image, T_final and n_last pixels are left as they were and they
 * contribute nothing to the loss or the gradient.  The fused MSE keeps its
 * normalisation over all pixels of the plan, so the losses and gradients of
 * disjoint windows sum to those of the whole canvas: this is how one canvas is
 * shared between ranks that hold the same parameters (Sec. 3.1.1, "Parallelization":
 * tiles are independent; the gradient, Eq. 6, is a sum over pixels).  y0 and y1
 * must be multiples of the plan's tile size with y0 < y1, else DBMP_ERR_INVALID_ARG;
 * DBMP_ERR_NOT_READY without a plan.  Host-only: queues nothing. */
int32_t dbmp_batch_set_rows(DbmpWorkspace *ws, int32_t y0, int32_t y1);

typedef enum { DBMP_BATCH_BIN = 1, DBMP_BATCH_FWD = 2, DBMP_BATCH_BWD = 4 } DbmpBatchMode;

/* Bins all canvases (one launch per stage), then renders every (canvas, tile,
 * region) work item with one persistent forward launch (and one backward
 * launch): resident warps pull items from an atomic queue, tiles ordered by
 * decreasing list length (longest-processing-time first).  `mode` is an OR of DbmpBatchMode.
 * Pointers follow the plan's concatenated layouts; bg must be NONE or CONST. */
int32_t dbmp_batch_render(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                          const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg,
                          float T_stop, int32_t mode, float *image_dev, float *T_final_dev,
                          int32_t *n_last_dev, const float *dL_dimage_dev, float *dparams_dev,
                          dbmp_stream_t stream);

/* dbmp_batch_render with the MSE loss (Tab. S1 `mse`, mean over 3 H W) fused into
 * the forward's epilogue: mode must include DBMP_BATCH_FWD.  The forward writes the
 * image as usual and, per pixel, dL/dI = 2 (I - I*) / n into dL_dimage_dev (the
 * same values dbmp_mse_grad would write) and adds its (I - I*)^2 / n into
 * *loss_dev (zeroed by the call; summation order unspecified), n = 3 x the planned
 * canvases' pixels; with DBMP_BATCH_BWD the backward then runs on that dL/dI.  This
 * saves the separate pass over the image that dbmp_mse_grad makes.
 *   target_dev     float32, the plan's concatenated planar 3 x H x W targets
 *   dL_dimage_dev  float32, same layout (out; the backward's input)
 *   loss_dev       double [1] (out) */
int32_t dbmp_batch_render_mse(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                              const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg, float T_stop,
                              int32_t mode, const float *target_dev, float *image_dev, float *T_final_dev,
                              int32_t *n_last_dev, float *dL_dimage_dev, float *dparams_dev, double *loss_dev,
                              dbmp_stream_t stream);

/* Autotuner: for every (tile, batch) it times, with CUDA events and reps times
 * each, the binning once and the forward and the backward (those `mode` asks
 * for) at every supported ppt; the tuning with the smallest bin + best forward +
 * best backward time, each pass at its own ppt, goes to *best and its time to
 * *best_ms.  Synchronises `stream`; re-plans the workspace with the winner. */
int32_t dbmp_autotune(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                      const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg,
                      float T_stop, int32_t mode, float *image_dev, float *T_final_dev,
                      int32_t *n_last_dev, const float *dL_dimage_dev, float *dparams_dev,
                      int32_t reps, DbmpTuning *best, float *best_ms, dbmp_stream_t stream);

/* Tile-density-guided autotuning (the scaling statistics of Sec. S4 feeding the
 * search).  With max_pairs_ratio > 0, dbmp_autotune first bins the plan's scene once
 * per tile size and reads its tile-density statistics (dbmp_bin_stats: the list
 * entries pairs = sum over tiles of d_t); it then times only the tile sizes whose
 * entries are at most max_pairs_ratio times the fewest of any size, in increasing
 * order of entries (a tile size whose binning overflows the workspace is dropped).
 * Every tile-list entry is binned, culled per warp region and walked by both
 * compositors, so a size with several times the entries of another rarely wins.
 * 0 (the default of a new workspace) times every tile size.  DBMP_ERR_INVALID_ARG
 * for a negative or non-finite ratio.  Host-only (no device work). */
int32_t dbmp_autotune_set_prune(DbmpWorkspace *ws, float max_pairs_ratio);

/* ------------------------------------------------------------------------- */
/* BF16 tensor-core GEMM (tcgen05, FP32 accumulation), used by the proposal    */
/* network below and exposed for testing                                      */
/* ------------------------------------------------------------------------- */
/* C[m][n] (op)= sum_k A[m][k] B[n][k] for m < M, n < N, k < K.
 *   A_dev, B_dev  bf16 (raw 16-bit), row-major M x K and N x K (K contiguous),
 *                 16-byte aligned, lda and ldb multiples of 8, K a multiple of 64;
 *                 with mode flag 16 (32) A (B) is given MN-major instead: the
 *                 K x M (K x N) row-major matrix, lda >= M (ldb >= N)
 *   mode 0: Cf[m][n] = acc            (float32, row stride ldc)
 *   mode 1: Cf[m][n] += acc           (float32 atomics; allows split_k > 1)
 *   mode 2: Cb[m][n] = bf16(max(acc + bias[n], 0))   (bf16, row stride ldc)
 *   mode 3: Cf[m][n] = acc + bias[n]
 *   mode 4: Cb[m][n] = bf16(acc)      (bf16, row stride ldc)
 *   split_k  number of CTAs sharing the K range of a tile (mode 1 only if > 1)
 *   mode flag 64: failure-detection test only: no operand copy is issued, so the
 *               pipeline's waits run out (2 s each) and status_dev is set to
 *               DBMP_ERR_TIMEOUT; C is not written; the context stays usable
 *   status_dev  optional device int32 set to DBMP_ERR_TIMEOUT if a bounded
 *               wait on the tensor-core pipeline gave up after 2 s (nullable) */
int32_t dbmp_gemm_bf16(const uint16_t *A_dev, int32_t lda, const uint16_t *B_dev, int32_t ldb,
                       int32_t M, int32_t N, int32_t K, int32_t mode, float *Cf_dev,
                       uint16_t *Cb_dev, int32_t ldc, const float *bias_dev, int32_t split_k,
                       int32_t *status_dev, dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* FP32 issue-rate microbenchmark (measurement aid, not part of the method)    */
/* ------------------------------------------------------------------------- */
/* Queues one launch of n_threads / 256 blocks of 256 threads; every thread runs
 * 16 independent multiply-add chains for iters x 8 steps, with scalar FFMA
 * (packed = 0) or packed FP32x2 FMA instructions (packed = 1), and stores one
 * float per thread into sink_dev (float32 [n_threads], device, caller-owned).
 * *flops (host) receives the launch's floating-point operations (2 per
 * multiply-add).  Time the launch with events on `stream`: flops / seconds is the
 * FP32 rate the compositors' ALU roofline is measured against.  n_threads must be
 * a positive multiple of 256 and iters > 0, else DBMP_ERR_INVALID_ARG. */
int32_t dbmp_fp32_peak(int32_t packed, int32_t iters, float *sink_dev, int64_t n_threads, double *flops,
                       dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Learned proposal network                                                   */
/* ------------------------------------------------------------------------- */
/* A small CNN that maps a target image to initial parameters of 512 primitives,
 * to be refined by the plain optimisation (Eqs. 1-5 + Adam).  The paper names
 * learned (autoregressive / RL) initialisation as future work (Sec. S5) and
 * shows that initialisation matters (Sec. 3.2.2); the network here is this
 * library's own design:
 *   input   256 x 256 RGB in [0, 1] -> bf16 NHWC, 2 (I - 0.5), channels padded to 4
 *   conv1-5 4x4 / stride 2 / pad 1, bias, ReLU: 4 -> 32 -> 64 -> 128 -> 256 -> 256
 *   head    1x1 conv 256 -> 64 on the 8 x 8 map = 8 slots x 8 outputs per cell
 *   decode  cell (cy, cx), slot k, outputs o: x = 32 cx + 8 (k % 4) + 8 s(o0),
 *           y = 32 cy + 16 (k / 4) + 16 s(o1), s = 6 + 8 s(o2), theta = 0,
 *           nu = o4, c = (o5, o6, o7); primitive index (8 cy + cx) 8 + k
 *   loss    mean squared error of the raw outputs against the targets of the
 *           anchored parameterisation (logit of the clipped in-cell offset and
 *           scale, nu and c clipped to [-6, 6]; theta not learned)
 * All products run on the tcgen05 tensor cores (BF16 operands, FP32
 * accumulation); weights are FP32 masters with BF16 copies.  Parameters are one
 * flat float32 vector: for each layer, W (Cout x K, K ordered (ky, kx, ci)) then
 * b (Cout).  A proposer owns its buffers for batches of up to max_batch images.
 * images_dev: B x 3 x 256 x 256 float32 planar (the concatenated per-canvas
 * images dbmp_batch_render writes for 256 x 256 canvases). */
typedef struct DbmpProposer DbmpProposer;

typedef struct {
    float lr, beta1, beta2, eps;
} DbmpProposerAdam;

int64_t dbmp_proposer_num_params(void);
/* Allocates (synchronises the device). */
int32_t dbmp_proposer_create(int32_t max_batch, DbmpProposer **out);
int32_t dbmp_proposer_destroy(DbmpProposer *p);
/* Uploads host float32 parameters (n = dbmp_proposer_num_params()), resets Adam.
 * Synchronous. */
int32_t dbmp_proposer_set_params(DbmpProposer *p, const float *host, int64_t n);
/* Downloads the parameters (which = 0) or the last gradient (which = 1);
 * synchronises the device; DBMP_ERR_TIMEOUT if a tensor-core wait gave up. */
int32_t dbmp_proposer_get(DbmpProposer *p, int32_t which, float *host, int64_t n);
/* Testing aid: downloads the activations the last forward (dbmp_propose or
 * dbmp_proposer_train_step) left on the device, as float32 in host memory:
 * layer 0 = the packed bf16 input (B x 256 x 256 x 4, NHWC), 1..5 = the bf16
 * post-ReLU outputs of the five convolutions (B x S x S x C, S = 128, 64, 32, 16, 8,
 * C = 32, 64, 128, 256, 256), 6 = the head's float32 outputs (B*64 x 64).  n must
 * be that count for the last forward's batch, else DBMP_ERR_INVALID_ARG;
 * DBMP_ERR_NOT_READY before the first forward.  Synchronises the device. */
int32_t dbmp_proposer_activations(DbmpProposer *p, int32_t layer, float *host, int64_t n);
/* Decoded proposals: params_out_dev float32 B x 512 x 8 (same layout as dbmp_bin's
 * params, primitive order as above).  Stream-ordered. */
int32_t dbmp_propose(DbmpProposer *p, const float *images_dev, int32_t B, float *params_out_dev,
                     dbmp_stream_t stream);
/* One training step on (image, target parameters) pairs: forward, loss
 * (loss_dev: device double, overwritten), gradient of every parameter, and, if
 * adam is not NULL, one Adam step on the FP32 masters.  target_params_dev:
 * B x 512 x 8 float32.  Stream-ordered. */
int32_t dbmp_proposer_train_step(DbmpProposer *p, const float *images_dev, const float *target_params_dev,
                                 int32_t B, const DbmpProposerAdam *adam, double *loss_dev,
                                 dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Gaussian blur of the primitive bitmaps (Sec. 3.2 "Blurring Primitives for  */
/* Enriching Gradients"; Tab. S1 do_gaussian_blur, blur_sigma = 1.0)          */
/* ------------------------------------------------------------------------- */
/* Soft rasterisation applied once before optimisation: out = each bitmap
 * convolved with the Gaussian exp(-(dy^2 + dx^2) / (2 sigma^2)), |dy|, |dx| <=
 * r = ceil(3 sigma), normalised to sum 1, with texels outside the bitmap taken as
 * zero (the radius is this library's reading; the paper gives sigma only).  Build
 * the atlas from `out` (dbmp_atlas_create / dbmp_atlas_update).
 *   texels_dev  float32 [n_bmp][H_b][W_b] (read only);  out_dev  same shape, must
 *               not overlap texels_dev;  sigma in (0, 5];  1 <= n_bmp <= 65535
 * FP32 arithmetic (separable passes), stream-ordered, no allocation. */
int32_t dbmp_blur_bitmaps(const float *texels_dev, int32_t n_bmp, int32_t H_b, int32_t W_b, float sigma,
                          float *out_dev, dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Structure-aware initialisation (Sec. 3.2 "Structure-aware Initialization"; */
/* Tab. S1: variance window 7, base probability 0.1, colour noise std 0.02)   */
/* ------------------------------------------------------------------------- */
/* Draws N initial primitives from a target image, dense and fine where the
 * image varies locally, sparse and coarse where it is flat:
 *   LV(p)   per channel the population variance of the image over the 7 x 7
 *           window centred on pixel p (clipped to the canvas), averaged over
 *           R, G, B, in FP64;
 *   NLV(p)  (LV(p) - min LV) / (max LV - min LV), 0 if LV is constant;
 *   draw    primitive i takes pixel p with probability proportional to
 *           w(p) = 0.1 + 0.9 NLV(p) (with replacement): w is quantised to
 *           q(p) = floor(w(p) 2^20) and i takes the p with
 *           Q(p) <= floor(u_pos[i] Q_total) < Q(p) + q(p), Q the exclusive prefix
 *           sum of q (exact integers, so the draw is reproducible bit for bit);
 *   params  x = px, y = py (the pixel centre), s = s_max - (s_max - s_min) NLV(p),
 *           theta = 2 pi u_theta[i], nu fixed, colour channel j: the logit of
 *           I_j(p) + sigma_c n_color[3 i + j] clamped to [1e-4, 1 - 1e-4].
 * Readings of the paper: the lattice points are the pixel centres, the colour
 * draw is on the activated colour, and the random numbers are inputs (the
 * caller's seeded generator).  The paper fixes nu = -2 in its text and lists
 * v_init_bias = -4 in Tab. S1; nu is an argument here.
 *   image_dev    float32 3 x H x W planar, values in [0, 1] (read only)
 *   mask_dev     float32 H x W or NULL: the spatially constrained variant (Sec.
 *                3.3.2) draws only pixels with mask > 0 (the target's alpha); an
 *                empty mask draws nothing and leaves params_dev untouched
 *   u_pos_dev, u_theta_dev   double [N] in [0, 1);  n_color_dev  double [N][3]
 *   scratch_dev  dbmp_structure_init_scratch_bytes(H, W) bytes, 256-byte aligned,
 *                caller-owned; overwritten
 *   params_dev   float32 [N][8] (out);  nlv_dev  double [H][W] (out, nullable)
 * Returns DBMP_ERR_INVALID_ARG for H, W < 1, H W > 2^31 - 1, N < 0, a NULL
 * required pointer, a misaligned scratch, s_min > s_max or sigma_c < 0.
 * Stream-ordered, no allocation, capturable in a CUDA graph. */
int32_t dbmp_structure_init_scratch_bytes(int32_t H, int32_t W, size_t *bytes);
int32_t dbmp_structure_init(const float *image_dev, const float *mask_dev, int32_t H, int32_t W, int32_t N,
                            const double *u_pos_dev, const double *u_theta_dev, const double *n_color_dev,
                            double s_min, double s_max, double sigma_c, double nu, void *scratch_dev,
                            float *params_dev, double *nlv_dev, dbmp_stream_t stream);

/* Re-initialisation of transparent primitives (Sec. 3.3.2; Sec. S3 "Re-initialization
 * Mechanism": opacity sigmoid(nu) below prune_threshold = 0.3, every 50 iterations
 * after a warm-up).  Every primitive i of params_dev (in/out, [N][8]) with
 * sigmoid(nu_i) < threshold (evaluated in FP64) takes draw i of
 * dbmp_structure_init with the same arguments; its Adam moments adam_m_dev /
 * adam_v_dev ([N][8], nullable) are zeroed (a reading: the redrawn primitive
 * starts afresh) and *count_dev (int32, nullable, not reset here) is incremented.
 * threshold in [0, 1].  Other arguments, errors and ordering as dbmp_structure_init. */
int32_t dbmp_structure_reinit(const float *image_dev, const float *mask_dev, int32_t H, int32_t W, int32_t N,
                              const double *u_pos_dev, const double *u_theta_dev, const double *n_color_dev,
                              double s_min, double s_max, double sigma_c, double nu, double threshold,
                              void *scratch_dev, float *params_dev, float *adam_m_dev, float *adam_v_dev,
                              int32_t *count_dev, dbmp_stream_t stream);

/* The rendered alpha channel (Sec. 3.3.2): alpha_dev[p] = 1 - T_final_dev[p] for
 * p < n_pix, from the T_final map of dbmp_render_fwd (float32, device; the two
 * buffers may be the same).  n_pix >= 0.  Stream-ordered. */
int32_t dbmp_render_alpha(const float *T_final_dev, float *alpha_dev, int64_t n_pix, dbmp_stream_t stream);

/* Spatially constrained loss (Eq. 9, Sec. 3.3.2), both squared norms read as means:
 *   L = sum_p [a*_p > 0] |I_p - I*_p|^2 / (3 n) + lambda_alpha sum_p (I_alpha,p - a*_p)^2 / n
 * with I_alpha = 1 - T_N (T_final of the forward), n = n_pix pixels; writes
 * dL/dI (3 planes) and dL/dI_alpha, the inputs of dbmp_render_bwd, and overwrites
 * *loss_dev (device double).  The paper weights the opacity term 0.3 (Sec. S3).
 *   image_dev, target_dev  float32 3 x n planar;  T_final_dev, target_alpha_dev
 *   float32 n;  outputs float32 3 x n and n.  lambda_alpha >= 0.  Stream-ordered. */
int32_t dbmp_alpha_loss_grad(const float *image_dev, const float *T_final_dev, const float *target_dev,
                             const float *target_alpha_dev, int64_t n_pix, float lambda_alpha, float *dL_dimage_dev,
                             float *dL_dalpha_dev, double *loss_dev, dbmp_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Forward render without device allocation                                   */
/* ------------------------------------------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory.  Examples: a host application or plugin
 * sandbox that owns a fixed device-memory budget, and real-time loops where
 * cudaMalloc/cudaFree cannot be afforded because they may synchronise the whole
 * device and can fail with out-of-memory partway through a long run.
 *
 * It renders one canvas exactly like dbmp_bin (tile 16) followed by
 * dbmp_render_fwd (default tuning), from the plain atlas texels
 * (float32 [n_bmp][H_b][W_b]), with no DbmpWorkspace and no DbmpAtlas.  All
 * intermediate state lives in one scratch array compiled into the library
 * (about 6.3 MB of device memory).  Every GPU that loads the library holds it
 * until the process exits.  Maximum sizes:
 *     H, W <= 512;  N <= 4096;  n_bmp (H_b + 1)(W_b + 1) <= 32768;
 *     tile-list entries (sum_t d_t) <= 1 048 576.
 * Larger sizes are rejected on the host with DBMP_ERR_INVALID_ARG; exceeding
 * the tile-list capacity can only be seen on the device (see status_out).
 *
 * The caller passes inputs and outputs as for dbmp_bin / dbmp_render_fwd
 * (params_dev 16-byte aligned; image 3 x H x W, T_final and n_last H x W).
 * This call calls no cudaMalloc, cudaFree or allocating library routine.  The
 * first call on each device does a one-time set-up with that device current: it
 * resolves the scratch array's device address and sets kernel attributes.  The
 * first call with each atlas shape (W_b, n_bmp (H_b + 1)) on a device creates a
 * texture object over the scratch texel plane, kept until the process exits (at
 * most 64 shapes).  Make those first calls before any stream capture.
 *
 * All calls share the one scratch array, which keeps the last call's contents.
 * The call itself clears what must start at zero.  Calls whose GPU work
 * overlaps (different streams without ordering between them, or several host
 * threads) race on the array and give wrong results: order them on one stream.
 *
 * status_out: NULL -> the call only queues work on `stream` and returns; if the
 * tile lists exceed the capacity, the outputs are left unwritten.  Non-NULL ->
 * the call synchronises `stream`, fills *status_out, and returns
 * DBMP_ERR_CAPACITY if the lists did not fit. */
int32_t dbmp_render_fwd_static(int32_t H, int32_t W, const float *params_dev,
                               const int32_t *bitmap_id_dev, int32_t N, const float *texels_dev,
                               int32_t n_bmp, int32_t H_b, int32_t W_b, float alpha_max,
                               const DbmpBackground *bg, float T_stop, float *image_dev,
                               float *T_final_dev, int32_t *n_last_dev, dbmp_stream_t stream,
                               DbmpDeviceStatus *status_out);

#ifdef __cplusplus
}
#endif
#endif /* DBMP_H */
