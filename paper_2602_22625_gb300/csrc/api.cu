// C ABI of libdbmp: argument checking, workspaces, plans, and the entry points
// declared in include/dbmp.h.  No exception crosses the ABI.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "dbmp_internal.cuh"

using namespace dbmp;

namespace {

thread_local char g_err[512] = "";

int32_t fail(int32_t code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int32_t cuda_fail(cudaError_t e, const char *what) {
    return fail(DBMP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define DBMP_CUDA(call, what)                          \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

constexpr int32_t kMaxTilesPerCanvas = 65536;  // tile index range of one canvas
// Passes with at most this many regions per SM take their regions in the order of the
// forward's measured costs (measured: main 1024^2 workload, 54 per SM, backward -10%;
// 2048^2 stress, 216 per SM, -1%; 64-canvas batch, 1 600 per SM, +3%, so not there).
constexpr int32_t kOrderMaxRegionsPerSM = 256;
constexpr int64_t kHistCap = 16 << 20;         // chunk x tile histogram entries

bool tile_ok(int32_t t) { return t == 8 || t == 16 || t == 32; }

}  // namespace

int32_t dbmp::record_error(int32_t code, const char *msg) { return fail(code, "%s", msg); }

struct DbmpAtlas {
    void *plane_alloc = nullptr;
    float *plane = nullptr;     // stacked texel plane (row pitch `pitch` bytes), 512-byte aligned
    size_t pitch = 0;
    cudaTextureObject_t tex = 0;
    int32_t *sat = nullptr;
    int4 *nzbox = nullptr;      // per bitmap: the box of its non-zero texels
    int32_t n_bmp = 0, Hb = 0, Wb = 0;
    AtlasView view() const { return AtlasView{tex, sat, n_bmp, Hb, Wb, nzbox}; }
};

struct DbmpWorkspace {
    DbmpLimits lim{};
    // device
    PrimRec *rec = nullptr;
    int4 *rect = nullptr;
    float *graw = nullptr;
    int64_t *tile_off = nullptr;
    int32_t *tile_order = nullptr;
    int32_t *list = nullptr;
    int32_t *hist = nullptr;
    CanvasDesc *canvas = nullptr;
    DevStatus *status = nullptr;
    unsigned long long *stats = nullptr;   // scaling statistics counters
    int32_t *item_cost = nullptr;          // [item_cap] per-region cost of the last forward
    int32_t *item_order = nullptr;         // [item_cap] regions by decreasing cost
    int64_t item_cap = 0;                  // regions the two arrays hold
    int32_t *item_hist = nullptr;          // [2][256] cost buckets and cursors of alternate forwards
    int32_t hist_half = 0;                 // the half the next forward counts into (zeroed)
    // the order matches the current plan and the forward's regions (0: none yet)
    int32_t order_items = 0;
    int2 *surv = nullptr;                  // [surv_cap] survivor record of the last forward
    int4 *surv_tab = nullptr;              // [item_cap] its per-region entries
    int64_t surv_cap = 0;
    // regions the last forward recorded survivors for, on the current lists (0: none)
    int32_t surv_items = 0;
    int32_t count_pairs = 0;               // forwards count the contributing pairs
    // the status block's forward / backward group was reset by the last kernel queued
    // before the next forward / backward (the tile scan / the region sort), which that
    // pass then follows as a programmatic dependent instead of after a memset
    bool fwd_group_reset = false, bwd_group_reset = false;
    // host copy of the current plan
    std::vector<CanvasDesc> plan;
    std::vector<int32_t> plan_H, plan_W, plan_off;
    int32_t n_canvas = 0, n_tiles = 0, n_chunks = 0, N = 0, max_tpc = 0;
    int64_t n_pix = 0;
    RenderCfg cfg{16, 32, 2, 2};
    bool persistent = false;
    bool binned = false;
    int32_t row0 = 0, row1 = 0;   // row window of the plan's renders (row1 0: all rows)
    float tune_prune = 0.0f;                // dbmp_autotune: tile sizes timed (0: all)
    const float *params = nullptr;  // of the last binning (gradient finalisation)
    int32_t Hb = 0, Wb = 0;
    float alpha_max = 1.0f;
};

namespace {

// Regions the per-region cost and order arrays hold: a region covers at least 32
// pixels (one per lane), so a pass has at most tile^2 / 32 <= 32 regions per tile, at
// whatever tile size max_tiles was counted.  A pass with more regions than this (more
// tiles than max_tiles) renders in list-length order without recording costs.
int64_t item_capacity(const DbmpLimits &l) { return 32 * (int64_t)l.max_tiles; }

// Entries of the survivor record: one per tile-list entry that passes a region test
// before its warp saturates, which on the workloads measured is under 1/8 of the list
// entries (a forward whose warps need more records fewer regions, never fails).
int64_t surv_capacity(const DbmpLimits &l) {
    return std::min<int64_t>(std::max<int64_t>(l.max_pairs / 8, 1 << 16), ((int64_t)1 << 31) - 1);
}

size_t ws_bytes(const DbmpLimits &l) {
    size_t b = 0;
    b += sizeof(PrimRec) * (size_t)l.max_prims;
    b += sizeof(int4) * (size_t)l.max_prims;
    b += sizeof(float) * 8 * (size_t)l.max_prims;
    b += sizeof(int64_t) * ((size_t)l.max_tiles + 1);
    b += sizeof(int32_t) * (size_t)l.max_tiles;
    b += sizeof(int32_t) * (size_t)l.max_pairs;
    b += sizeof(int32_t) * (size_t)kHistCap;
    b += sizeof(CanvasDesc) * (size_t)l.max_canvases;
    b += sizeof(DevStatus);
    b += sizeof(unsigned long long) * kBinStatsWords;
    b += 2 * sizeof(int32_t) * (size_t)item_capacity(l) + sizeof(int32_t) * 512;
    b += sizeof(int2) * (size_t)surv_capacity(l) + sizeof(int4) * (size_t)item_capacity(l);
    return b;
}

int32_t check_limits(const DbmpLimits *l) {
    if (!l) return fail(DBMP_ERR_INVALID_ARG, "limits is NULL");
    if (l->max_prims < 0 || l->max_tiles < 1 || l->max_pairs < 1 || l->max_canvases < 1)
        return fail(DBMP_ERR_INVALID_ARG, "limits: max_prims >= 0, max_tiles/max_pairs/max_canvases >= 1");
    if (l->max_pairs > ((int64_t)1 << 31) - 1)
        return fail(DBMP_ERR_INVALID_ARG, "limits: max_pairs must fit int32 list positions");
    return DBMP_OK;
}

// Builds canvas descriptors for a plan (host), choosing the binning chunk size so
// the chunk x tile histogram fits its capacity.
int32_t build_plan(DbmpWorkspace *ws, int32_t n, const int32_t *H, const int32_t *W,
                   const int32_t *off, int32_t tile) {
    if (!tile_ok(tile)) return fail(DBMP_ERR_INVALID_ARG, "tile must be 8, 16 or 32 (got %d)", tile);
    if (n < 1 || n > ws->lim.max_canvases)
        return fail(DBMP_ERR_INVALID_ARG, "n_canvas %d outside [1, %d]", n, ws->lim.max_canvases);
    std::vector<CanvasDesc> cv((size_t)n);
    int64_t tiles = 0, pix = 0;
    int32_t max_tpc = 0;
    if (off[0] != 0) return fail(DBMP_ERR_INVALID_ARG, "prim_offset[0] must be 0");
    for (int c = 0; c < n; ++c) {
        if (H[c] < 1 || W[c] < 1) return fail(DBMP_ERR_INVALID_ARG, "canvas %d: H, W must be >= 1", c);
        if (off[c + 1] < off[c]) return fail(DBMP_ERR_INVALID_ARG, "prim_offset must be non-decreasing");
        CanvasDesc &d = cv[c];
        d.H = H[c];
        d.W = W[c];
        d.ntx = (W[c] + tile - 1) / tile;
        d.nty = (H[c] + tile - 1) / tile;
        const int64_t t = (int64_t)d.ntx * d.nty;
        if (t > kMaxTilesPerCanvas)
            return fail(DBMP_ERR_INVALID_ARG, "canvas %d has %lld tiles of %d px (max %d per canvas)", c,
                        (long long)t, tile, kMaxTilesPerCanvas);
        max_tpc = std::max<int32_t>(max_tpc, (int32_t)t);
        d.tile_base = (int32_t)tiles;
        d.prim_base = off[c];
        d.N = off[c + 1] - off[c];
        d.pix_base = pix;
        tiles += t;
        pix += (int64_t)H[c] * W[c];
    }
    const int64_t N = off[n];
    if (N > ws->lim.max_prims)
        return fail(DBMP_ERR_INVALID_ARG, "%lld primitives exceed the workspace limit %d", (long long)N,
                    ws->lim.max_prims);
    if (tiles > ws->lim.max_tiles)
        return fail(DBMP_ERR_INVALID_ARG, "%lld tiles exceed the workspace limit %d", (long long)tiles,
                    ws->lim.max_tiles);
    // smallest common chunk size (>= 512 primitives: fewer, longer runs per tile in the
    // scatter) whose histogram fits.  The count and the scatter do a fixed amount of
    // work per (chunk, tile) pair, so a plan with more than kBinPairsLarge pairs at
    // 512 primitives takes chunks of 1024 (stress canvas, 2048^2 x 200k: binning
    // 0.24 -> 0.19 ms); smaller plans keep 512, whose CTAs fill the GPU better
    // (main workload, 1024^2 x 20k: 0.033 ms against 0.042 ms with 1024).
    int lg = 9;
    {
        int64_t pairs9 = 0;
        for (auto &d : cv) pairs9 += (int64_t)((d.N + 511) >> 9) * d.ntx * d.nty;
        if (pairs9 > kBinPairsLarge) lg = 10;
    }
    for (;; ++lg) {
        if (lg > 24) return fail(DBMP_ERR_INVALID_ARG, "binning histogram does not fit");
        int64_t h = 0;
        for (auto &d : cv) h += (int64_t)((d.N + (1 << lg) - 1) >> lg) * d.ntx * d.nty;
        if (h <= kHistCap) break;
    }
    int64_t hb = 0;
    int32_t chunks = 0;
    for (auto &d : cv) {
        d.chunk_log2 = lg;
        d.n_chunks = (d.N + (1 << lg) - 1) >> lg;
        d.chunk_base = chunks;
        d.hist_base = hb;
        chunks += d.n_chunks;
        hb += (int64_t)d.n_chunks * d.ntx * d.nty;
    }
    for (auto &d : cv) {
        if (!bin_slab_ok(d.ntx, lg))
            return fail(DBMP_ERR_INVALID_ARG, "canvas too wide for binning (%d tiles per row)", d.ntx);
        d.slab_rows = bin_slab_rows(d.ntx, d.nty, lg, chunks);
        d.n_slabs = (d.nty + d.slab_rows - 1) / d.slab_rows;
    }
    ws->plan = cv;
    ws->plan_H.assign(H, H + n);
    ws->plan_W.assign(W, W + n);
    ws->plan_off.assign(off, off + n + 1);
    ws->n_canvas = n;
    ws->n_tiles = (int32_t)tiles;
    ws->n_chunks = chunks;
    ws->N = (int32_t)N;
    ws->max_tpc = max_tpc;
    ws->n_pix = pix;
    ws->cfg.tile = tile;
    return DBMP_OK;
}

__global__ void k_set_canvas(CanvasDesc d, CanvasDesc *dst) { *dst = d; }

int32_t check_atlas(const DbmpAtlas *atlas) {
    if (!atlas || !atlas->plane || !atlas->sat) return fail(DBMP_ERR_INVALID_ARG, "atlas is NULL");
    return DBMP_OK;
}

BinBuffers bin_buffers(DbmpWorkspace *ws) {
    BinBuffers b;
    b.rec = ws->rec;
    b.rect = ws->rect;
    b.hist = ws->hist;
    b.tile_off = ws->tile_off;
    b.list = ws->list;
    b.cap = ws->lim.max_pairs;
    b.tile_order = ws->persistent ? ws->tile_order : nullptr;
    b.status = ws->status;
    b.canvas = ws->canvas;
    b.n_canvas = ws->n_canvas;
    b.n_tiles = ws->n_tiles;
    b.n_chunks = ws->n_chunks;
    b.N = ws->N;
    b.max_tiles_per_canvas = ws->max_tpc;
    b.chunk_log2 = ws->plan.empty() ? 7 : ws->plan[0].chunk_log2;
    b.max_slabs = 1;
    b.smem_count = 16;
    b.smem_scatter = 16;
    for (const auto &d : ws->plan) {
        b.max_slabs = std::max(b.max_slabs, d.n_slabs);
        b.smem_count = std::max<int32_t>(b.smem_count, (int32_t)bin_smem_bytes(d.ntx, d.slab_rows, d.chunk_log2, false));
        b.smem_scatter = std::max<int32_t>(b.smem_scatter, (int32_t)bin_smem_bytes(d.ntx, d.slab_rows, d.chunk_log2, true));
    }
    return b;
}

int32_t do_bin(DbmpWorkspace *ws, const float *params, const int32_t *bid, const DbmpAtlas *atlas,
               float alpha_max, cudaStream_t st) {
    const BinBuffers b = bin_buffers(ws);
    DBMP_CUDA(cudaMemsetAsync(&ws->status->n_degenerate, 0, sizeof(int32_t), st), "status reset");
    DBMP_CUDA(launch_bin(b, params, bid, atlas->view(), alpha_max, ws->cfg.tile, st, true), "bin launch");
    ws->fwd_group_reset = true;
    ws->params = params;
    ws->Hb = atlas->Hb;
    ws->Wb = atlas->Wb;
    ws->alpha_max = alpha_max;
    ws->binned = true;
    ws->surv_items = 0;   // new lists: the survivor record no longer applies
    return DBMP_OK;
}

RenderArgs make_args(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg, float T_stop) {
    RenderArgs a{};
    a.rec = ws->rec;
    a.tile_off = ws->tile_off;
    a.list = ws->list;
    a.tile_order = ws->persistent ? ws->tile_order : nullptr;
    a.canvas = ws->canvas;
    a.n_canvas = ws->n_canvas;
    a.n_tiles = ws->n_tiles;
    a.status = ws->status;
    a.atlas = atlas->view();
    a.bg_mode = bg ? bg->mode : DBMP_BG_NONE;
    if (bg && bg->mode == DBMP_BG_CONST) {
        a.bg0 = bg->rgb[0];
        a.bg1 = bg->rgb[1];
        a.bg2 = bg->rgb[2];
    }
    a.bg_buf = bg ? bg->buf_dev : nullptr;
    a.T_stop = T_stop;
    a.graw = ws->graw;
    a.row0 = ws->row0;
    a.row1 = ws->row1;
    a.n_prims = ws->N;
    a.surv = ws->surv;
    a.surv_tab = ws->surv_tab;
    a.surv_cap = ws->surv_cap;
    a.count_pairs = ws->count_pairs;
    return a;
}

int32_t check_bg(const DbmpBackground *bg) {
    if (!bg) return DBMP_OK;
    if (bg->mode != DBMP_BG_NONE && bg->mode != DBMP_BG_CONST && bg->mode != DBMP_BG_BUFFER)
        return fail(DBMP_ERR_INVALID_ARG, "background mode %d unknown", bg->mode);
    if (bg->mode == DBMP_BG_BUFFER && !bg->buf_dev)
        return fail(DBMP_ERR_INVALID_ARG, "background buffer is NULL");
    return DBMP_OK;
}

int32_t do_fwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg, float T_stop,
               float *image, float *T_final, int32_t *n_last, cudaStream_t st,
               const float *mse_target = nullptr, float *mse_dL = nullptr, double *mse_loss = nullptr) {
    RenderArgs a = make_args(ws, atlas, bg, T_stop);
    a.image = image;
    a.T_final = T_final;
    a.n_last = n_last;
    if (mse_target) {
        int64_t pixels = 0;
        for (int c = 0; c < ws->n_canvas; ++c) pixels += (int64_t)ws->plan_H[c] * ws->plan_W[c];
        const double n = 3.0 * (double)pixels;
        a.mse_target = mse_target;
        a.mse_dL = mse_dL;
        a.mse_loss = mse_loss;
        a.mse_scale = (float)(2.0 / n);
        a.mse_inv_n = 1.0 / n;
        DBMP_CUDA(cudaMemsetAsync(mse_loss, 0, sizeof(double), st), "loss reset");
    }
    // regions in the order of the previous forward's costs (when it had the same
    // regions); this forward records the costs again and the order is re-sorted
    // Regions in cost order pay off when a pass has few regions per warp, where the
    // last ones to finish set the pass' time; with many (a large batch of canvases)
    // there is no tail to shorten and the list-length order keeps a tile's regions
    // together.  The arrays must also hold every region.
    const int32_t items = render_items(ws->cfg, ws->n_tiles, false);
    const bool ordered = items <= ws->item_cap && items <= kOrderMaxRegionsPerSM * sm_count();
    int32_t *hist = ws->item_hist + 256 * ws->hist_half, *next = ws->item_hist + 256 * (1 - ws->hist_half);
    if (ordered) {
        if (ws->order_items == items) a.item_order = ws->item_order;
        a.item_cost = ws->item_cost;
        a.item_hist = hist;
    }
    const bool pdl = ws->fwd_group_reset;
    if (!pdl) DBMP_CUDA(cudaMemsetAsync(&ws->status->pairs_eval_fwd, 0, kFwdGroupBytes, st), "status reset");
    ws->fwd_group_reset = false;
    // survivors recorded for the backward when it composites the same regions
    const bool record = ws->surv && items <= ws->item_cap && ws->cfg.ppt == ws->cfg.bwd_ppt();
    if (!record) a.surv = nullptr;
    ws->surv_items = 0;
    DBMP_CUDA(launch_fwd(a, ws->cfg, st, pdl), "forward launch");
    if (record) ws->surv_items = items;
    if (ordered) {
        DBMP_CUDA(launch_item_order(ws->item_cost, hist, next, ws->item_order, items, ws->status, st),
                  "region order");
        ws->order_items = items;
        ws->hist_half = 1 - ws->hist_half;
        ws->bwd_group_reset = true;
    } else {
        ws->order_items = 0;
        ws->bwd_group_reset = false;
    }
    return DBMP_OK;
}

int32_t do_bwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg, float T_stop,
               const float *dL_dimage, const float *dL_dalpha, const float *T_final,
               const int32_t *n_last, float *dparams, cudaStream_t st) {
    RenderArgs a = make_args(ws, atlas, bg, T_stop);
    a.T_final = const_cast<float *>(T_final);
    a.n_last = const_cast<int32_t *>(n_last);
    a.dL_dimage = dL_dimage;
    a.dL_dalpha = dL_dalpha;
    // the forward's regions in decreasing cost, when the backward has the same regions
    if (ws->order_items > 0 && ws->order_items <= ws->item_cap &&
        ws->order_items == render_items(ws->cfg, ws->n_tiles, true))
        a.item_order = ws->item_order;
    // the forward's survivors, when it recorded them for these regions on these lists
    a.surv_use = ws->surv_items > 0 && ws->surv_items == render_items(ws->cfg, ws->n_tiles, true) &&
                 ws->cfg.ppt == ws->cfg.bwd_ppt();
    const bool pdl = ws->bwd_group_reset;
    if (!pdl) DBMP_CUDA(cudaMemsetAsync(&ws->status->pairs_eval_bwd, 0, kBwdGroupBytes, st), "status reset");
    ws->bwd_group_reset = false;
    DBMP_CUDA(launch_bwd(a, ws->cfg, st, pdl), "backward launch");
    DBMP_CUDA(launch_grad_finalize(ws->params, ws->rec, ws->graw, dparams, ws->N, 0.5f * (float)(atlas->Wb - 1), 0.5f * (float)(atlas->Hb - 1), st), "gradient finalize");
    return DBMP_OK;
}

}  // namespace

extern "C" {

const char *dbmp_last_error(void) { return g_err; }

int32_t dbmp_abi_version(void) { return 1; }

int32_t dbmp_atlas_create(const float *texels_dev, int32_t n_bmp, int32_t H_b, int32_t W_b,
                          dbmp_stream_t stream, DbmpAtlas **out) {
    if (!out) return fail(DBMP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!texels_dev) return fail(DBMP_ERR_INVALID_ARG, "texels_dev is NULL");
    if (n_bmp < 1 || H_b < 2 || W_b < 2)
        return fail(DBMP_ERR_INVALID_ARG, "atlas needs n_bmp >= 1 and H_b, W_b >= 2");
    if ((int64_t)n_bmp * (H_b + 1) * (W_b + 1) > ((int64_t)1 << 31) - 1)
        return fail(DBMP_ERR_INVALID_ARG, "atlas too large for int32 texel offsets");
    bool fits = false;
    if (cudaError_t e = atlas_texture_fits(n_bmp, H_b, W_b, &fits)) return cuda_fail(e, "texture limits");
    if (!fits)
        return fail(DBMP_ERR_INVALID_ARG,
                    "atlas %d x %dx%d exceeds the device's 2-D texture limits (n_bmp (H_b + 1) rows of W_b texels)",
                    n_bmp, H_b, W_b);
    DbmpAtlas *a = new DbmpAtlas;
    a->n_bmp = n_bmp;
    a->Hb = H_b;
    a->Wb = W_b;
    a->pitch = atlas_plane_pitch(W_b);
    const size_t rows = (size_t)n_bmp * (H_b + 1);
    const size_t cells = rows * (W_b + 1);
    cudaError_t e = cudaMalloc(&a->plane_alloc, a->pitch * rows + kTexAlign);
    if (e == cudaSuccess) e = cudaMalloc(&a->sat, sizeof(int32_t) * cells);
    if (e == cudaSuccess) e = cudaMalloc(&a->nzbox, sizeof(int4) * (size_t)n_bmp);
    if (e != cudaSuccess) {
        cudaFree(a->plane_alloc);
        cudaFree(a->sat);
        delete a;
        return fail(DBMP_ERR_NO_MEMORY, "atlas allocation: %s", cudaGetErrorString(e));
    }
    a->plane = reinterpret_cast<float *>(((uintptr_t)a->plane_alloc + kTexAlign - 1) & ~(uintptr_t)(kTexAlign - 1));
    cudaStream_t st = (cudaStream_t)stream;
    e = atlas_texture_create(a->plane, a->pitch, n_bmp, H_b, W_b, &a->tex);
    if (e == cudaSuccess)
        e = launch_atlas_build(texels_dev, a->plane, (int64_t)(a->pitch / sizeof(float)), a->sat, a->nzbox, n_bmp,
                               H_b, W_b, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        if (a->tex) cudaDestroyTextureObject(a->tex);
        cudaFree(a->plane_alloc);
        cudaFree(a->sat);
        delete a;
        return cuda_fail(e, "atlas build");
    }
    *out = a;
    return DBMP_OK;
}

int32_t dbmp_atlas_update(DbmpAtlas *atlas, const float *texels_dev, dbmp_stream_t stream) {
    if (int32_t r = check_atlas(atlas)) return r;
    if (!texels_dev) return fail(DBMP_ERR_INVALID_ARG, "texels_dev is NULL");
    DBMP_CUDA(launch_atlas_build(texels_dev, atlas->plane, (int64_t)(atlas->pitch / sizeof(float)), atlas->sat,
                                 atlas->nzbox, atlas->n_bmp, atlas->Hb, atlas->Wb, (cudaStream_t)stream),
              "atlas update");
    return DBMP_OK;
}

int32_t dbmp_atlas_destroy(DbmpAtlas *atlas) {
    if (!atlas) return DBMP_OK;
    if (atlas->tex) cudaDestroyTextureObject(atlas->tex);
    cudaFree(atlas->plane_alloc);
    cudaFree(atlas->sat);
    cudaFree(atlas->nzbox);
    delete atlas;
    return DBMP_OK;
}

int32_t dbmp_workspace_bytes(const DbmpLimits *limits, size_t *bytes) {
    if (int32_t r = check_limits(limits)) return r;
    if (!bytes) return fail(DBMP_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = ws_bytes(*limits);
    return DBMP_OK;
}

int32_t dbmp_workspace_create(const DbmpLimits *limits, DbmpWorkspace **out) {
    if (!out) return fail(DBMP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (int32_t r = check_limits(limits)) return r;
    DbmpWorkspace *ws = new DbmpWorkspace;
    ws->lim = *limits;
    ws->item_cap = item_capacity(ws->lim);
    const DbmpLimits &l = *limits;
    struct Req {
        void **p;
        size_t n;
    } reqs[] = {
        {(void **)&ws->rec, sizeof(PrimRec) * (size_t)std::max(l.max_prims, 1)},
        {(void **)&ws->rect, sizeof(int4) * (size_t)std::max(l.max_prims, 1)},
        {(void **)&ws->graw, sizeof(float) * 8 * (size_t)std::max(l.max_prims, 1)},
        {(void **)&ws->tile_off, sizeof(int64_t) * ((size_t)l.max_tiles + 1)},
        {(void **)&ws->tile_order, sizeof(int32_t) * (size_t)l.max_tiles},
        {(void **)&ws->list, sizeof(int32_t) * (size_t)l.max_pairs},
        {(void **)&ws->hist, sizeof(int32_t) * (size_t)kHistCap},
        {(void **)&ws->canvas, sizeof(CanvasDesc) * (size_t)l.max_canvases},
        {(void **)&ws->status, sizeof(DevStatus)},
        {(void **)&ws->stats, sizeof(unsigned long long) * kBinStatsWords},
        {(void **)&ws->item_cost, sizeof(int32_t) * (size_t)item_capacity(l)},
        {(void **)&ws->item_order, sizeof(int32_t) * (size_t)item_capacity(l)},
        {(void **)&ws->item_hist, sizeof(int32_t) * 512},
        {(void **)&ws->surv, sizeof(int2) * (size_t)surv_capacity(l)},
        {(void **)&ws->surv_tab, sizeof(int4) * (size_t)item_capacity(l)},
    };
    ws->surv_cap = surv_capacity(l);
    for (auto &r : reqs) {
        cudaError_t e = cudaMalloc(r.p, r.n);
        if (e != cudaSuccess) {
            dbmp_workspace_destroy(ws);
            return fail(DBMP_ERR_NO_MEMORY, "workspace allocation of %zu bytes: %s", r.n,
                        cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMemset(ws->status, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(ws->graw, 0, sizeof(float) * 8 * (size_t)std::max(l.max_prims, 1));
    if (e == cudaSuccess) e = cudaMemset(ws->item_hist, 0, sizeof(int32_t) * 512);
    if (e == cudaSuccess) e = init_bin_kernels(kMaxTilesPerCanvas);
    if (e == cudaSuccess) e = init_render_kernels();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dbmp_workspace_destroy(ws);
        return cuda_fail(e, "workspace init");
    }
    *out = ws;
    return DBMP_OK;
}

int32_t dbmp_workspace_poison(DbmpWorkspace *ws, dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const DbmpLimits &l = ws->lim;
    struct {
        void *p;
        size_t n;
    } bufs[] = {
        {ws->rec, sizeof(PrimRec) * (size_t)std::max(l.max_prims, 1)},
        {ws->rect, sizeof(int4) * (size_t)std::max(l.max_prims, 1)},
        {ws->tile_off, sizeof(int64_t) * ((size_t)l.max_tiles + 1)},
        {ws->tile_order, sizeof(int32_t) * (size_t)l.max_tiles},
        {ws->list, sizeof(int32_t) * (size_t)l.max_pairs},
        {ws->hist, sizeof(int32_t) * (size_t)kHistCap},
        {ws->canvas, sizeof(CanvasDesc) * (size_t)l.max_canvases},
        {ws->stats, sizeof(unsigned long long) * kBinStatsWords},
        {ws->item_cost, sizeof(int32_t) * (size_t)item_capacity(l)},
        {ws->item_order, sizeof(int32_t) * (size_t)item_capacity(l)},
        {ws->item_hist, sizeof(int32_t) * 512},
        {ws->surv, sizeof(int2) * (size_t)surv_capacity(l)},
        {ws->surv_tab, sizeof(int4) * (size_t)item_capacity(l)},
    };
    for (auto &b : bufs) DBMP_CUDA(cudaMemsetAsync(b.p, 0xFF, b.n, st), "poison");
    // the bucket counts are state that must start at zero, not scratch
    DBMP_CUDA(cudaMemsetAsync(ws->item_hist, 0, sizeof(int32_t) * 512, st), "poison");
    ws->order_items = 0;
    ws->surv_items = 0;
    return DBMP_OK;
}

int32_t dbmp_workspace_count_pairs(DbmpWorkspace *ws, int32_t on) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "workspace is NULL");
    ws->count_pairs = on != 0;
    return DBMP_OK;
}

int32_t dbmp_workspace_destroy(DbmpWorkspace *ws) {
    if (!ws) return DBMP_OK;
    void *ptrs[] = {ws->rec,    ws->rect,   ws->graw,      ws->tile_off,   ws->tile_order, ws->list,
                    ws->hist,   ws->canvas, ws->status,    ws->stats,      ws->item_cost,  ws->item_order,
                    ws->item_hist, ws->surv, ws->surv_tab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete ws;
    return DBMP_OK;
}

int32_t dbmp_status_poll(DbmpWorkspace *ws, dbmp_stream_t stream, DbmpDeviceStatus *out) {
    if (!ws || !out) return fail(DBMP_ERR_INVALID_ARG, "ws/out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(cudaStreamSynchronize(st), "status sync");
    DevStatus s;
    DBMP_CUDA(cudaMemcpy(&s, ws->status, sizeof s, cudaMemcpyDeviceToHost), "status copy");
    out->code = s.code;
    out->n_degenerate = s.n_degenerate;
    out->pairs_required = s.pairs_required;
    out->pairs_evaluated = s.pairs_eval_fwd;
    out->pairs_evaluated_bwd = s.pairs_eval_bwd;
    out->pairs_contributing = s.pairs_contrib;
    out->warp_steps = s.warp_steps_fwd;
    out->warp_steps_bwd = s.warp_steps_bwd;
    out->survivors = s.survivors_fwd;
    out->survivors_bwd = s.survivors_bwd;
    out->bad_kind = s.bad_kind;
    out->bad_pad = 0;
    out->bad_index = s.bad_index;
    const int32_t zero = 0;
    DBMP_CUDA(cudaMemcpy(&ws->status->code, &zero, sizeof zero, cudaMemcpyHostToDevice), "status clear");
    if (s.bad_kind) {
        const int64_t z64[2] = {0, 0};   // bad_kind + pad, bad_index
        DBMP_CUDA(cudaMemcpy(&ws->status->bad_kind, z64, sizeof z64, cudaMemcpyHostToDevice), "status clear");
    }
    if (s.code == DBMP_ERR_CAPACITY)
        fail(DBMP_ERR_CAPACITY, "tile lists need %lld entries, workspace holds %lld",
             (long long)s.pairs_required, (long long)ws->lim.max_pairs);
    return s.code;
}

int32_t dbmp_bin(DbmpWorkspace *ws, int32_t H, int32_t W, int32_t tile, const float *params_dev,
                 const int32_t *bitmap_id_dev, int32_t N, const DbmpAtlas *atlas, float alpha_max,
                 dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (int32_t r = check_atlas(atlas)) return r;
    if (N < 0) return fail(DBMP_ERR_INVALID_ARG, "N must be >= 0");
    if (N > 0 && (!params_dev || !bitmap_id_dev))
        return fail(DBMP_ERR_INVALID_ARG, "params_dev / bitmap_id_dev is NULL");
    if (!(alpha_max > 0.0f && alpha_max <= 1.0f))
        return fail(DBMP_ERR_INVALID_ARG, "alpha_max must be in (0, 1]");
    if (N > 0 && (((uintptr_t)params_dev) & 15))
        return fail(DBMP_ERR_INVALID_ARG, "params_dev must be 16-byte aligned");
    const int32_t off[2] = {0, N};
    const bool same = !ws->persistent && ws->n_canvas == 1 && ws->plan_H.size() == 1 && ws->plan_H[0] == H &&
                      ws->plan_W[0] == W && ws->cfg.tile == tile;
    if (int32_t r = build_plan(ws, 1, &H, &W, off, tile)) return r;
    if (!same) {   // another canvas: the region order and the survivor record no longer apply
        ws->order_items = 0;
        ws->surv_items = 0;
    }
    ws->persistent = false;
    cudaStream_t st = (cudaStream_t)stream;
    k_set_canvas<<<1, 1, 0, st>>>(ws->plan[0], ws->canvas);
    DBMP_CUDA(cudaGetLastError(), "plan upload");
    return do_bin(ws, params_dev, bitmap_id_dev, atlas, alpha_max, st);
}

int32_t dbmp_get_tile_lists(DbmpWorkspace *ws, int64_t *offsets_dev, int32_t *list_dev, int64_t cap,
                            int32_t *n_tiles_out, dbmp_stream_t stream) {
    if (!ws || !offsets_dev || (!list_dev && cap > 0))
        return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (!ws->binned) return fail(DBMP_ERR_NOT_READY, "no binning in this workspace");
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(cudaMemcpyAsync(offsets_dev, ws->tile_off, sizeof(int64_t) * ((size_t)ws->n_tiles + 1),
                              cudaMemcpyDeviceToDevice, st),
              "offsets copy");
    const int64_t n = std::min<int64_t>(cap, ws->lim.max_pairs);
    if (n > 0)
        DBMP_CUDA(cudaMemcpyAsync(list_dev, ws->list, sizeof(int32_t) * (size_t)n,
                                  cudaMemcpyDeviceToDevice, st),
                  "list copy");
    if (n_tiles_out) *n_tiles_out = ws->n_tiles;
    return DBMP_OK;
}

int32_t dbmp_render_fwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg,
                        float T_stop, float *image_dev, float *T_final_dev, int32_t *n_last_dev,
                        dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (int32_t r = check_atlas(atlas)) return r;
    if (int32_t r = check_bg(bg)) return r;
    if (!ws->binned) return fail(DBMP_ERR_NOT_READY, "dbmp_render_fwd needs a prior dbmp_bin");
    if (atlas->Hb != ws->Hb || atlas->Wb != ws->Wb)
        return fail(DBMP_ERR_INVALID_ARG, "atlas differs from the binned one");
    if (!image_dev || !T_final_dev || !n_last_dev) return fail(DBMP_ERR_INVALID_ARG, "output is NULL");
    if (!(T_stop >= 0.0f && T_stop < 1.0f)) return fail(DBMP_ERR_INVALID_ARG, "T_stop must be in [0, 1)");
    return do_fwd(ws, atlas, bg, T_stop, image_dev, T_final_dev, n_last_dev, (cudaStream_t)stream);
}

int32_t dbmp_render_bwd(DbmpWorkspace *ws, const DbmpAtlas *atlas, const DbmpBackground *bg,
                        float T_stop, const float *dL_dimage_dev, const float *dL_dalpha_dev,
                        const float *T_final_dev, const int32_t *n_last_dev, float *dparams_dev,
                        dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (int32_t r = check_atlas(atlas)) return r;
    if (int32_t r = check_bg(bg)) return r;
    if (!ws->binned) return fail(DBMP_ERR_NOT_READY, "dbmp_render_bwd needs a prior dbmp_bin");
    if (!dL_dimage_dev || !T_final_dev || !n_last_dev || (!dparams_dev && ws->N > 0))
        return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (!(T_stop >= 0.0f && T_stop < 1.0f)) return fail(DBMP_ERR_INVALID_ARG, "T_stop must be in [0, 1)");
    return do_bwd(ws, atlas, bg, T_stop, dL_dimage_dev, dL_dalpha_dev, T_final_dev, n_last_dev,
                  dparams_dev, (cudaStream_t)stream);
}

int32_t dbmp_mse_grad(const float *image_dev, const float *target_dev, int64_t n, float *dL_dI_dev,
                      double *loss_dev, dbmp_stream_t stream) {
    if (n < 0) return fail(DBMP_ERR_INVALID_ARG, "n must be >= 0");
    if (!loss_dev || (n > 0 && (!image_dev || !target_dev || !dL_dI_dev)))
        return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    DBMP_CUDA(launch_mse_grad(image_dev, target_dev, n, dL_dI_dev, loss_dev, (cudaStream_t)stream),
              "mse launch");
    return DBMP_OK;
}

int32_t dbmp_adam_step(float *params_dev, float *grad_dev, float *m_dev, float *v_dev,
                       int32_t N, int32_t *step_dev, const DbmpAdamConfig *cfg, dbmp_stream_t stream) {
    if (!cfg || !step_dev) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (N < 0) return fail(DBMP_ERR_INVALID_ARG, "N must be >= 0");
    if (N > 0 && (!params_dev || !grad_dev || !m_dev || !v_dev))
        return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (!(cfg->beta1 >= 0 && cfg->beta1 < 1 && cfg->beta2 >= 0 && cfg->beta2 < 1 && cfg->eps > 0))
        return fail(DBMP_ERR_INVALID_ARG, "Adam betas must be in [0, 1) and eps > 0");
    DBMP_CUDA(launch_adam(params_dev, grad_dev, m_dev, v_dev, N, step_dev, *cfg, (cudaStream_t)stream),
              "adam launch");
    return DBMP_OK;
}

int32_t dbmp_batch_plan(DbmpWorkspace *ws, int32_t n_canvas, const int32_t *H, const int32_t *W,
                        const int32_t *prim_offset, const DbmpTuning *tuning, dbmp_stream_t stream) {
    if (!ws || !H || !W || !prim_offset) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    RenderCfg cfg{16, 32, 2, 2};
    if (tuning) cfg = RenderCfg{tuning->tile, tuning->batch, tuning->ppt, tuning->ppt_bwd ? tuning->ppt_bwd : tuning->ppt};
    if (!render_cfg_supported(cfg))
        return fail(DBMP_ERR_INVALID_ARG, "unsupported tuning (tile %d, batch %d, ppt %d, ppt_bwd %d)", cfg.tile,
                    cfg.batch, cfg.ppt, cfg.ppt_bwd);
    if (int32_t r = build_plan(ws, n_canvas, H, W, prim_offset, cfg.tile)) return r;
    ws->cfg = cfg;
    ws->persistent = true;
    ws->binned = false;
    ws->row0 = ws->row1 = 0;
    ws->order_items = 0;
    ws->surv_items = 0;
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(cudaStreamSynchronize(st), "plan sync");
    DBMP_CUDA(cudaMemcpy(ws->canvas, ws->plan.data(), sizeof(CanvasDesc) * ws->plan.size(),
                         cudaMemcpyHostToDevice),
              "plan upload");
    return DBMP_OK;
}

}  // extern "C"

namespace {

// dbmp_batch_render, and with target_dev the MSE loss fused into the forward.
int32_t batch_render(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                     const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg, float T_stop,
                     int32_t mode, float *image_dev, float *T_final_dev, int32_t *n_last_dev,
                     const float *dL_dimage_dev, float *dparams_dev, const float *target_dev, float *dL_out_dev,
                     double *loss_dev, dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (!ws->persistent || ws->n_canvas < 1)
        return fail(DBMP_ERR_NOT_READY, "dbmp_batch_render needs dbmp_batch_plan first");
    if (int32_t r = check_atlas(atlas)) return r;
    if (int32_t r = check_bg(bg)) return r;
    if (mode & ~(DBMP_BATCH_BIN | DBMP_BATCH_FWD | DBMP_BATCH_BWD) || mode == 0)
        return fail(DBMP_ERR_INVALID_ARG, "mode must be an OR of BIN, FWD, BWD");
    if (!(alpha_max > 0.0f && alpha_max <= 1.0f))
        return fail(DBMP_ERR_INVALID_ARG, "alpha_max must be in (0, 1]");
    if (!(T_stop >= 0.0f && T_stop < 1.0f)) return fail(DBMP_ERR_INVALID_ARG, "T_stop must be in [0, 1)");
    cudaStream_t st = (cudaStream_t)stream;
    if (mode & DBMP_BATCH_BIN) {
        if (ws->N > 0 && (!params_dev || !bitmap_id_dev))
            return fail(DBMP_ERR_INVALID_ARG, "params_dev / bitmap_id_dev is NULL");
        if (ws->N > 0 && (((uintptr_t)params_dev) & 15))
            return fail(DBMP_ERR_INVALID_ARG, "params_dev must be 16-byte aligned");
        if (int32_t r = do_bin(ws, params_dev, bitmap_id_dev, atlas, alpha_max, st)) return r;
    } else if (!ws->binned) {
        return fail(DBMP_ERR_NOT_READY, "no binning for this plan yet (include DBMP_BATCH_BIN)");
    }
    if (mode & (DBMP_BATCH_FWD | DBMP_BATCH_BWD)) {
        if (!T_final_dev || !n_last_dev) return fail(DBMP_ERR_INVALID_ARG, "T_final / n_last is NULL");
    }
    if (mode & DBMP_BATCH_FWD) {
        if (!image_dev) return fail(DBMP_ERR_INVALID_ARG, "image is NULL");
        if (int32_t r = do_fwd(ws, atlas, bg, T_stop, image_dev, T_final_dev, n_last_dev, st, target_dev,
                               dL_out_dev, loss_dev))
            return r;
    }
    if (mode & DBMP_BATCH_BWD) {
        if (!dL_dimage_dev || (!dparams_dev && ws->N > 0))
            return fail(DBMP_ERR_INVALID_ARG, "dL_dimage / dparams is NULL");
        if (int32_t r = do_bwd(ws, atlas, bg, T_stop, dL_dimage_dev, nullptr, T_final_dev, n_last_dev,
                               dparams_dev, st))
            return r;
    }
    return DBMP_OK;
}

}  // namespace

extern "C" {

int32_t dbmp_batch_render(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                          const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg,
                          float T_stop, int32_t mode, float *image_dev, float *T_final_dev,
                          int32_t *n_last_dev, const float *dL_dimage_dev, float *dparams_dev,
                          dbmp_stream_t stream) {
    return batch_render(ws, params_dev, bitmap_id_dev, atlas, alpha_max, bg, T_stop, mode, image_dev, T_final_dev,
                        n_last_dev, dL_dimage_dev, dparams_dev, nullptr, nullptr, nullptr, stream);
}

int32_t dbmp_batch_render_mse(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                              const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg, float T_stop,
                              int32_t mode, const float *target_dev, float *image_dev, float *T_final_dev,
                              int32_t *n_last_dev, float *dL_dimage_dev, float *dparams_dev, double *loss_dev,
                              dbmp_stream_t stream) {
    if (!(mode & DBMP_BATCH_FWD)) return fail(DBMP_ERR_INVALID_ARG, "dbmp_batch_render_mse needs DBMP_BATCH_FWD");
    if (!target_dev || !dL_dimage_dev || !loss_dev)
        return fail(DBMP_ERR_INVALID_ARG, "target / dL_dimage / loss is NULL");
    return batch_render(ws, params_dev, bitmap_id_dev, atlas, alpha_max, bg, T_stop, mode, image_dev, T_final_dev,
                        n_last_dev, dL_dimage_dev, dparams_dev, target_dev, dL_dimage_dev, loss_dev, stream);
}

int32_t dbmp_index_checks(void) { return DBMP_CHECKED; }

int32_t dbmp_workspace_debug_set(DbmpWorkspace *ws, int32_t what, int64_t index, int64_t value,
                                 dbmp_stream_t stream) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    // the value is copied from this call's host memory, so the call synchronises
    // `stream` before returning
    if (what == 0) {
        if (index < 0 || index > ws->lim.max_tiles) return fail(DBMP_ERR_INVALID_ARG, "tile offset %lld outside the workspace", (long long)index);
        DBMP_CUDA(cudaMemcpyAsync(ws->tile_off + index, &value, sizeof(int64_t), cudaMemcpyHostToDevice, st), "poke");
    } else if (what == 1 || what == 2) {
        const int64_t cap = what == 1 ? ws->lim.max_pairs : std::max(ws->lim.max_prims, 1);
        if (index < 0 || index >= cap) return fail(DBMP_ERR_INVALID_ARG, "index %lld outside the workspace", (long long)index);
        if (value < INT32_MIN || value > INT32_MAX) return fail(DBMP_ERR_INVALID_ARG, "value outside int32");
        const int32_t v = (int32_t)value;
        int32_t *dst = what == 1 ? ws->list + index : &ws->rec[index].bmp_row;
        DBMP_CUDA(cudaMemcpyAsync(dst, &v, sizeof v, cudaMemcpyHostToDevice, st), "poke");
        DBMP_CUDA(cudaStreamSynchronize(st), "poke sync");
        return DBMP_OK;
    } else {
        return fail(DBMP_ERR_INVALID_ARG, "what must be 0 (tile offset), 1 (list entry) or 2 (bitmap row)");
    }
    DBMP_CUDA(cudaStreamSynchronize(st), "poke sync");
    return DBMP_OK;
}

int32_t dbmp_batch_set_rows(DbmpWorkspace *ws, int32_t y0, int32_t y1) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (!ws->persistent || ws->n_canvas < 1) return fail(DBMP_ERR_NOT_READY, "dbmp_batch_set_rows needs a plan");
    const int32_t t = ws->cfg.tile;
    if (y0 == 0 && y1 == 0) {
        ws->row0 = ws->row1 = 0;
        return DBMP_OK;
    }
    if (y0 < 0 || y1 <= y0 || y0 % t != 0 || y1 % t != 0)
        return fail(DBMP_ERR_INVALID_ARG, "row window [%d, %d) must be non-empty multiples of the tile size %d", y0,
                    y1, t);
    ws->row0 = y0;
    ws->row1 = y1;
    return DBMP_OK;
}

int32_t dbmp_autotune_set_prune(DbmpWorkspace *ws, float max_pairs_ratio) {
    if (!ws) return fail(DBMP_ERR_INVALID_ARG, "ws is NULL");
    if (!(max_pairs_ratio >= 0.0f) || !std::isfinite(max_pairs_ratio))
        return fail(DBMP_ERR_INVALID_ARG, "max_pairs_ratio must be finite and >= 0");
    ws->tune_prune = max_pairs_ratio;
    return DBMP_OK;
}

int32_t dbmp_autotune(DbmpWorkspace *ws, const float *params_dev, const int32_t *bitmap_id_dev,
                      const DbmpAtlas *atlas, float alpha_max, const DbmpBackground *bg, float T_stop,
                      int32_t mode, float *image_dev, float *T_final_dev, int32_t *n_last_dev,
                      const float *dL_dimage_dev, float *dparams_dev, int32_t reps, DbmpTuning *best,
                      float *best_ms, dbmp_stream_t stream) {
    if (!ws || !best) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (!ws->persistent || ws->n_canvas < 1)
        return fail(DBMP_ERR_NOT_READY, "dbmp_autotune needs dbmp_batch_plan first");
    if (reps < 1) reps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<int32_t> H = ws->plan_H, W = ws->plan_W, off = ws->plan_off;
    const int n = ws->n_canvas;
    cudaEvent_t e0, e1;
    DBMP_CUDA(cudaEventCreate(&e0), "event");
    DBMP_CUDA(cudaEventCreate(&e1), "event");
    float best_t = 1e30f;
    DbmpTuning bt{ws->cfg.tile, ws->cfg.batch, ws->cfg.ppt, ws->cfg.ppt_bwd};
    int32_t tiles[] = {8, 16, 32};
    int n_tiles_try = 3;
    if (ws->tune_prune > 0.0f) {
        // Tile-density guided: the list entries sum_t d_t (Sec. S4) of one binning per
        // tile size set the order, and sizes above tune_prune x the fewest are not timed.
        int64_t pairs[3] = {-1, -1, -1};
        int64_t fewest = -1;
        for (int i = 0; i < 3; ++i) {
            DbmpTuning c{tiles[i], 32, 1, 1};
            if (dbmp_batch_plan(ws, n, H.data(), W.data(), off.data(), &c, stream) != DBMP_OK) continue;
            if (dbmp_batch_render(ws, params_dev, bitmap_id_dev, atlas, alpha_max, bg, T_stop, DBMP_BATCH_BIN,
                                  image_dev, T_final_dev, n_last_dev, dL_dimage_dev, dparams_dev, stream) != DBMP_OK)
                continue;
            DbmpDeviceStatus s0;
            DbmpBinStats bs;
            if (dbmp_status_poll(ws, stream, &s0) != DBMP_OK) continue;   // e.g. capacity: not a candidate
            if (dbmp_bin_stats(ws, stream, &bs) != DBMP_OK) continue;
            pairs[i] = bs.pairs;
            if (fewest < 0 || bs.pairs < fewest) fewest = bs.pairs;
        }
        n_tiles_try = 0;
        int32_t kept[3];
        int64_t kp[3];
        for (int i = 0; i < 3; ++i) {
            if (pairs[i] < 0 || (double)pairs[i] > (double)ws->tune_prune * (double)std::max<int64_t>(fewest, 1))
                continue;
            int j = n_tiles_try++;   // insertion by increasing entries
            while (j > 0 && kp[j - 1] > pairs[i]) {
                kept[j] = kept[j - 1];
                kp[j] = kp[j - 1];
                --j;
            }
            kept[j] = tiles[i];
            kp[j] = pairs[i];
        }
        for (int i = 0; i < n_tiles_try; ++i) tiles[i] = kept[i];
    }
    const int32_t batches[] = {32, 64};
    const int32_t ppts[] = {1, 2, 4};
    const bool want_f = (mode & DBMP_BATCH_FWD) != 0, want_b = (mode & DBMP_BATCH_BWD) != 0;
    int32_t rc = DBMP_OK;
    // mean time of `reps` renders of `m`; < 0 on a launch error (rc set)
    auto time_mode = [&](int32_t m) -> float {
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
            dbmp_batch_render(ws, params_dev, bitmap_id_dev, atlas, alpha_max, bg, T_stop, m, image_dev,
                              T_final_dev, n_last_dev, dL_dimage_dev, dparams_dev, stream);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            return -1.0f;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / (float)reps;
    };
    for (int ti = 0; ti < n_tiles_try; ++ti) {
        const int32_t t = tiles[ti];
        for (int32_t b : batches) {
            float bin_ms = -1.0f, f_best = 1e30f, g_best = 1e30f;
            int32_t pf = 0, pb = 0;
            for (int32_t p : ppts) {
                if (!render_cfg_supported(RenderCfg{t, b, p, p})) continue;
                DbmpTuning cand{t, b, p, p};
                if (dbmp_batch_plan(ws, n, H.data(), W.data(), off.data(), &cand, stream) != DBMP_OK) continue;
                // warm-up (also validates the capacity for this tile size)
                rc = dbmp_batch_render(ws, params_dev, bitmap_id_dev, atlas, alpha_max, bg, T_stop,
                                       mode | DBMP_BATCH_BIN, image_dev, T_final_dev, n_last_dev,
                                       dL_dimage_dev, dparams_dev, stream);
                if (rc != DBMP_OK) break;
                DbmpDeviceStatus s;
                if (dbmp_status_poll(ws, stream, &s) != DBMP_OK) break;  // e.g. capacity: skip the tile
                if (bin_ms < 0.0f && (bin_ms = time_mode(DBMP_BATCH_BIN)) < 0.0f) break;
                if (want_f) {
                    const float f = time_mode(DBMP_BATCH_FWD);
                    if (f < 0.0f) break;
                    if (f < f_best) f_best = f, pf = p;
                }
                if (want_b) {
                    const float g = time_mode(DBMP_BATCH_BWD);
                    if (g < 0.0f) break;
                    if (g < g_best) g_best = g, pb = p;
                }
            }
            if (rc != DBMP_OK) break;
            if (bin_ms < 0.0f) continue;
            if (!want_f) pf = pb ? pb : 2;
            if (!want_b) pb = pf;
            const float total = bin_ms + (want_f ? f_best : 0.0f) + (want_b ? g_best : 0.0f);
            if (total < best_t) {
                best_t = total;
                bt = DbmpTuning{t, b, pf, pb};
            }
        }
        if (rc != DBMP_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DBMP_OK) return rc;
    if (best_t >= 1e30f) return fail(DBMP_ERR_CAPACITY, "no (tile, batch) candidate fits the workspace");
    *best = bt;
    if (best_ms) *best_ms = best_t;
    return dbmp_batch_plan(ws, n, H.data(), W.data(), off.data(), &bt, stream);
}

int32_t dbmp_bin_stats(DbmpWorkspace *ws, dbmp_stream_t stream, DbmpBinStats *out) {
    if (!ws || !out) return fail(DBMP_ERR_INVALID_ARG, "ws / out is NULL");
    if (!ws->binned || (ws->N > 0 && !ws->params)) return fail(DBMP_ERR_NOT_READY, "no binning in this workspace yet");
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(launch_bin_stats(bin_buffers(ws), ws->params, ws->Hb, ws->Wb, ws->stats, st), "stats launch");
    unsigned long long h[kBinStatsWords];
    DBMP_CUDA(cudaMemcpyAsync(h, ws->stats, sizeof h, cudaMemcpyDeviceToHost, st), "stats copy");
    DBMP_CUDA(cudaStreamSynchronize(st), "stats sync");
    out->n_listed = (int64_t)h[0];
    out->pairs = (int64_t)h[1];
    out->tau_max = (int64_t)h[2];
    out->d_max = (int64_t)h[3];
    out->n_tiles = (int64_t)h[4];
    out->empty_tiles = (int64_t)h[5];
    for (int b = 0; b < 32; ++b) {
        out->tau_hist[b] = (int64_t)h[8 + b];
        out->d_hist[b] = (int64_t)h[40 + b];
        out->foot_hist[b] = (int64_t)h[72 + b];
    }
    return DBMP_OK;
}

int32_t dbmp_blur_bitmaps(const float *texels_dev, int32_t n_bmp, int32_t H_b, int32_t W_b, float sigma,
                          float *out_dev, dbmp_stream_t stream) {
    if (!texels_dev || !out_dev) return fail(DBMP_ERR_INVALID_ARG, "texels / out is NULL");
    if (n_bmp < 1 || n_bmp > 65535 || H_b < 1 || W_b < 1)
        return fail(DBMP_ERR_INVALID_ARG, "need 1 <= n_bmp <= 65535 and H_b, W_b >= 1");
    if (!(sigma > 0.0f && sigma <= 5.0f)) return fail(DBMP_ERR_INVALID_ARG, "sigma must be in (0, 5]");
    const size_t bytes = sizeof(float) * (size_t)n_bmp * H_b * W_b;
    const char *a = reinterpret_cast<const char *>(texels_dev), *b = reinterpret_cast<const char *>(out_dev);
    if (a < b + bytes && b < a + bytes) return fail(DBMP_ERR_INVALID_ARG, "out overlaps texels");
    DBMP_CUDA(launch_blur(texels_dev, out_dev, n_bmp, H_b, W_b, blur_taps(sigma), (cudaStream_t)stream),
              "blur launch");
    return DBMP_OK;
}

int32_t dbmp_structure_init_scratch_bytes(int32_t H, int32_t W, size_t *bytes) {
    if (!bytes) return fail(DBMP_ERR_INVALID_ARG, "bytes is NULL");
    if (H < 1 || W < 1 || (int64_t)H * W > 2147483647LL)
        return fail(DBMP_ERR_INVALID_ARG, "H, W must be >= 1 with H W < 2^31");
    *bytes = structure_init_scratch((int64_t)H * W);
    return DBMP_OK;
}

namespace {
int32_t check_structure_args(const float *image_dev, int32_t H, int32_t W, int32_t N, const double *u_pos_dev,
                             const double *u_theta_dev, const double *n_color_dev, double s_min, double s_max,
                             double sigma_c, void *scratch_dev, float *params_dev) {
    if (H < 1 || W < 1 || (int64_t)H * W > 2147483647LL)
        return fail(DBMP_ERR_INVALID_ARG, "H, W must be >= 1 with H W < 2^31");
    if (N < 0) return fail(DBMP_ERR_INVALID_ARG, "N must be >= 0");
    if (!image_dev || !scratch_dev) return fail(DBMP_ERR_INVALID_ARG, "image / scratch is NULL");
    if (N > 0 && (!u_pos_dev || !u_theta_dev || !n_color_dev || !params_dev))
        return fail(DBMP_ERR_INVALID_ARG, "random draws / params is NULL");
    if (((uintptr_t)scratch_dev) & 255) return fail(DBMP_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    if (!(s_min <= s_max) || !(sigma_c >= 0.0)) return fail(DBMP_ERR_INVALID_ARG, "need s_min <= s_max, sigma_c >= 0");
    return DBMP_OK;
}
}  // namespace

int32_t dbmp_structure_reinit(const float *image_dev, const float *mask_dev, int32_t H, int32_t W, int32_t N,
                              const double *u_pos_dev, const double *u_theta_dev, const double *n_color_dev,
                              double s_min, double s_max, double sigma_c, double nu, double threshold,
                              void *scratch_dev, float *params_dev, float *adam_m_dev, float *adam_v_dev,
                              int32_t *count_dev, dbmp_stream_t stream) {
    if (int32_t r = check_structure_args(image_dev, H, W, N, u_pos_dev, u_theta_dev, n_color_dev, s_min, s_max,
                                         sigma_c, scratch_dev, params_dev))
        return r;
    if (!(threshold >= 0.0 && threshold <= 1.0)) return fail(DBMP_ERR_INVALID_ARG, "threshold must be in [0, 1]");
    DBMP_CUDA(launch_structure_init(image_dev, mask_dev, H, W, N, u_pos_dev, u_theta_dev, n_color_dev, s_min, s_max,
                                    sigma_c, nu, scratch_dev, params_dev, nullptr, threshold, adam_m_dev,
                                    adam_v_dev, count_dev, (cudaStream_t)stream),
              "structure reinit launch");
    return DBMP_OK;
}

int32_t dbmp_render_alpha(const float *T_final_dev, float *alpha_dev, int64_t n_pix, dbmp_stream_t stream) {
    if (n_pix < 0) return fail(DBMP_ERR_INVALID_ARG, "n_pix must be >= 0");
    if (n_pix > 0 && (!T_final_dev || !alpha_dev)) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    DBMP_CUDA(launch_alpha_from_T(T_final_dev, alpha_dev, n_pix, (cudaStream_t)stream), "alpha launch");
    return DBMP_OK;
}

int32_t dbmp_alpha_loss_grad(const float *image_dev, const float *T_final_dev, const float *target_dev,
                             const float *target_alpha_dev, int64_t n_pix, float lambda_alpha, float *dL_dimage_dev,
                             float *dL_dalpha_dev, double *loss_dev, dbmp_stream_t stream) {
    if (n_pix < 0) return fail(DBMP_ERR_INVALID_ARG, "n_pix must be >= 0");
    if (!image_dev || !T_final_dev || !target_dev || !target_alpha_dev || !dL_dimage_dev || !dL_dalpha_dev || !loss_dev)
        return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (!(lambda_alpha >= 0.0f)) return fail(DBMP_ERR_INVALID_ARG, "lambda_alpha must be >= 0");
    DBMP_CUDA(launch_alpha_loss(image_dev, T_final_dev, target_dev, target_alpha_dev, n_pix, lambda_alpha,
                                dL_dimage_dev, dL_dalpha_dev, loss_dev, (cudaStream_t)stream),
              "alpha loss launch");
    return DBMP_OK;
}

int32_t dbmp_structure_init(const float *image_dev, const float *mask_dev, int32_t H, int32_t W, int32_t N,
                            const double *u_pos_dev, const double *u_theta_dev, const double *n_color_dev,
                            double s_min, double s_max, double sigma_c, double nu, void *scratch_dev,
                            float *params_dev, double *nlv_dev, dbmp_stream_t stream) {
    if (int32_t r = check_structure_args(image_dev, H, W, N, u_pos_dev, u_theta_dev, n_color_dev, s_min, s_max,
                                         sigma_c, scratch_dev, params_dev))
        return r;
    DBMP_CUDA(launch_structure_init(image_dev, mask_dev, H, W, N, u_pos_dev, u_theta_dev, n_color_dev, s_min, s_max,
                                    sigma_c, nu, scratch_dev, params_dev, nlv_dev, -1.0, nullptr, nullptr, nullptr,
                                    (cudaStream_t)stream),
              "structure init launch");
    return DBMP_OK;
}

int32_t dbmp_gemm_bf16(const uint16_t *A_dev, int32_t lda, const uint16_t *B_dev, int32_t ldb, int32_t M,
                       int32_t N, int32_t K, int32_t mode, float *Cf_dev, uint16_t *Cb_dev, int32_t ldc,
                       const float *bias_dev, int32_t split_k, int32_t *status_dev, dbmp_stream_t stream) {
    if (!A_dev || !B_dev) return fail(DBMP_ERR_INVALID_ARG, "A / B is NULL");
    if (M < 1 || N < 1 || K < 64 || K % 64) return fail(DBMP_ERR_INVALID_ARG, "need M, N >= 1 and K a multiple of 64");
    const int a_mn = (mode & GEMM_A_MN) != 0, b_mn = (mode & GEMM_B_MN) != 0;
    const int stall = (mode & GEMM_TEST_STALL) != 0;
    mode &= ~(GEMM_A_MN | GEMM_B_MN | GEMM_TEST_STALL);
    if (lda < (a_mn ? M : K) || ldb < (b_mn ? N : K) || (lda & 7) || (ldb & 7) || (((uintptr_t)A_dev) & 15) ||
        (((uintptr_t)B_dev) & 15))
        return fail(DBMP_ERR_INVALID_ARG,
                    "A / B rows must be 16-byte aligned, lda / ldb multiples of 8 and >= the contiguous extent");
    if (mode < 0 || mode > 4) return fail(DBMP_ERR_INVALID_ARG, "mode must be 0..4 (+ flags 16, 32, 64)");
    if (ldc < N) return fail(DBMP_ERR_INVALID_ARG, "ldc < N");
    const bool bf16_out = mode == 2 || mode == 4;
    if ((bf16_out && !Cb_dev) || (!bf16_out && !Cf_dev)) return fail(DBMP_ERR_INVALID_ARG, "output is NULL");
    if ((mode == 2 || mode == 3) && !bias_dev) return fail(DBMP_ERR_INVALID_ARG, "bias is NULL");
    if (split_k < 1 || (split_k > 1 && mode != 1)) return fail(DBMP_ERR_INVALID_ARG, "split_k > 1 needs mode 1");
    DBMP_CUDA(init_gemm_kernels(), "gemm set-up");
    GemmArgs g{A_dev, B_dev, M, N, K, lda, ldb, ldc, mode, a_mn, b_mn, Cf_dev, Cb_dev, bias_dev, status_dev};
    g.stall = stall;
    DBMP_CUDA(launch_gemm(g, split_k, (cudaStream_t)stream), "gemm launch");
    return DBMP_OK;
}

struct DbmpProposer {
    CnnBuffers c;
    int32_t step = 0;
    int32_t last_batch = 0;   // batch of the last forward (dbmp_propose / train step)
};

int64_t dbmp_proposer_num_params(void) { return cnn_num_params(); }

int32_t dbmp_proposer_create(int32_t max_batch, DbmpProposer **out) {
    if (!out) return fail(DBMP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1) return fail(DBMP_ERR_INVALID_ARG, "max_batch must be >= 1");
    DbmpProposer *p = new DbmpProposer;
    cudaError_t e = cnn_alloc(p->c, max_batch);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cnn_free(p->c);
        delete p;
        return fail(DBMP_ERR_NO_MEMORY, "proposer allocation (%zu bytes): %s", cnn_bytes(max_batch),
                    cudaGetErrorString(e));
    }
    *out = p;
    return DBMP_OK;
}

int32_t dbmp_proposer_destroy(DbmpProposer *p) {
    if (!p) return DBMP_OK;
    cudaDeviceSynchronize();
    cnn_free(p->c);
    delete p;
    return DBMP_OK;
}

int32_t dbmp_proposer_set_params(DbmpProposer *p, const float *host, int64_t n) {
    if (!p || !host) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    const int64_t np = cnn_num_params();
    if (n != np) return fail(DBMP_ERR_INVALID_ARG, "expected %lld parameters, got %lld", (long long)np, (long long)n);
    DBMP_CUDA(cudaMemcpy(p->c.theta, host, sizeof(float) * np, cudaMemcpyHostToDevice), "params upload");
    DBMP_CUDA(cudaMemset(p->c.m, 0, sizeof(float) * np), "adam reset");
    DBMP_CUDA(cudaMemset(p->c.v, 0, sizeof(float) * np), "adam reset");
    DBMP_CUDA(cnn_sync_weights(p->c, 0), "bf16 copies");
    DBMP_CUDA(cudaDeviceSynchronize(), "params sync");
    p->step = 0;
    return DBMP_OK;
}

int32_t dbmp_proposer_get(DbmpProposer *p, int32_t which, float *host, int64_t n) {
    if (!p || !host) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    const int64_t np = cnn_num_params();
    if (n != np) return fail(DBMP_ERR_INVALID_ARG, "expected %lld values, got %lld", (long long)np, (long long)n);
    if (which != 0 && which != 1) return fail(DBMP_ERR_INVALID_ARG, "which must be 0 (params) or 1 (grads)");
    DBMP_CUDA(cudaDeviceSynchronize(), "sync");
    DBMP_CUDA(cudaMemcpy(host, which == 0 ? p->c.theta : p->c.grad, sizeof(float) * np, cudaMemcpyDeviceToHost),
              "download");
    int32_t st = 0;
    DBMP_CUDA(cudaMemcpy(&st, p->c.status, sizeof st, cudaMemcpyDeviceToHost), "status");
    if (st) return fail(st, "a tensor-core wait gave up");
    return DBMP_OK;
}

int32_t dbmp_propose(DbmpProposer *p, const float *images_dev, int32_t B, float *params_out_dev,
                     dbmp_stream_t stream) {
    if (!p || !images_dev || !params_out_dev) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (B < 1 || B > p->c.max_batch) return fail(DBMP_ERR_INVALID_ARG, "B = %d outside 1..%d", B, p->c.max_batch);
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(cnn_forward(p->c, images_dev, B, st), "proposer forward");
    DBMP_CUDA(cnn_decode(p->c, B, params_out_dev, st), "proposer decode");
    p->last_batch = B;
    return DBMP_OK;
}

int32_t dbmp_proposer_activations(DbmpProposer *p, int32_t layer, float *host, int64_t n) {
    if (!p || !host) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (p->last_batch < 1) return fail(DBMP_ERR_NOT_READY, "no forward of the proposer yet");
    const int64_t want = cnn_activation_count(layer, p->last_batch);
    if (want < 0) return fail(DBMP_ERR_INVALID_ARG, "layer %d outside 0..6", layer);
    if (n != want) return fail(DBMP_ERR_INVALID_ARG, "expected %lld values, got %lld", (long long)want, (long long)n);
    DBMP_CUDA(cudaDeviceSynchronize(), "sync");
    DBMP_CUDA(cnn_activation(p->c, layer, p->last_batch, host), "download");
    return DBMP_OK;
}

int32_t dbmp_proposer_train_step(DbmpProposer *p, const float *images_dev, const float *target_params_dev,
                                 int32_t B, const DbmpProposerAdam *adam, double *loss_dev, dbmp_stream_t stream) {
    if (!p || !images_dev || !target_params_dev || !loss_dev) return fail(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (B < 1 || B > p->c.max_batch) return fail(DBMP_ERR_INVALID_ARG, "B = %d outside 1..%d", B, p->c.max_batch);
    if (adam && !(adam->lr >= 0 && adam->beta1 >= 0 && adam->beta1 < 1 && adam->beta2 >= 0 && adam->beta2 < 1 &&
                  adam->eps > 0))
        return fail(DBMP_ERR_INVALID_ARG, "bad Adam settings");
    cudaStream_t st = (cudaStream_t)stream;
    DBMP_CUDA(cnn_forward(p->c, images_dev, B, st), "proposer forward");
    p->last_batch = B;
    DBMP_CUDA(cnn_backward(p->c, target_params_dev, B, loss_dev, st), "proposer backward");
    if (adam) {
        p->step += 1;
        DBMP_CUDA(cnn_adam(p->c, adam->lr, adam->beta1, adam->beta2, adam->eps, p->step, st), "proposer adam");
    }
    return DBMP_OK;
}

}  // extern "C"
