// dbmp_render_fwd_static: the forward render of one canvas without any device
// allocation, for callers that must not allocate (see include/dbmp.h).
//
// All intermediate state (bitmap sampling layout, per-primitive records, tile
// lists, histograms, status) lives in one file-scope __device__ array of fixed
// size.  Host code cannot use the array's name as a device address, so the first
// call on each device resolves it with cudaGetSymbolAddress (with that device
// current) and caches the pointer; the kernels then receive ordinary pointers
// into it.  The binning and compositing kernels are the library's usual ones.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "dbmp_internal.cuh"

using namespace dbmp;

namespace {

// Stated maximum sizes of one call.
constexpr int32_t kMaxPrims = 4096;
constexpr int32_t kMaxSide = 512;
constexpr int32_t kTile = 16;
constexpr int32_t kMaxTiles = (kMaxSide / kTile) * (kMaxSide / kTile);   // 1024
constexpr int64_t kMaxPairs = 1 << 20;                                  // tile-list entries
constexpr int64_t kMaxAtlasCells = 32768;                               // n_bmp (H_b+1)(W_b+1)
constexpr int32_t kChunkLog2 = 7;                                       // 128 primitives per chunk
constexpr int32_t kMaxChunks = kMaxPrims >> kChunkLog2;                 // 32

constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffCanvas = kOffStatus + align256(sizeof(DevStatus));
constexpr size_t kOffRec = kOffCanvas + align256(sizeof(CanvasDesc));
constexpr size_t kOffRect = kOffRec + align256(sizeof(PrimRec) * kMaxPrims);
constexpr size_t kOffHist = kOffRect + align256(sizeof(int4) * kMaxPrims);
constexpr size_t kOffTileOff = kOffHist + align256(sizeof(int32_t) * kMaxChunks * kMaxTiles);
constexpr size_t kOffList = kOffTileOff + align256(sizeof(int64_t) * (kMaxTiles + 1));
// texel plane: n_bmp (H_b+1) rows of atlas_plane_pitch(W_b) <= 4 W_b + 124 bytes, and
// n_bmp (H_b+1) <= cells / 3; plus room to align its base to kTexAlign
constexpr size_t kPlaneBytes = 4 * kMaxAtlasCells + 124 * (kMaxAtlasCells / 3 + 1) + kTexAlign;
constexpr size_t kOffPlane = kOffList + align256(sizeof(int32_t) * kMaxPairs);
constexpr size_t kOffSat = kOffPlane + align256(kPlaneBytes);
// per-bitmap non-zero boxes: n_bmp <= cells / 9 (H_b, W_b >= 2)
constexpr size_t kOffNzbox = kOffSat + align256(sizeof(int32_t) * kMaxAtlasCells);
constexpr size_t kScratchBytes = kOffNzbox + align256(sizeof(int4) * (kMaxAtlasCells / 9));  // ~6.2 MB

// The scratch area: every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Texture objects over the scratch texel plane, one per atlas shape (W_b, plane rows)
// and device, created on first use and kept until the process exits (a launch still
// queued may read one).
struct TexEntry {
    int dev;
    int32_t Wb;
    int64_t rows;
    cudaTextureObject_t tex;
};
constexpr int kMaxTexEntries = 64;
TexEntry g_tex[kMaxTexEntries];
int g_n_tex = 0;

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Formats the message and stores it where dbmp_last_error() reads it.
int32_t fail_static(int32_t code, const char *fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return record_error(code, msg);
}

__global__ void k_static_canvas(CanvasDesc d, CanvasDesc *dst) { *dst = d; }

// Resolves the scratch array's device address for the current device (once).
int32_t scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_static(DBMP_ERR_INVALID_ARG, "device %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail_static(DBMP_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    // The binning kernels need at most 8 B x 1024 tiles of dynamic shared memory
    // here, under the default limit, so only the compositors' set-up (once per
    // device, inside init_render_kernels) is needed.
    e = init_render_kernels();
    if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "kernel set-up: %s", cudaGetErrorString(e));
    *out = g_scratch_ptr[dev];
    return DBMP_OK;
}

// The texture object for an n_bmp x H_b x W_b atlas in the scratch plane at `plane`.
int32_t scratch_texture(float *plane, int32_t n_bmp, int32_t Hb, int32_t Wb, cudaTextureObject_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    const int64_t rows = (int64_t)n_bmp * (Hb + 1);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    for (int i = 0; i < g_n_tex; ++i)
        if (g_tex[i].dev == dev && g_tex[i].Wb == Wb && g_tex[i].rows == rows) {
            *out = g_tex[i].tex;
            return DBMP_OK;
        }
    if (g_n_tex == kMaxTexEntries)
        return fail_static(DBMP_ERR_INVALID_ARG, "more than %d distinct atlas shapes", kMaxTexEntries);
    cudaTextureObject_t t = 0;
    e = atlas_texture_create(plane, atlas_plane_pitch(Wb), n_bmp, Hb, Wb, &t);
    if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "texture object: %s", cudaGetErrorString(e));
    g_tex[g_n_tex++] = TexEntry{dev, Wb, rows, t};
    *out = t;
    return DBMP_OK;
}

}  // namespace

extern "C" int32_t dbmp_render_fwd_static(int32_t H, int32_t W, const float *params_dev,
                                          const int32_t *bitmap_id_dev, int32_t N, const float *texels_dev,
                                          int32_t n_bmp, int32_t H_b, int32_t W_b, float alpha_max,
                                          const DbmpBackground *bg, float T_stop, float *image_dev,
                                          float *T_final_dev, int32_t *n_last_dev, dbmp_stream_t stream,
                                          DbmpDeviceStatus *status_out) {
    // ---- host-side checks: nothing is queued when one fails ----
    if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide)
        return fail_static(DBMP_ERR_INVALID_ARG, "canvas %dx%d outside 1..%d", H, W, kMaxSide);
    if (N < 0 || N > kMaxPrims)
        return fail_static(DBMP_ERR_INVALID_ARG, "N = %d outside 0..%d", N, kMaxPrims);
    if (n_bmp < 1 || H_b < 2 || W_b < 2 || (int64_t)n_bmp * (H_b + 1) * (W_b + 1) > kMaxAtlasCells)
        return fail_static(DBMP_ERR_INVALID_ARG,
                           "atlas %d x %dx%d: needs n_bmp >= 1, H_b, W_b >= 2, n_bmp (H_b+1)(W_b+1) <= %lld",
                           n_bmp, H_b, W_b, (long long)kMaxAtlasCells);
    if (!texels_dev || !image_dev || !T_final_dev || !n_last_dev || (N > 0 && (!params_dev || !bitmap_id_dev)))
        return fail_static(DBMP_ERR_INVALID_ARG, "NULL argument");
    if (N > 0 && (((uintptr_t)params_dev) & 15))
        return fail_static(DBMP_ERR_INVALID_ARG, "params_dev must be 16-byte aligned");
    if (!(alpha_max > 0.0f && alpha_max <= 1.0f))
        return fail_static(DBMP_ERR_INVALID_ARG, "alpha_max must be in (0, 1]");
    if (!(T_stop >= 0.0f && T_stop < 1.0f)) return fail_static(DBMP_ERR_INVALID_ARG, "T_stop must be in [0, 1)");
    if (bg && bg->mode != DBMP_BG_NONE && bg->mode != DBMP_BG_CONST && bg->mode != DBMP_BG_BUFFER)
        return fail_static(DBMP_ERR_INVALID_ARG, "background mode %d unknown", bg->mode);
    if (bg && bg->mode == DBMP_BG_BUFFER && !bg->buf_dev)
        return fail_static(DBMP_ERR_INVALID_ARG, "background buffer is NULL");

    unsigned char *base = nullptr;
    if (int32_t r = scratch_for_current_device(&base)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    DevStatus *status = reinterpret_cast<DevStatus *>(base + kOffStatus);
    CanvasDesc *canvas = reinterpret_cast<CanvasDesc *>(base + kOffCanvas);

    // ---- one-canvas plan ----
    CanvasDesc d{};
    d.H = H;
    d.W = W;
    d.ntx = (W + kTile - 1) / kTile;
    d.nty = (H + kTile - 1) / kTile;
    d.tile_base = 0;
    d.prim_base = 0;
    d.N = N;
    d.chunk_base = 0;
    d.chunk_log2 = kChunkLog2;
    d.n_chunks = (N + (1 << kChunkLog2) - 1) >> kChunkLog2;
    d.slab_rows = bin_slab_rows(d.ntx, d.nty, kChunkLog2, d.n_chunks);
    d.n_slabs = (d.nty + d.slab_rows - 1) / d.slab_rows;
    d.pix_base = 0;
    d.hist_base = 0;

    float *plane = reinterpret_cast<float *>(((uintptr_t)(base + kOffPlane) + kTexAlign - 1) &
                                             ~(uintptr_t)(kTexAlign - 1));
    cudaTextureObject_t tex = 0;
    if (int32_t r = scratch_texture(plane, n_bmp, H_b, W_b, &tex)) return r;
    AtlasView atlas{tex, reinterpret_cast<const int32_t *>(base + kOffSat), n_bmp, H_b, W_b,
                    reinterpret_cast<const int4 *>(base + kOffNzbox)};

    // The previous call's contents are still in the array: the status block (error
    // code, counters, work queues) must start at zero; everything else read later is
    // fully rewritten below before it is read.
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) {
        k_static_canvas<<<1, 1, 0, st>>>(d, canvas);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_atlas_build(texels_dev, plane, (int64_t)(atlas_plane_pitch(W_b) / sizeof(float)),
                               reinterpret_cast<int32_t *>(base + kOffSat), reinterpret_cast<int4 *>(base + kOffNzbox),
                               n_bmp, H_b, W_b, st);
    if (e == cudaSuccess) {
        BinBuffers b{};
        b.rec = reinterpret_cast<PrimRec *>(base + kOffRec);
        b.rect = reinterpret_cast<int4 *>(base + kOffRect);
        b.hist = reinterpret_cast<int32_t *>(base + kOffHist);
        b.tile_off = reinterpret_cast<int64_t *>(base + kOffTileOff);
        b.list = reinterpret_cast<int32_t *>(base + kOffList);
        b.cap = kMaxPairs;
        b.tile_order = nullptr;
        b.status = status;
        b.canvas = canvas;
        b.n_canvas = 1;
        b.n_tiles = d.ntx * d.nty;
        b.n_chunks = d.n_chunks;
        b.N = N;
        b.max_tiles_per_canvas = d.ntx * d.nty;
        b.chunk_log2 = kChunkLog2;
        b.max_slabs = d.n_slabs;
        b.smem_count = (int32_t)bin_smem_bytes(d.ntx, d.slab_rows, kChunkLog2, false);
        b.smem_scatter = (int32_t)bin_smem_bytes(d.ntx, d.slab_rows, kChunkLog2, true);
        e = launch_bin(b, params_dev, bitmap_id_dev, atlas, alpha_max, kTile, st);
    }
    if (e == cudaSuccess) {
        RenderArgs a{};
        a.rec = reinterpret_cast<const PrimRec *>(base + kOffRec);
        a.tile_off = reinterpret_cast<const int64_t *>(base + kOffTileOff);
        a.list = reinterpret_cast<const int32_t *>(base + kOffList);
        a.tile_order = nullptr;
        a.canvas = canvas;
        a.n_canvas = 1;
        a.n_tiles = d.ntx * d.nty;
        a.status = status;
        a.atlas = atlas;
        a.bg_mode = bg ? bg->mode : DBMP_BG_NONE;
        if (bg && bg->mode == DBMP_BG_CONST) {
            a.bg0 = bg->rgb[0];
            a.bg1 = bg->rgb[1];
            a.bg2 = bg->rgb[2];
        }
        a.bg_buf = bg ? bg->buf_dev : nullptr;
        a.T_stop = T_stop;
        a.n_prims = N;
        a.image = image_dev;
        a.T_final = T_final_dev;
        a.n_last = n_last_dev;
        e = launch_fwd(a, RenderCfg{kTile, 32, 2, 2}, st);
    }
    if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "launch: %s", cudaGetErrorString(e));

    if (status_out) {
        DevStatus s;
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(&s, status, sizeof s, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_static(DBMP_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
        status_out->code = s.code;
        status_out->n_degenerate = s.n_degenerate;
        status_out->pairs_required = s.pairs_required;
        status_out->pairs_evaluated = s.pairs_eval_fwd;
        status_out->pairs_evaluated_bwd = 0;
        status_out->pairs_contributing = s.pairs_contrib;
        status_out->warp_steps = s.warp_steps_fwd;
        status_out->warp_steps_bwd = 0;
        status_out->survivors = s.survivors_fwd;
        status_out->survivors_bwd = 0;
        status_out->bad_kind = s.bad_kind;
        status_out->bad_pad = 0;
        status_out->bad_index = s.bad_index;
        if (s.code == DBMP_ERR_CAPACITY)
            return fail_static(DBMP_ERR_CAPACITY, "tile lists need %lld entries, the static scratch holds %lld",
                               (long long)s.pairs_required, (long long)kMaxPairs);
    }
    return DBMP_OK;
}
