// Internal declarations of libdbmp (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/dbmp.h"
#include "compositor.cuh"

namespace dbmp {
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each).
// ---------------------------------------------------------------------------
struct BinBuffers {
    PrimRec *rec;
    int4 *rect;               // per primitive: tx0, ty0, tx1, ty1 (canvas-local); empty: tx1 < tx0
    int32_t *hist;            // chunk x tile counts, then bases
    int64_t *tile_off;        // [n_tiles + 1]
    int32_t *list;            // [cap] primitive indices (global)
    int64_t cap;
    int32_t *tile_order;      // [n_tiles] processing order (longest lists first)
    DevStatus *status;
    const CanvasDesc *canvas; // [n_canvas]
    int32_t n_canvas;
    int32_t n_tiles;          // total tiles
    int32_t n_chunks;         // total chunks
    int32_t N;                // total primitives
    int32_t max_tiles_per_canvas;
    int32_t chunk_log2;       // primitives per binning chunk (all canvases), 7..10
    int32_t max_slabs;        // largest n_slabs over the canvases
    int32_t smem_count;       // dynamic shared memory of k_count / k_scatter (largest
    int32_t smem_scatter;     //   over the canvases)
};

// Stores a one-line message for dbmp_last_error() on this thread; returns code.
int32_t record_error(int32_t code, const char *msg);

// One-time kernel set-up (shared-memory opt-in, occupancy), called at workspace
// creation so that later launches can be captured in CUDA graphs.
cudaError_t init_bin_kernels(int32_t max_tiles_per_canvas);
// Scaling statistics of the last binning (bin.cu); st holds kBinStatsWords counters.
constexpr int32_t kBinStatsWords = 104;
cudaError_t launch_bin_stats(const BinBuffers &b, const float *params, int32_t Hb, int32_t Wb,
                             unsigned long long *st, cudaStream_t s);
// Gaussian blur of the bitmaps (blur.cu): normalised 1-D taps of radius r.
constexpr int32_t kMaxBlurRadius = 15;
struct BlurTaps {
    int32_t r;
    float w[2 * kMaxBlurRadius + 1];
};
BlurTaps blur_taps(double sigma);
cudaError_t launch_blur(const float *in, float *out, int32_t n_bmp, int32_t Hb, int32_t Wb, const BlurTaps &taps,
                        cudaStream_t st);
// Structure-aware initialisation (init.cu).
size_t structure_init_scratch(int64_t n_pixels);
cudaError_t launch_structure_init(const float *image, const float *mask, int32_t H, int32_t W, int32_t N,
                                  const double *u_pos, const double *u_theta, const double *n_color, double s_min,
                                  double s_max, double sigma_c, double nu, void *scratch, float *params,
                                  double *nlv_out, double reinit_thr, float *adam_m, float *adam_v,
                                  int32_t *count, cudaStream_t st);
// I_alpha = 1 - T_final (optim.cu).
cudaError_t launch_alpha_from_T(const float *T_final, float *alpha, int64_t n, cudaStream_t st);
// Spatially constrained loss, Eq. 9 (optim.cu).
cudaError_t launch_alpha_loss(const float *image, const float *T_final, const float *target,
                              const float *target_alpha, int64_t n_pix, float lam, float *dL_dimage,
                              float *dL_dalpha, double *loss, cudaStream_t st);
// Binning slab geometry.  One CTA of min(2^chunk_log2, 1024) threads takes a chunk
// in passes of one primitive per thread and covers a slab of tile rows.  Shared
// memory: one mask word per (tile column, warp) and per (slab row, warp), plus a
// running count per slab tile (scatter only).
constexpr int32_t kBinSmemCap = 96 * 1024;
constexpr int32_t kBinTargetCtas = 8 * 152;   // enough CTAs to fill every SM several times
constexpr int64_t kBinPairsLarge = (int64_t)1 << 19;   // (chunk, tile) pairs above which chunks hold 1024
inline int32_t bin_threads(int32_t chunk_log2) { return chunk_log2 >= 10 ? 1024 : (1 << chunk_log2); }
inline int64_t bin_smem_bytes(int32_t ntx, int32_t rows, int32_t chunk_log2, bool scatter) {
    const int64_t nw = bin_threads(chunk_log2) / 32;
    return ((int64_t)ntx + rows) * nw * 4 + (scatter ? 4 * (int64_t)rows * ntx : 0);
}
inline bool bin_slab_ok(int32_t ntx, int32_t chunk_log2) {
    return bin_smem_bytes(ntx, 1, chunk_log2, true) <= kBinSmemCap;
}
// Rows per slab: enough slabs that all chunks x slabs reach kBinTargetCtas, within
// the shared-memory cap.
inline int32_t bin_slab_rows(int32_t ntx, int32_t nty, int32_t chunk_log2, int64_t total_chunks) {
    const int64_t want = (kBinTargetCtas + total_chunks - 1) / (total_chunks > 0 ? total_chunks : 1);
    int32_t rows = want >= nty ? 1 : (int32_t)((nty + want - 1) / want);
    while (rows > 1 && bin_smem_bytes(ntx, rows, chunk_log2, true) > kBinSmemCap) --rows;
    return rows;
}
cudaError_t init_render_kernels();

// With reset_fwd the binning also resets the status block's forward group (the tile
// scan does), so that a forward can follow it as a programmatic dependent.
cudaError_t launch_bin(const BinBuffers &b, const float *params, const int32_t *bitmap_id,
                       const AtlasView &atlas, float alpha_max, int32_t tile, cudaStream_t st,
                       bool reset_fwd = false);


bool render_cfg_supported(const RenderCfg &cfg);
cudaError_t launch_fwd(const RenderArgs &a, const RenderCfg &cfg, cudaStream_t st, bool pdl = false);
// Work items (regions) of a forward (bwd false) or backward pass over n_tiles tiles.
int32_t render_items(const RenderCfg &cfg, int32_t n_tiles, bool bwd);
// Region order by decreasing forward cost (counting sort of the forward's buckets).
// With reset_bwd it also resets the backward's status group (see launch_bwd).
cudaError_t launch_item_order(const int32_t *cost, int32_t *hist, int32_t *next_hist, int32_t *order,
                              int32_t n_items, DevStatus *reset_bwd, cudaStream_t st);
cudaError_t launch_bwd(const RenderArgs &a, const RenderCfg &cfg, cudaStream_t st, bool pdl = false);
// dparams += chain rule of the raw sums graw, which are zeroed after reading (graw is
// zero before every backward: zeroed at workspace creation, left zero by this kernel).
cudaError_t launch_grad_finalize(const float *params, const PrimRec *rec, float *graw,
                                 float *dparams, int32_t N, float kw, float kv, cudaStream_t st);
// Streaming multiprocessors of the current device (queried once per device).
int sm_count();
// Texel plane (row pitch `pitch` floats) and summed-area tables of an atlas from
// its dense texels [n_bmp][H_b][W_b].
cudaError_t launch_atlas_build(const float *texels, float *plane, int64_t pitch, int32_t *sat, int4 *nzbox, int32_t n_bmp,
                               int32_t Hb, int32_t Wb, cudaStream_t st);
// Row pitch (bytes) of an atlas texel plane, and the texture object over it (the
// plane's base must be kTexAlign-aligned).
constexpr size_t kTexAlign = 512;
size_t atlas_plane_pitch(int32_t Wb);
cudaError_t atlas_texture_create(float *plane, size_t pitch_bytes, int32_t n_bmp, int32_t Hb, int32_t Wb,
                                 cudaTextureObject_t *out);
// Whether an n_bmp x H_b x W_b atlas fits the device's pitch-linear texture limits.
cudaError_t atlas_texture_fits(int32_t n_bmp, int32_t Hb, int32_t Wb, bool *fits);
cudaError_t launch_mse_grad(const float *image, const float *target, int64_t n, float *dL,
                            double *loss, cudaStream_t st);
cudaError_t launch_adam(float *p, float *g, float *m, float *v, int32_t N, int32_t *step,
                        const DbmpAdamConfig &cfg, cudaStream_t st);

// ---------------------------------------------------------------------------
// Tensor-core GEMM (gemm_tc.cu): C[m][n] (op)= sum_k A[m][k] B[n][k], BF16 in, FP32
// accumulation.  A, B are raw bf16 bits, K-contiguous, 16-byte aligned rows
// (lda, ldb multiples of 8), K a multiple of 64.
// ---------------------------------------------------------------------------
enum GemmMode { GEMM_STORE_F32 = 0, GEMM_ATOMIC_F32 = 1, GEMM_BIAS_RELU_BF16 = 2, GEMM_BIAS_F32 = 3, GEMM_STORE_BF16 = 4 };
// Operand layout flags of dbmp_gemm_bf16's mode: A (B) given MN-major, i.e. as the
// K x M (K x N) matrix with M (N) contiguous.
constexpr int32_t GEMM_A_MN = 16, GEMM_B_MN = 32;
// dbmp_gemm_bf16 mode flag of the timeout test (see GemmArgs::stall)
constexpr int32_t GEMM_TEST_STALL = 64;

struct GemmArgs {
    const uint16_t *A;
    const uint16_t *B;
    int32_t M, N, K, lda, ldb, ldc;
    int32_t mode;       // GemmMode (the epilogue)
    int32_t a_mn, b_mn; // operands MN-major (A: K x M, B: K x N, lda / ldb their row strides)
    float *Cf;          // GEMM_STORE_F32, GEMM_ATOMIC_F32, GEMM_BIAS_F32
    uint16_t *Cb;       // GEMM_BIAS_RELU_BF16, GEMM_STORE_BF16
    const float *bias;  // [N] for the bias modes
    int32_t *status;    // set to DBMP_ERR_TIMEOUT if a bounded wait gives up (may be null)
    int32_t tma_c;      // set by the launcher: C written by TMA tensor stores (aligned C)
    int32_t split;      // set by the launcher: K splits (partial tiles added into C)
    int32_t stall;      // test hook: the producer issues no copies, so the MMA and
                        // epilogue waits run out and status becomes DBMP_ERR_TIMEOUT
    // Implicit convolution (the proposal network's 4x4 / stride-2 / pad-1 layers).  A
    // conv operand is read with 4-D tensor copies of an activation tensor instead of
    // 2-D copies of a matrix; pixel rows m = (b, oy, ox) of the Ho x Ho output grid
    // (ox fastest), one K step = one tap (dy, dx) of a 2 x 2 stencil x 64 channels:
    //   CONV_BLOCKED  source Xb [nb][Ho+1][Ho+1][chan] in the blocked layout (below);
    //                 element (m, tap*chan + q) = Xb[b][oy+dy][ox+dx][q].  As A (K-major)
    //                 of the forward; as B (MN-major, K = pixels) of the weight gradient.
    //   CONV_DGRAD    source dZ [nb][Ho][Ho][chan] (NHWC); parity class g = (sy, sx) of
    //                 the group: element (m, tap*chan + q) = dZ[b][oy+1-sy-dy][ox+1-sx-dx][q]
    //                 (zero outside).  As A of the input gradient.
    int32_t a_conv = 0, b_conv = 0;   // ConvKind of the operand (CONV_NONE: a plain matrix)
    int32_t conv_chan = 0;            // channels of the source tensor (multiple of 64)
    int32_t conv_side = 0;            // Ho, a power of two >= 8
    int32_t conv_batch = 0;           // images in the source tensor (>= 2: a box may span two)
    int32_t groups = 1;               // independent products: tile groups, B rows N apart
    // Epilogue row placement (per-lane stores; the TMA-store path is plain only):
    //   OUT_BLOCKED  row m = (b, y, x) of an S x S grid goes to the blocked layout of the
    //                next layer's input: [nb][S/2+1][S/2+1][4N], element
    //                ((b, (y+1)/2, (x+1)/2), ((y+1)%2 * 2 + (x+1)%2) * N + n);
    //   OUT_DGRAD    row m = (b, i, j) of group g = (sy, sx) is pixel (2i+1-sy, 2j+1-sx) of
    //                the NHWC [nb][2S][2S][N] output; with `mask` (the blocked input of the
    //                layer), a value whose input element is not > 0 is written as 0.
    int32_t out_kind = 0;
    int32_t out_side = 0;             // S
    const uint16_t *mask = nullptr;
    // Column placement of a weight gradient computed in the blocked tap order: column
    // n = tap*4C + (sy*2 + sx)*C + c is written at ((2dy + sy)*4 + 2dx + sx)*C + c
    // (0: columns in place).
    int32_t col_remap = 0;            // C
};
// CONV_PAIRS (the first conv, 4 channels): source = the padded input [nb][2Ho][2Ho+2][4]
// read as pixel pairs, one 16-byte K chunk (taps kx = 2p, 2p+1 of tap row ky) per copy,
// unswizzled; K = 64 as A (forward), N = 64 as B (weight gradient, MN-major).
enum ConvKind { CONV_NONE = 0, CONV_BLOCKED = 1, CONV_DGRAD = 2, CONV_PAIRS = 3 };
enum OutKind { OUT_PLAIN = 0, OUT_BLOCKED = 1, OUT_DGRAD = 2 };

cudaError_t init_gemm_kernels();
cudaError_t launch_gemm(const GemmArgs &g, int split_k, cudaStream_t st);

// ---------------------------------------------------------------------------
// Proposal network (cnn.cu)
// ---------------------------------------------------------------------------
struct CnnBuffers {
    int32_t max_batch;
    int32_t nb;                    // images the activation buffers hold (max_batch, at least 2)
    float *theta, *grad, *m, *v;   // fp32 master parameters, gradient, Adam moments
    uint16_t *wbf;                 // bf16 copies of the weights, K in (ky, kx, c) order
    uint16_t *wf, *wd;             // convs 2-5: forward weights in blocked tap order, and the
                                   // input-gradient weights per parity class (at wbf's offsets)
    uint16_t *X[6];                // activations: X[0] the input (NHWC, 4 channels, rows padded
                                   // by one pixel on each side), X[1..4] in the blocked
                                   // layout, X[5] NHWC
    float *O, *dO, *dx;            // head outputs, their gradient, the head's input gradient
    uint16_t *dz, *dzp;            // conv output gradients (two buffers)
    int32_t *status;
};

int64_t cnn_num_params();
size_t cnn_bytes(int32_t max_batch);
cudaError_t cnn_alloc(CnnBuffers &c, int32_t max_batch);
void cnn_free(CnnBuffers &c);
cudaError_t cnn_sync_weights(CnnBuffers &c, cudaStream_t st);
cudaError_t cnn_forward(CnnBuffers &c, const float *images, int32_t B, cudaStream_t st);
cudaError_t cnn_decode(CnnBuffers &c, int32_t B, float *params, cudaStream_t st);
// Activations of the last forward (layer 0 input, 1-5 conv outputs as float32, 6 head
// outputs) copied to the host; count -1 for a bad layer or batch.
int64_t cnn_activation_count(int32_t layer, int32_t B);
cudaError_t cnn_activation(const CnnBuffers &c, int32_t layer, int32_t B, float *host);
cudaError_t cnn_backward(CnnBuffers &c, const float *target_params, int32_t B, double *loss, cudaStream_t st);
cudaError_t cnn_adam(CnnBuffers &c, float lr, float b1, float b2, float eps, int32_t t, cudaStream_t st);

}  // namespace dbmp
