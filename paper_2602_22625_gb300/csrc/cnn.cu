// The learned proposal network: a small CNN that maps a 256 x 256 target image to
// initial parameters of 512 primitives, refined afterwards by the plain gradient
// optimisation.  (The paper leaves learned initialisation to future work, Sec. S5,
// and shows that initialisation matters, Sec. 3.2.2.)
//
//   input   B x 256 x 256 x 4 bf16 (NHWC; channels 0-2 = 2 (I - 0.5), 3 = 0), rows padded
//           by one zero pixel on each side
//   conv1-5 4x4 / stride 2 / pad 1, bias, ReLU: 4 -> 32 -> 64 -> 128 -> 256 -> 256
//   head    1x1 conv 256 -> 64 on the 8 x 8 map: 8 slots x 8 outputs per cell
//
// Every product is the tcgen05 GEMM of gemm_tc.cu (BF16 operands, FP32 accumulation),
// and every convolution is an implicit GEMM: no im2col matrix is written.  conv1
// (K = 16 taps x 4 channels = 64) reads its input as 16-byte pixel pairs: for output
// pixel ox, taps kx = 2p, 2p+1 of tap row ky are padded pixels 2(ox+p), 2(ox+p)+1, so
// one tensor copy of 128 consecutive pairs is one 16-byte K chunk of 128 output rows
// (the tensor cores' unswizzled layout), eight copies one K step.  conv2-5 are implicit
// GEMMs over activations kept in a blocked (space-to-depth) layout:
//
//   Xb[b][i][j][(sy*2 + sx)*C + c] = X[b][2i+sy-1][2j+sx-1][c]  (0 outside),
//   i, j in [0, H/2], sy, sx in {0, 1}
//
// Tap (ky, kx) = (2dy + sy, 2dx + sx) of output (oy, ox) reads X[2oy-1+ky][2ox-1+kx] =
// block (oy+dy, ox+dx), sub-pixel (sy, sx): the 4x4 / stride-2 conv is a 2x2 / stride-1
// conv over the blocks with 4C channels, so one 64-wide K step is one block tap x 64
// contiguous channels, read by a 4-D tensor copy (no im2col matrix in HBM; the four
// reads of each block come from L2).  The previous layer's epilogue writes its output
// straight into this layout (the padding entries stay zero from allocation).
//   forward  X_l = relu(conv(X_{l-1}) + b_l)       (A = blocked X_{l-1}, B = W_l in the
//                                                    blocked tap order; bias + ReLU fused)
//   wgrad    dW_l = dZ_l^T conv-rows(X_{l-1})       (dZ MN-major, blocked X read MN-major,
//                                                    split-K; columns written back in the
//                                                    (ky, kx, c) order)
//   dgrad    for each parity class (sy, sx): the input pixels (2i+1-sy, 2j+1-sx) get
//            sum over (dy, dx, co) of dZ[i+1-sy-dy][j+1-sx-dx][co] W[co][2dy+sy][2dx+sx][c],
//            four GEMMs of K = 4 Co in one launch; the epilogue applies the mask
//            X_{l-1} > 0 and writes dZ_{l-1} (NHWC, bf16) in place: no column matrix,
//            no col2im.
// Weights are FP32 masters with BF16 copies (and the two rearranged copies above);
// Adam updates the masters.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

__device__ __forceinline__ uint16_t f2bf(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// The input image as the first layer's 4 channels (NHWC bf16): 2 (I - 0.5), and a zero
// fourth channel, in rows of 258 pixels with one zero pixel on each side (written once,
// at allocation), so that the first conv reads its taps as 16-byte pixel pairs.
__global__ void k_pack_input(const float *__restrict__ img, int32_t B, uint16_t *__restrict__ X0) {
    const int64_t n = (int64_t)B * 65536;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i >> 16, pix = i & 65535;
        const float *I = img + b * 3 * 65536 + pix;
        __align__(8) uint16_t h[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c] = f2bf(2.0f * (I[c * 65536] - 0.5f));
        h[3] = 0;
        const int64_t y = pix >> 8, x = pix & 255;
        reinterpret_cast<uint2 *>(X0)[(b * 256 + y) * 258 + x + 1] = *reinterpret_cast<const uint2 *>(h);
    }
}

// The network's sides and channel counts are powers of two; the index arithmetic
// below uses their log2 (shifts and masks instead of 64-bit divisions).

// Rearranged bf16 weights of convs 2-5 (layer table t), from the (ky, kx, c) copies:
//   wf[co][k'],            k'  = (dy*2 + dx)*4C + (sy*2 + sx)*C + c   (forward, blocked taps)
//   wd[cls*C + c][k''],    k'' = (dy*2 + dx)*Co + co, cls = sy*2 + sx (input gradient)
// both = W[co][(2dy+sy)*4 + 2dx+sx][c].
struct ConvWeightTable {
    int64_t w_off[4], start[5];
    int32_t lc[4], lco[4];   // log2 C, log2 Co
};
__global__ void k_conv_weights(const uint16_t *__restrict__ wbf, ConvWeightTable t, uint16_t *__restrict__ wf,
                               uint16_t *__restrict__ wd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.start[4];
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (i >= t.start[1]) + (i >= t.start[2]) + (i >= t.start[3]);
        const int64_t e = i - t.start[l];
        const int lc = t.lc[l], lco = t.lco[l];
        const int C = 1 << lc;
        const uint16_t *W = wbf + t.w_off[l];
        // forward copy: e = co * 16C + k'
        {
            const int64_t co = e >> (lc + 4);
            const int kp = (int)(e & ((16 << lc) - 1));
            const int tap = kp >> (lc + 2), s = (kp >> lc) & 3, c = kp & (C - 1);
            const int ky = 2 * (tap >> 1) + (s >> 1), kx = 2 * (tap & 1) + (s & 1);
            wf[t.w_off[l] + e] = W[(co << (lc + 4)) + ((ky * 4 + kx) << lc) + c];
        }
        // input-gradient copy: e = (cls * C + c) * 4Co + k''
        {
            const int64_t row = e >> (lco + 2);
            const int kpp = (int)(e & ((4 << lco) - 1));
            const int cls = (int)(row >> lc), c = (int)(row & (C - 1));
            const int tap = kpp >> lco, co = kpp & ((1 << lco) - 1);
            const int ky = 2 * (tap >> 1) + (cls >> 1), kx = 2 * (tap & 1) + (cls & 1);
            wd[t.w_off[l] + e] = W[((int64_t)co << (lc + 4)) + ((ky * 4 + kx) << lc) + c];
        }
    }
}

// out[n] += sum_m in[m][n] (in: bf16 or fp32; N a multiple of VEC = 16 / sizeof(T), at
// most 256 VEC); out must be zeroed by the caller.  Each thread
// reads 16 bytes (VEC consecutive columns) of a row, so a warp reads whole rows
// contiguously; the block's 256 threads cover N / VEC column groups x R rows per step,
// accumulate in registers over a grid-stride loop on rows, and reduce over their R row
// slots in shared memory before one atomic per column.
template <typename T>
__global__ void __launch_bounds__(256) k_colsum(const T *__restrict__ in, int32_t M, int32_t N,
                                                float *__restrict__ out) {
    constexpr int VEC = 16 / sizeof(T);
    __shared__ float part[256][VEC + 1];
    const int G = N / VEC, R = 256 / G;          // column groups, row slots
    const int gi = threadIdx.x % G, ri = threadIdx.x / G;
    float acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = 0.0f;
    if (ri < R) {
        for (int64_t m = (int64_t)blockIdx.x * R + ri; m < M; m += (int64_t)gridDim.x * R) {
            const uint4 v = *reinterpret_cast<const uint4 *>(in + m * N + gi * VEC);
            if constexpr (sizeof(T) == 2) {
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[2 * k] += bf2f((uint16_t)(w[k] & 0xffffu));
                    acc[2 * k + 1] += bf2f((uint16_t)(w[k] >> 16));
                }
            } else {
                acc[0] += __uint_as_float(v.x);
                acc[1] += __uint_as_float(v.y);
                acc[2] += __uint_as_float(v.z);
                acc[3] += __uint_as_float(v.w);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) part[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += 256) {   // column c = group c / VEC, element c % VEC
        float sum = 0.0f;
        for (int r = 0; r < R; ++r) sum += part[r * G + c / VEC][c % VEC];
        atomicAdd(out + c, sum);
    }
}

// Blocks of k_colsum: about 4 per SM, each taking at least 16 steps of rows.
inline int colsum_blocks(int64_t M, int N, int elem_bytes) {
    const int R = 256 / (N / (16 / elem_bytes));
    const int64_t cap = (M + 16 * R - 1) / (16 * R);
    return (int)std::max<int64_t>(1, std::min<int64_t>(4 * 152, cap));
}

__global__ void k_mask_to_bf16(const float *__restrict__ dX, const uint16_t *__restrict__ X, int64_t n,
                               uint16_t *__restrict__ dZ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dZ[i] = bf2f(X[i]) > 0.0f ? f2bf(dX[i]) : (uint16_t)0;
}

__global__ void k_to_bf16(const float *__restrict__ in, int64_t n, uint16_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = f2bf(in[i]);
}

__device__ __forceinline__ float logit_clip(float p) {
    p = fminf(fmaxf(p, 0.02f), 0.98f);
    return logf(p / (1.0f - p));
}

// Anchored decoding of the head outputs: cell (cy, cx) = row m % 64 of scene m / 64,
// slot k = column / 8.  Loss over the raw outputs (see k_head_decode for the map).
__global__ void k_head_loss(const float *__restrict__ O, const float *__restrict__ tp, int32_t B,
                            float *__restrict__ dO, double *loss) {
    __shared__ double red[8];
    const int64_t n = (int64_t)B * 512 * 8;
    const double inv = 1.0 / ((double)B * 512.0 * 7.0);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i & 7);
        const int64_t bp = i >> 3;
        const int p = (int)(bp & 511);
        const int64_t b = bp >> 9;
        const int cell = p >> 3, k = p & 7;
        const int cy = cell >> 3, cx = cell & 7;
        const int64_t oi = (b * 64 + cell) * 64 + k * 8 + j;
        const float *q = tp + bp * 8;
        float t = 0.0f, w = 1.0f;
        if (j == 0) t = logit_clip((q[0] - (float)(cx * 32 + (k & 3) * 8)) / 8.0f);
        else if (j == 1) t = logit_clip((q[1] - (float)(cy * 32 + (k >> 2) * 16)) / 16.0f);
        else if (j == 2) t = logit_clip((q[2] - 6.0f) / 8.0f);
        else if (j == 3) w = 0.0f;
        else t = fminf(fmaxf(q[j], -6.0f), 6.0f);
        const float d = (O[oi] - t) * w;
        dO[oi] = (float)(2.0 * (double)d * inv);
        acc += (double)d * (double)d * inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s);
    }
}

// params[b][p] = (cx*32 + (k%4)*8 + 8 s(o0), cy*32 + (k/4)*16 + 16 s(o1), 6 + 8 s(o2), 0, o4, o5, o6, o7)
__global__ void k_head_decode(const float *__restrict__ O, int32_t B, float *__restrict__ params) {
    const int64_t n = (int64_t)B * 512;
    for (int64_t bp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; bp < n; bp += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(bp & 511);
        const int64_t b = bp >> 9;
        const int cell = p >> 3, k = p & 7;
        const int cy = cell >> 3, cx = cell & 7;
        const float *o = O + (b * 64 + cell) * 64 + k * 8;
        float *out = params + bp * 8;
        out[0] = (float)(cx * 32 + (k & 3) * 8) + 8.0f / (1.0f + expf(-o[0]));
        out[1] = (float)(cy * 32 + (k >> 2) * 16) + 16.0f / (1.0f + expf(-o[1]));
        out[2] = 6.0f + 8.0f / (1.0f + expf(-o[2]));
        out[3] = 0.0f;
        out[4] = o[4];
        out[5] = o[5];
        out[6] = o[6];
        out[7] = o[7];
    }
}

__global__ void k_adam_flat(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, int32_t t,
                            uint16_t *__restrict__ pbf) {
    const float bc1 = 1.0f - powf(b1, (float)t), bc2 = 1.0f - powf(b2, (float)t);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        pbf[i] = f2bf(pi);
    }
}

// log2 of a power of two
int ilog2(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

int grid1d(int64_t n, int threads = 256) {
    const int64_t g = (n + threads - 1) / threads;
    return (int)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

}  // namespace

// ---------------------------------------------------------------------------
// Layer table
// ---------------------------------------------------------------------------
struct CnnLayer {
    int cin, cout, k, hin;   // padded input channels, output channels, kernel, input side
    int64_t K, w_off, b_off;
};

static void layer_table(CnnLayer L[6], int64_t *n_params) {
    const int cin[6] = {4, 32, 64, 128, 256, 256}, cout[6] = {32, 64, 128, 256, 256, 64};
    const int ks[6] = {4, 4, 4, 4, 4, 1}, hin[6] = {256, 128, 64, 32, 16, 8};
    int64_t o = 0;
    for (int l = 0; l < 6; ++l) {
        L[l].cin = cin[l];
        L[l].cout = cout[l];
        L[l].k = ks[l];
        L[l].hin = hin[l];
        L[l].K = (int64_t)ks[l] * ks[l] * cin[l];
        L[l].w_off = o;
        o += L[l].K * cout[l];
        L[l].b_off = o;
        o += cout[l];
    }
    *n_params = o;
}

int64_t cnn_num_params() {
    CnnLayer L[6];
    int64_t n;
    layer_table(L, &n);
    return n;
}

// sizes in elements for a given max batch
struct CnnSizes {
    int64_t X[6], dx, dz;
};

// Images held by the buffers that 4-D tensor copies read: a box may span two images.
static int32_t held_images(int32_t B) { return B < 2 ? 2 : B; }

static CnnSizes cnn_sizes(int32_t B) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    const int64_t nb = held_images(B);
    CnnSizes s{};
    s.X[0] = nb * 256 * 258 * 4;   // rows padded by one pixel on each side
    for (int l = 1; l < 5; ++l) {   // blocked: (H/2 + 1)^2 blocks of 4C channels
        const int64_t hb = L[l].hin / 2 + 1;
        s.X[l] = nb * hb * hb * 4 * L[l].cin;
    }
    s.X[5] = nb * 64 * 256;
    s.dx = nb * 64 * 256;
    s.dz = nb * 64 * 64;
    for (int l = 0; l < 5; ++l) {
        const int64_t Ho = L[l].hin / 2;
        s.dz = std::max<int64_t>(s.dz, nb * Ho * Ho * L[l].cout);
    }
    return s;
}

size_t cnn_bytes(int32_t B) {
    const CnnSizes s = cnn_sizes(B);
    int64_t np = cnn_num_params();
    size_t b = 4 * sizeof(float) * np + 3 * sizeof(uint16_t) * np;
    for (int l = 0; l < 6; ++l) b += sizeof(uint16_t) * s.X[l];
    b += 2 * sizeof(float) * (size_t)B * 64 * 64 + sizeof(float) * s.dx;
    b += 2 * sizeof(uint16_t) * s.dz + sizeof(int32_t) * 4;
    return b;
}

cudaError_t cnn_alloc(CnnBuffers &c, int32_t B) {
    const CnnSizes s = cnn_sizes(B);
    const int64_t np = cnn_num_params();
    c = CnnBuffers{};
    c.max_batch = B;
    c.nb = held_images(B);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, n > 0 ? n : 16);
    };
    A((void **)&c.theta, sizeof(float) * np);
    A((void **)&c.grad, sizeof(float) * np);
    A((void **)&c.m, sizeof(float) * np);
    A((void **)&c.v, sizeof(float) * np);
    A((void **)&c.wbf, sizeof(uint16_t) * np);
    A((void **)&c.wf, sizeof(uint16_t) * np);
    A((void **)&c.wd, sizeof(uint16_t) * np);
    for (int l = 0; l < 6; ++l) A((void **)&c.X[l], sizeof(uint16_t) * s.X[l]);
    A((void **)&c.O, sizeof(float) * B * 64 * 64);
    A((void **)&c.dO, sizeof(float) * B * 64 * 64);
    A((void **)&c.dx, sizeof(float) * s.dx);
    A((void **)&c.dz, sizeof(uint16_t) * s.dz);
    A((void **)&c.dzp, sizeof(uint16_t) * s.dz);
    A((void **)&c.status, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(c.status, 0, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(c.m, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemset(c.v, 0, sizeof(float) * np);
    // the padding entries of the input and of the blocked activations (never written)
    // read as zeros; so do the images past the batch that a two-image box may touch
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) e = cudaMemset(c.X[l], 0, sizeof(uint16_t) * s.X[l]);
    if (e == cudaSuccess) e = cudaMemset(c.X[5], 0, sizeof(uint16_t) * s.X[5]);
    if (e == cudaSuccess) e = cudaMemset(c.dz, 0, sizeof(uint16_t) * s.dz);
    if (e == cudaSuccess) e = cudaMemset(c.dzp, 0, sizeof(uint16_t) * s.dz);
    if (e == cudaSuccess) e = init_gemm_kernels();
    return e;
}

void cnn_free(CnnBuffers &c) {
    void *ps[] = {c.theta, c.grad, c.m, c.v, c.wbf, c.wf, c.wd, c.X[0], c.X[1], c.X[2], c.X[3], c.X[4], c.X[5],
                  c.O, c.dO, c.dx, c.dz, c.dzp, c.status};
    for (void *p : ps)
        if (p) cudaFree(p);
    c = CnnBuffers{};
}

// The rearranged weight copies of convs 2-5 from the bf16 copies.
static cudaError_t conv_weights(CnnBuffers &c, cudaStream_t st) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    ConvWeightTable t{};
    t.start[0] = 0;
    for (int i = 0; i < 4; ++i) {
        const CnnLayer &l = L[i + 1];
        t.w_off[i] = l.w_off;
        t.lc[i] = ilog2(l.cin);
        t.lco[i] = ilog2(l.cout);
        t.start[i + 1] = t.start[i] + l.K * l.cout;
    }
    k_conv_weights<<<grid1d(t.start[4]), 256, 0, st>>>(c.wbf, t, c.wf, c.wd);
    return cudaGetLastError();
}

// After new master weights: bf16 copies for the products.
cudaError_t cnn_sync_weights(CnnBuffers &c, cudaStream_t st) {
    const int64_t np = cnn_num_params();
    k_to_bf16<<<grid1d(np), 256, 0, st>>>(c.theta, np, c.wbf);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : conv_weights(c, st);
}

// mode: a GemmMode, plus GEMM_A_MN / GEMM_B_MN when an operand is given MN-major.
static GemmArgs gemm_args(const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N, int K, int mode,
                          float *Cf, uint16_t *Cb, int ldc, const float *bias, int32_t *status) {
    GemmArgs g{A,    B,    M,  N,  K,   lda,  ldb,   ldc, mode & 15, (mode & GEMM_A_MN) != 0, (mode & GEMM_B_MN) != 0,
               Cf,   Cb,   bias, status};
    return g;
}
static cudaError_t gemm(const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N, int K, int mode,
                        float *Cf, uint16_t *Cb, int ldc, const float *bias, int split, int32_t *status,
                        cudaStream_t st) {
    return launch_gemm(gemm_args(A, lda, B, ldb, M, N, K, mode, Cf, Cb, ldc, bias, status), split, st);
}

// Forward of B images (fp32, 3 x 256 x 256 each, concatenated) into c.O.
cudaError_t cnn_forward(CnnBuffers &c, const float *images, int32_t B, cudaStream_t st) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    k_pack_input<<<grid1d((int64_t)B * 65536), 256, 0, st>>>(images, B, c.X[0]);
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
        const int Ho = L[l].hin / 2;
        const int M = B * Ho * Ho, Co = L[l].cout, K = (int)L[l].K;
        // conv1: weights in their (ky, kx, c) order, which the pair chunks follow
        GemmArgs g = gemm_args(c.X[l], 0, (l == 0 ? c.wbf : c.wf) + L[l].w_off, K, M, Co, K, GEMM_BIAS_RELU_BF16,
                               nullptr, c.X[l + 1], Co, c.theta + L[l].b_off, c.status);
        g.a_conv = l == 0 ? CONV_PAIRS : CONV_BLOCKED;
        g.conv_chan = l == 0 ? 0 : 4 * L[l].cin;
        g.conv_side = Ho;
        g.conv_batch = c.nb;
        if (l < 4) {   // the next conv's input, blocked
            g.out_kind = OUT_BLOCKED;
            g.out_side = Ho;
        }
        e = launch_gemm(g, 1, st);
    }
    if (e == cudaSuccess)
        e = gemm(c.X[5], 256, c.wbf + L[5].w_off, 256, B * 64, 64, 256, GEMM_BIAS_F32, c.O, nullptr, 64,
                 c.theta + L[5].b_off, 1, c.status, st);
    return e;
}

int64_t cnn_activation_count(int32_t layer, int32_t B) {
    if (layer < 0 || layer > 6 || B < 1) return -1;
    if (layer == 6) return (int64_t)B * 64 * 64;
    if (layer == 0) return (int64_t)B * 256 * 256 * 4;
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    const int64_t H = L[layer - 1].hin / 2;
    return (int64_t)B * H * H * L[layer - 1].cout;
}

cudaError_t cnn_activation(const CnnBuffers &c, int32_t layer, int32_t B, float *host) {
    const int64_t n = cnn_activation_count(layer, B);
    if (layer == 6) return cudaMemcpy(host, c.O, sizeof(float) * n, cudaMemcpyDeviceToHost);
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    const bool blocked = layer >= 1 && layer <= 4;
    const int64_t H = layer == 0 ? 256 : L[layer - 1].hin / 2, C = n / ((int64_t)B * H * H), hb = H / 2 + 1;
    const int64_t stored = blocked ? (int64_t)B * hb * hb * 4 * C : layer == 0 ? (int64_t)B * 256 * 258 * 4 : n;
    // bf16 bits are the upper half of the float32 they round to
    uint16_t *tmp = static_cast<uint16_t *>(malloc(sizeof(uint16_t) * (size_t)stored));
    if (!tmp) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMemcpy(tmp, c.X[layer], sizeof(uint16_t) * stored, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        for (int64_t i = 0; i < n; ++i) {
            int64_t src = i;
            const int64_t ch = i % C, p = i / C, x = p % H, y = (p / H) % H, b = p / (H * H);
            if (blocked)   // NHWC element (b, y, x, ch) from block ((y+1)/2, (x+1)/2)
                src = ((b * hb + (y + 1) / 2) * hb + (x + 1) / 2) * 4 * C + (((y + 1) & 1) * 2 + ((x + 1) & 1)) * C + ch;
            else if (layer == 0)   // rows padded by one pixel on each side
                src = ((b * 256 + y) * 258 + x + 1) * 4 + ch;
            const uint32_t u = (uint32_t)tmp[src] << 16;
            memcpy(host + i, &u, sizeof u);
        }
    }
    free(tmp);
    return e;
}

cudaError_t cnn_decode(CnnBuffers &c, int32_t B, float *params, cudaStream_t st) {
    k_head_decode<<<grid1d((int64_t)B * 512), 256, 0, st>>>(c.O, B, params);
    return cudaGetLastError();
}

static int split_for(int M, int N, int K) {
    const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
    int s = (2 * 152 + tiles - 1) / tiles;
    const int kt = K / 64;
    if (s > kt / 2) s = kt / 2 > 0 ? kt / 2 : 1;
    return s < 1 ? 1 : s;
}

// Loss and gradient w.r.t. all parameters into c.grad (overwritten).  Reads the
// activations that the forward of the same batch left in c.
cudaError_t cnn_backward(CnnBuffers &c, const float *target_params, int32_t B, double *loss, cudaStream_t st) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    cudaMemsetAsync(c.grad, 0, sizeof(float) * np, st);
    const int M6 = B * 64;
    k_head_loss<<<grid1d((int64_t)B * 4096), 256, 0, st>>>(c.O, target_params, B, c.dO, loss);
    k_to_bf16<<<grid1d((int64_t)M6 * 64), 256, 0, st>>>(c.dO, (int64_t)M6 * 64, c.dz);
    // head: wgrad (dZ^T X5: both operands read MN-major), bias, dgrad (dZ W: W read MN-major)
    cudaError_t e = gemm(c.dz, 64, c.X[5], 256, 64, 256, M6, GEMM_ATOMIC_F32 | GEMM_A_MN | GEMM_B_MN,
                         c.grad + L[5].w_off, nullptr, 256, nullptr, split_for(64, 256, M6), c.status, st);
    k_colsum<float><<<colsum_blocks(M6, 64, 4), 256, 0, st>>>(c.dO, M6, 64, c.grad + L[5].b_off);
    if (e == cudaSuccess)
        e = gemm(c.dz, 64, c.wbf + L[5].w_off, 256, M6, 256, 64, GEMM_STORE_F32 | GEMM_B_MN, c.dx, nullptr, 256,
                 nullptr, 1, c.status, st);
    k_mask_to_bf16<<<grid1d((int64_t)M6 * 256), 256, 0, st>>>(c.dx, c.X[5], (int64_t)M6 * 256, c.dz);
    for (int l = 4; l >= 0 && e == cudaSuccess; --l) {
        const int Ho = L[l].hin / 2, M = B * Ho * Ho;
        const int K = (int)L[l].K, Co = L[l].cout, C = L[l].cin;
        if (l == 0) {   // wgrad with B = the padded input's pixel pairs (MN-major)
            GemmArgs g = gemm_args(c.dz, Co, c.X[0], 0, Co, K, M, GEMM_ATOMIC_F32 | GEMM_A_MN | GEMM_B_MN,
                                   c.grad + L[l].w_off, nullptr, K, nullptr, c.status);
            g.b_conv = CONV_PAIRS;
            g.conv_side = Ho;
            g.conv_batch = c.nb;
            e = launch_gemm(g, split_for(Co, K, M), st);
        } else {        // wgrad with B = the blocked input, columns back in (ky, kx, c) order
            GemmArgs g = gemm_args(c.dz, Co, c.X[l], 0, Co, K, M, GEMM_ATOMIC_F32 | GEMM_A_MN | GEMM_B_MN,
                                   c.grad + L[l].w_off, nullptr, K, nullptr, c.status);
            g.b_conv = CONV_BLOCKED;
            g.conv_chan = 4 * C;
            g.conv_side = Ho;
            g.conv_batch = c.nb;
            g.col_remap = C;
            e = launch_gemm(g, split_for(Co, K, M), st);
        }
        k_colsum<uint16_t><<<colsum_blocks(M, Co, 2), 256, 0, st>>>(c.dz, M, Co, c.grad + L[l].b_off);
        if (l == 0 || e != cudaSuccess) break;
        // dgrad: four parity classes, masked by the layer's input, into dZ_{l-1} (NHWC)
        GemmArgs g = gemm_args(c.dz, 0, c.wd + L[l].w_off, 4 * Co, M, C, 4 * Co, GEMM_STORE_BF16, nullptr, c.dzp,
                               C, nullptr, c.status);
        g.a_conv = CONV_DGRAD;
        g.conv_chan = Co;
        g.conv_side = Ho;
        g.conv_batch = c.nb;
        g.groups = 4;
        g.out_kind = OUT_DGRAD;
        g.out_side = Ho;
        g.mask = c.X[l];
        e = launch_gemm(g, 1, st);
        uint16_t *t = c.dz;
        c.dz = c.dzp;
        c.dzp = t;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t cnn_adam(CnnBuffers &c, float lr, float b1, float b2, float eps, int32_t t, cudaStream_t st) {
    const int64_t np = cnn_num_params();
    k_adam_flat<<<grid1d(np), 256, 0, st>>>(c.theta, c.grad, c.m, c.v, np, lr, b1, b2, eps, t, c.wbf);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : conv_weights(c, st);
}

}  // namespace dbmp
