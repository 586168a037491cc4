// The learned proposal network: a small CNN that maps a 256 x 256 target image to
// initial parameters of 512 primitives, refined afterwards by the plain gradient
// optimisation.  (The paper leaves learned initialisation to future work, Sec. S5,
// and shows that initialisation matters, Sec. 3.2.2.)
//
//   input   B x 256 x 256 x 8 bf16 (NHWC; channels 0-2 = 2 (I - 0.5), 3-7 = 0)
//   conv1-5 4x4 / stride 2 / pad 1, bias, ReLU: 8 -> 32 -> 64 -> 128 -> 256 -> 256
//   head    1x1 conv 256 -> 64 on the 8 x 8 map: 8 slots x 8 outputs per cell
//
// Every product is the tcgen05 GEMM of gemm_tc.cu (BF16 operands, FP32 accumulation):
//   forward  X_l = relu(im2col(X_{l-1}) W_l^T + b_l)   (bias + ReLU fused, bf16 out)
//   wgrad    dW_l = dZ_l^T im2col(X_{l-1})               (both operands read MN-major,
//                                                          split-K with fp32 atomics)
//   dgrad    dX_{l-1} = col2im(dZ_l W_l) masked by X_{l-1} > 0   (W_l read MN-major)
// Weights are FP32 masters with BF16 copies; Adam updates the masters.
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
// fourth channel (the first layer's K = 16 taps x 4 channels = 64, one GEMM K step).
__global__ void k_pack_input(const float *__restrict__ img, int32_t B, uint16_t *__restrict__ X0) {
    const int64_t n = (int64_t)B * 65536;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i >> 16, pix = i & 65535;
        const float *I = img + b * 3 * 65536 + pix;
        __align__(8) uint16_t h[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c] = f2bf(2.0f * (I[c * 65536] - 0.5f));
        h[3] = 0;
        reinterpret_cast<uint2 *>(X0)[i] = *reinterpret_cast<const uint2 *>(h);
    }
}

// im2col of the 4-channel input: col[m][(ky*4 + kx)*4 + c] = X[b][2oy-1+ky][2ox-1+kx][c]
// (0 outside), m = (b, oy, ox), H = W = 2^lh; one 8-byte chunk (4 channels) per thread.
__global__ void k_im2col4(const uint16_t *__restrict__ X, int32_t B, int32_t lh, uint16_t *__restrict__ col) {
    const int lo = lh - 1;
    const int H = 1 << lh;
    const int64_t n = (int64_t)B << (2 * lo + 4);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(i & 15);
        const int64_t m = i >> 4;
        const int ox = (int)(m & ((1 << lo) - 1)), oy = (int)((m >> lo) & ((1 << lo) - 1));
        const int64_t b = m >> (2 * lo);
        const int y = 2 * oy - 1 + (kk >> 2), x = 2 * ox - 1 + (kk & 3);
        uint2 v = make_uint2(0, 0);
        if (y >= 0 && y < H && x >= 0 && x < H) v = reinterpret_cast<const uint2 *>(X)[(((b << lh) + y) << lh) + x];
        reinterpret_cast<uint2 *>(col)[i] = v;
    }
}

// The network's sides and channel counts are powers of two; the index arithmetic
// below uses their log2 (shifts and masks instead of 64-bit divisions).
//
// col[m][(ky*4 + kx)*C + c] = X[b][2oy-1+ky][2ox-1+kx][c] (0 outside), m = (b, oy, ox),
// H = W = 2^lh, C = 8 * 2^lc8; one 16-byte chunk (8 channels) per thread.
__global__ void k_im2col(const uint16_t *__restrict__ X, int32_t B, int32_t lh, int32_t lc8,
                         uint16_t *__restrict__ col) {
    const int lo = lh - 1;   // log2 of the output side
    const int H = 1 << lh, C8 = 1 << lc8;
    const int64_t n = ((int64_t)B << (2 * lo + 4 + lc8));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(i & (C8 - 1));
        const int kk = (int)((i >> lc8) & 15);
        const int64_t m = i >> (lc8 + 4);
        const int ox = (int)(m & ((1 << lo) - 1)), oy = (int)((m >> lo) & ((1 << lo) - 1));
        const int64_t b = m >> (2 * lo);
        const int y = 2 * oy - 1 + (kk >> 2), x = 2 * ox - 1 + (kk & 3);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (y >= 0 && y < H && x >= 0 && x < H)
            v = reinterpret_cast<const uint4 *>(X + ((((b << lh) + y) << lh) + x) * (8 << lc8))[c8];
        reinterpret_cast<uint4 *>(col)[i] = v;
    }
}

// dX[b][y][x][c] = sum over (ky, kx) with 2oy-1+ky = y, 2ox-1+kx = x of
// dcol[(b,oy,ox)][(ky*4+kx)*C + c] (bf16, summed in fp32); then dZ = X > 0 ? bf16(dX) : 0.
// H = W = 2^lh, C = 2^lc (>= 4); four channels per thread (8-byte loads of dcol).
__global__ void k_col2im_mask(const uint16_t *__restrict__ dcol, const uint16_t *__restrict__ X, int32_t B,
                              int32_t lh, int32_t lc, uint16_t *__restrict__ dZ) {
    const int lo = lh - 1, Ho = 1 << lo, C = 1 << lc;
    const int64_t n4 = ((int64_t)B << (2 * lh + lc)) >> 2;
    for (int64_t i4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i4 < n4;
         i4 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i4 << 2;
        const int c = (int)(i & (C - 1));
        const int64_t p = i >> lc;
        const int x = (int)(p & ((1 << lh) - 1)), y = (int)((p >> lh) & ((1 << lh) - 1));
        const int64_t b = p >> (2 * lh);
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        // ky = y + 1 - 2 oy in [0, 4): two candidates of matching parity
        for (int ky = (y + 1) & 1; ky < 4; ky += 2) {
            const int oy = (y + 1 - ky) >> 1;
            if (oy < 0 || oy >= Ho) continue;
            for (int kx = (x + 1) & 1; kx < 4; kx += 2) {
                const int ox = (x + 1 - kx) >> 1;
                if (ox < 0 || ox >= Ho) continue;
                const uint2 d = *reinterpret_cast<const uint2 *>(
                    dcol + ((((b << lo) + oy) << lo) + ox) * ((int64_t)16 << lc) + ((ky * 4 + kx) << lc) + c);
                acc.x += bf2f((uint16_t)(d.x & 0xffffu));
                acc.y += bf2f((uint16_t)(d.x >> 16));
                acc.z += bf2f((uint16_t)(d.y & 0xffffu));
                acc.w += bf2f((uint16_t)(d.y >> 16));
            }
        }
        const uint2 xv = *reinterpret_cast<const uint2 *>(X + i);
        const float a[4] = {acc.x, acc.y, acc.z, acc.w};
        const uint16_t xs[4] = {(uint16_t)(xv.x & 0xffffu), (uint16_t)(xv.x >> 16), (uint16_t)(xv.y & 0xffffu),
                                (uint16_t)(xv.y >> 16)};
        uint16_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = bf2f(xs[k]) > 0.0f ? f2bf(a[k]) : (uint16_t)0;
        *reinterpret_cast<uint2 *>(dZ + i) = make_uint2((uint32_t)o[0] | ((uint32_t)o[1] << 16),
                                                        (uint32_t)o[2] | ((uint32_t)o[3] << 16));
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
    int64_t X[6], col, dx, dz;
};

static CnnSizes cnn_sizes(int32_t B) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    CnnSizes s{};
    s.X[0] = (int64_t)B * 256 * 256 * 4;
    for (int l = 0; l < 5; ++l) s.X[l + 1] = (int64_t)B * (L[l].hin / 2) * (L[l].hin / 2) * L[l].cout;
    s.col = 0;   // all five layers' im2col matrices (kept from the forward for the weight gradients)
    s.dx = (int64_t)B * 64 * 256;
    s.dz = (int64_t)B * 64 * 64;
    for (int l = 0; l < 5; ++l) {
        const int64_t M = (int64_t)B * (L[l].hin / 2) * (L[l].hin / 2);
        s.col += M * L[l].K;
        if (l > 0) s.dx = s.dx > M * L[l].K ? s.dx : M * L[l].K;
        s.dz = s.dz > M * L[l].cout ? s.dz : M * L[l].cout;
    }
    return s;
}

size_t cnn_bytes(int32_t B) {
    const CnnSizes s = cnn_sizes(B);
    int64_t np = cnn_num_params();
    size_t b = 4 * sizeof(float) * np + 2 * sizeof(uint16_t) * np;
    for (int l = 0; l < 6; ++l) b += sizeof(uint16_t) * s.X[l];
    b += 2 * sizeof(float) * (size_t)B * 64 * 64 + sizeof(float) * s.dx;
    b += sizeof(uint16_t) * s.col + 2 * sizeof(uint16_t) * s.dz + sizeof(int32_t) * 4;
    return b;
}

cudaError_t cnn_alloc(CnnBuffers &c, int32_t B) {
    const CnnSizes s = cnn_sizes(B);
    const int64_t np = cnn_num_params();
    c = CnnBuffers{};
    c.max_batch = B;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, n > 0 ? n : 16);
    };
    A((void **)&c.theta, sizeof(float) * np);
    A((void **)&c.grad, sizeof(float) * np);
    A((void **)&c.m, sizeof(float) * np);
    A((void **)&c.v, sizeof(float) * np);
    A((void **)&c.wbf, sizeof(uint16_t) * np);
    for (int l = 0; l < 6; ++l) A((void **)&c.X[l], sizeof(uint16_t) * s.X[l]);
    A((void **)&c.O, sizeof(float) * B * 64 * 64);
    A((void **)&c.dO, sizeof(float) * B * 64 * 64);
    A((void **)&c.dx, sizeof(float) * s.dx);
    A((void **)&c.col, sizeof(uint16_t) * s.col);
    A((void **)&c.dz, sizeof(uint16_t) * s.dz);
    A((void **)&c.dzp, sizeof(uint16_t) * s.dz);
    A((void **)&c.status, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(c.status, 0, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(c.m, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemset(c.v, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = init_gemm_kernels();
    return e;
}

void cnn_free(CnnBuffers &c) {
    void *ps[] = {c.theta, c.grad, c.m, c.v, c.wbf, c.X[0], c.X[1], c.X[2], c.X[3], c.X[4], c.X[5],
                  c.O, c.dO, c.dx, c.col, c.dz, c.dzp, c.status};
    for (void *p : ps)
        if (p) cudaFree(p);
    c = CnnBuffers{};
}

// After new master weights: bf16 copies for the products.
cudaError_t cnn_sync_weights(CnnBuffers &c, cudaStream_t st) {
    const int64_t np = cnn_num_params();
    k_to_bf16<<<grid1d(np), 256, 0, st>>>(c.theta, np, c.wbf);
    return cudaGetLastError();
}

// mode: a GemmMode, plus GEMM_A_MN / GEMM_B_MN when an operand is given MN-major.
static cudaError_t gemm(const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N, int K, int mode,
                        float *Cf, uint16_t *Cb, int ldc, const float *bias, int split, int32_t *status,
                        cudaStream_t st) {
    GemmArgs g{A,    B,    M,  N,  K,   lda,  ldb,   ldc, mode & 15, (mode & GEMM_A_MN) != 0, (mode & GEMM_B_MN) != 0,
               Cf,   Cb,   bias, status};
    return launch_gemm(g, split, st);
}

// Forward of B images (fp32, 3 x 256 x 256 each, concatenated) into c.O.
cudaError_t cnn_forward(CnnBuffers &c, const float *images, int32_t B, cudaStream_t st) {
    CnnLayer L[6];
    int64_t np;
    layer_table(L, &np);
    k_pack_input<<<grid1d((int64_t)B * 65536), 256, 0, st>>>(images, B, c.X[0]);
    cudaError_t e = cudaGetLastError();
    uint16_t *col = c.col;
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
        const int H = L[l].hin, Ho = H / 2;
        const int M = B * Ho * Ho;
        if (l > 0) col += (int64_t)B * (L[l - 1].hin / 2) * (L[l - 1].hin / 2) * L[l - 1].K;
        if (L[l].cin == 4)
            k_im2col4<<<grid1d((int64_t)M * 16), 256, 0, st>>>(c.X[l], B, ilog2(H), col);
        else
            k_im2col<<<grid1d((int64_t)M * 16 * (L[l].cin / 8)), 256, 0, st>>>(c.X[l], B, ilog2(H),
                                                                           ilog2(L[l].cin / 8), col);
        e = gemm(col, (int)L[l].K, c.wbf + L[l].w_off, (int)L[l].K, M, L[l].cout, (int)L[l].K,
                 GEMM_BIAS_RELU_BF16, nullptr, c.X[l + 1], L[l].cout, c.theta + L[l].b_off, 1, c.status, st);
    }
    if (e == cudaSuccess)
        e = gemm(c.X[5], 256, c.wbf + L[5].w_off, 256, B * 64, 64, 256, GEMM_BIAS_F32, c.O, nullptr, 64,
                 c.theta + L[5].b_off, 1, c.status, st);
    return e;
}

int64_t cnn_activation_count(int32_t layer, int32_t B) {
    if (layer < 0 || layer > 6 || B < 1) return -1;
    if (layer == 6) return (int64_t)B * 64 * 64;
    return cnn_sizes(B).X[layer];
}

cudaError_t cnn_activation(const CnnBuffers &c, int32_t layer, int32_t B, float *host) {
    const int64_t n = cnn_activation_count(layer, B);
    if (layer == 6) return cudaMemcpy(host, c.O, sizeof(float) * n, cudaMemcpyDeviceToHost);
    // bf16 bits are the upper half of the float32 they round to
    uint16_t *tmp = static_cast<uint16_t *>(malloc(sizeof(uint16_t) * (size_t)n));
    if (!tmp) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMemcpy(tmp, c.X[layer], sizeof(uint16_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t u = (uint32_t)tmp[i] << 16;
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
// activations and im2col matrices the forward of the same batch left in c.
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
    int64_t col_off[5];
    col_off[0] = 0;
    for (int l = 1; l < 5; ++l) col_off[l] = col_off[l - 1] + (int64_t)B * (L[l - 1].hin / 2) * (L[l - 1].hin / 2) * L[l - 1].K;
    for (int l = 4; l >= 0 && e == cudaSuccess; --l) {
        const int H = L[l].hin, Ho = H / 2, M = B * Ho * Ho;
        const int K = (int)L[l].K, Co = L[l].cout;
        // the forward of this batch left im2col(X_{l-1}) at col + col_off[l]
        e = gemm(c.dz, Co, c.col + col_off[l], K, Co, K, M, GEMM_ATOMIC_F32 | GEMM_A_MN | GEMM_B_MN, c.grad + L[l].w_off, nullptr,
                 K, nullptr, split_for(Co, K, M), c.status, st);
        k_colsum<uint16_t><<<colsum_blocks(M, Co, 2), 256, 0, st>>>(c.dz, M, Co, c.grad + L[l].b_off);
        if (l == 0 || e != cudaSuccess) break;
        // the input-gradient columns in bf16 (the product buffer holds twice as many fp32)
        uint16_t *dcol = reinterpret_cast<uint16_t *>(c.dx);
        e = gemm(c.dz, Co, c.wbf + L[l].w_off, K, M, K, Co, GEMM_STORE_BF16 | GEMM_B_MN, nullptr, dcol, K, nullptr, 1,
                 c.status, st);
        k_col2im_mask<<<grid1d((int64_t)B * H * H * L[l].cin / 4), 256, 0, st>>>(dcol, c.X[l], B, ilog2(H),
                                                                                   ilog2(L[l].cin), c.dzp);
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
    return cudaGetLastError();
}

}  // namespace dbmp
