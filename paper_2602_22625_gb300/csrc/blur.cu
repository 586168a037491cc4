// Gaussian blur of the primitive bitmaps (Sec. 3.2 "Blurring Primitives for
// Enriching Gradients"; Tab. S1 do_gaussian_blur, blur_sigma = 1.0): each bitmap
// convolved with the normalised Gaussian truncated at r = ceil(3 sigma), texels
// outside the bitmap zero.  The 2-D kernel is the outer product of the 1-D one, so
// one CTA blurs a 32 x 32 output tile in two passes through shared memory: the
// (32 + 2r)^2 input window, then its rows, then the columns of that.
#include <cuda_runtime.h>
#include <math.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr int kBlurTile = 32;

__global__ void __launch_bounds__(256) k_blur(const float *__restrict__ in, float *__restrict__ out, int32_t Hb,
                                              int32_t Wb, BlurTaps taps) {
    extern __shared__ float sm[];
    __shared__ float w_sh[2 * kMaxBlurRadius + 1];   // taps, indexed at run time
    const int r = taps.r, span = kBlurTile + 2 * r;
    float *win = sm;                   // [span][span] input window
    float *rows = sm + span * span;    // [span][kBlurTile] horizontal pass
    const int64_t plane = (int64_t)Hb * Wb;
    const float *src = in + blockIdx.z * plane;
    float *dst = out + blockIdx.z * plane;
    const int y0 = blockIdx.y * kBlurTile - r, x0 = blockIdx.x * kBlurTile - r;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    if (tid <= 2 * r) w_sh[tid] = taps.w[tid];
    for (int i = tid; i < span * span; i += nth) {
        const int y = y0 + i / span, x = x0 + i % span;
        win[i] = (y >= 0 && y < Hb && x >= 0 && x < Wb) ? src[(int64_t)y * Wb + x] : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < span * kBlurTile; i += nth) {
        const int yy = i / kBlurTile, xx = i % kBlurTile;
        const float *w = win + yy * span + xx;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) acc = fmaf(w_sh[k], w[k], acc);
        rows[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < kBlurTile * kBlurTile; i += nth) {
        const int yy = i / kBlurTile, xx = i % kBlurTile;
        const int y = blockIdx.y * kBlurTile + yy, x = blockIdx.x * kBlurTile + xx;
        if (y >= Hb || x >= Wb) continue;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) acc = fmaf(w_sh[k], rows[(yy + k) * kBlurTile + xx], acc);
        dst[(int64_t)y * Wb + x] = acc;
    }
}

}  // namespace

BlurTaps blur_taps(double sigma) {
    BlurTaps t{};
    t.r = (int32_t)ceil(3.0 * sigma);
    double w[2 * kMaxBlurRadius + 1], sum = 0.0;
    for (int k = -t.r; k <= t.r; ++k) sum += (w[k + t.r] = exp(-(double)(k * k) / (2.0 * sigma * sigma)));
    for (int k = 0; k <= 2 * t.r; ++k) t.w[k] = (float)(w[k] / sum);
    return t;
}

size_t blur_smem_bytes(int32_t r) {
    const int span = kBlurTile + 2 * r;
    return sizeof(float) * ((size_t)span * span + (size_t)span * kBlurTile);
}

cudaError_t launch_blur(const float *in, float *out, int32_t n_bmp, int32_t Hb, int32_t Wb, const BlurTaps &taps,
                        cudaStream_t st) {
    // at most (32 + 30)^2 + 62 x 32 floats = 23 KB of shared memory: no opt-in needed
    const dim3 grid((Wb + kBlurTile - 1) / kBlurTile, (Hb + kBlurTile - 1) / kBlurTile, n_bmp);
    k_blur<<<grid, dim3(32, 8), blur_smem_bytes(taps.r), st>>>(in, out, Hb, Wb, taps);
    return cudaGetLastError();
}

}  // namespace dbmp
