// FP32 issue-rate microbenchmark: the denominator of the compositors' ALU roofline.
//
// Every thread runs kChains independent multiply-add chains, x <- x a + b, so that
// no instruction waits on the one before it.  The scalar form issues one FFMA per
// chain step (one multiply-add per lane); the packed form issues one FP32x2 FMA per
// two chains (two multiply-adds per lane per instruction).  Timing the two shows
// how many FP32 multiply-adds an SM completes per clock with either instruction.
// a and b are kernel arguments, and every chain's final value is stored, so the
// compiler can neither fold nor drop a step.
#include <cuda_runtime.h>

#include "dbmp_internal.cuh"

namespace dbmp {
namespace {

constexpr int kChains = 16;   // independent chains per thread (8 packed pairs)
constexpr int kUnroll = 8;    // chain steps per loop iteration
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_ffma(float *sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma2(float *sink, int iters, float a, float b) {
    float2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        x[c] = make_float2((float)(threadIdx.x + 2 * c) * 1e-3f, (float)(threadIdx.x + 2 * c + 1) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace dbmp

extern "C" int32_t dbmp_fp32_peak(int32_t packed, int32_t iters, float *sink_dev, int64_t n_threads,
                                  double *flops, dbmp_stream_t stream) {
    using namespace dbmp;
    if (!sink_dev || !flops || iters <= 0 || n_threads <= 0 || n_threads % kThreads != 0 ||
        n_threads / kThreads > 0x7fffffff || (packed != 0 && packed != 1))
        return record_error(DBMP_ERR_INVALID_ARG,
                            "dbmp_fp32_peak: need sink, flops, iters > 0, n_threads a positive multiple of 256, "
                            "packed 0 or 1");
    const dim3 grid((unsigned)(n_threads / kThreads)), block(kThreads);
    const float a = 0.999999f, b = 1e-7f;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (packed) k_ffma2<<<grid, block, 0, st>>>(sink_dev, iters, a, b);
    else k_ffma<<<grid, block, 0, st>>>(sink_dev, iters, a, b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(DBMP_ERR_CUDA, cudaGetErrorString(e));
    // two floating-point operations per multiply-add
    *flops = 2.0 * (double)n_threads * (double)iters * kUnroll * kChains;
    return DBMP_OK;
}
