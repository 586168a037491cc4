// Structure-aware initialisation (Sec. 3.2, "Structure-aware Initialization";
// Tab. S1: local-variance window 7, base probability 0.1, colour noise std 0.02).
//
//   k_lvar      per pixel: population variance of each channel over the 7 x 7 window
//               clipped to the canvas, averaged over R, G, B (FP64); the canvas-wide
//               minimum and maximum by atomics on the bit patterns (LV >= 0, so the
//               unsigned order of the bits is the numeric order);
//   k_qweights  NLV = (LV - min) / (max - min) and the draw weight 0.1 + 0.9 NLV,
//               quantised to an integer multiple of 2^-20;
//   k_seg_*     exclusive prefix sum of the integer weights (exact, so the draw of a
//               pixel does not depend on the order of a parallel sum);
//   k_sample    per primitive: the pixel whose cumulative-weight interval holds
//               floor(u Q_total), and its initial parameters (or, re-initialising,
//               only for primitives whose opacity sigmoid(nu) fell below a threshold).
// An optional mask (the target's alpha) restricts the draws to its support.
// Every FP64 operation that decides a pixel is explicitly rounded and taken in a
// fixed order (the window row-major, mean first), so the draws are reproducible
// bit for bit by any implementation of the same definition.
#include <cuda_runtime.h>
#include <math.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr int kLvTile = 16;
constexpr int kLvHalo = kLvTile + 6;
constexpr int kScanMaxSegs = 1024;

__global__ void k_minmax_reset(unsigned long long *minmax) {
    minmax[0] = ~0ull;
    minmax[1] = 0ull;
}

__global__ void __launch_bounds__(kLvTile * kLvTile) k_lvar(const float *__restrict__ image, int32_t H, int32_t W,
                                                            double *__restrict__ lv, unsigned long long *minmax) {
    __shared__ float tile[3][kLvHalo][kLvHalo];
    const int bx = blockIdx.x * kLvTile - 3, by = blockIdx.y * kLvTile - 3;
    const int tid = threadIdx.y * kLvTile + threadIdx.x;
    const int64_t HW = (int64_t)H * W;
    for (int i = tid; i < 3 * kLvHalo * kLvHalo; i += kLvTile * kLvTile) {
        const int c = i / (kLvHalo * kLvHalo), r = (i / kLvHalo) % kLvHalo, q = i % kLvHalo;
        const int y = by + r, x = bx + q;
        tile[c][r][q] = (y >= 0 && y < H && x >= 0 && x < W) ? image[c * HW + (int64_t)y * W + x] : 0.0f;
    }
    __syncthreads();
    const int x = blockIdx.x * kLvTile + threadIdx.x, y = blockIdx.y * kLvTile + threadIdx.y;
    double v = -1.0;
    if (x < W && y < H) {
        const int y0 = max(y - 3, 0), y1 = min(y + 3, H - 1), x0 = max(x - 3, 0), x1 = min(x + 3, W - 1);
        const double n = (double)((y1 - y0 + 1) * (x1 - x0 + 1));
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) {
            double sum = 0.0;
            for (int yy = y0; yy <= y1; ++yy)
                for (int xx = x0; xx <= x1; ++xx) sum = __dadd_rn(sum, (double)tile[c][yy - by][xx - bx]);
            const double mean = __ddiv_rn(sum, n);
            double ss = 0.0;
            for (int yy = y0; yy <= y1; ++yy)
                for (int xx = x0; xx <= x1; ++xx) {
                    const double d = __dsub_rn((double)tile[c][yy - by][xx - bx], mean);
                    ss = __dadd_rn(ss, __dmul_rn(d, d));
                }
            acc = __dadd_rn(acc, __ddiv_rn(ss, n));
        }
        v = __ddiv_rn(acc, 3.0);
        lv[(int64_t)y * W + x] = v;
    }
    // block minimum / maximum of the (non-negative) values
    __shared__ unsigned long long smin[kLvTile * kLvTile / 32], smax[kLvTile * kLvTile / 32];
    unsigned long long bmin = v >= 0.0 ? (unsigned long long)__double_as_longlong(v) : ~0ull;
    unsigned long long bmax = v >= 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
        bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    if ((tid & 31) == 0) {
        smin[tid >> 5] = bmin;
        smax[tid >> 5] = bmax;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kLvTile * kLvTile / 32; ++w) {
            bmin = min(bmin, smin[w]);
            bmax = max(bmax, smax[w]);
        }
        if (bmin != ~0ull) atomicMin(&minmax[0], bmin);
        atomicMax(&minmax[1], bmax);
    }
}

__global__ void k_qweights(double *__restrict__ lv, int64_t n, const unsigned long long *minmax,
                           const float *__restrict__ mask, int32_t *__restrict__ q, double *__restrict__ nlv_out) {
    const double mn = __longlong_as_double((long long)minmax[0]);
    const double mx = __longlong_as_double((long long)minmax[1]);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double nlv = mx > mn ? __ddiv_rn(__dsub_rn(lv[p], mn), __dsub_rn(mx, mn)) : 0.0;
        lv[p] = nlv;
        if (nlv_out) nlv_out[p] = nlv;
        const double w = __dadd_rn(0.1, __dmul_rn(0.9, nlv));
        // w in [0.1, 1]: q <= 2^20; pixels outside the mask are never drawn
        q[p] = (mask && !(mask[p] > 0.0f)) ? 0 : (int32_t)floor(__dmul_rn(w, 1048576.0));
    }
}

// Exclusive prefix sum Q[0..n] of q[0..n) (int64, exact), in three passes over
// `segs` contiguous segments of `seg` elements.
__global__ void k_seg_sum(const int32_t *__restrict__ q, int64_t n, int64_t seg, int64_t *__restrict__ bsum) {
    __shared__ long long part[32];
    const int64_t s0 = blockIdx.x * seg, s1 = min(n, s0 + seg);
    long long acc = 0;
    for (int64_t p = s0 + threadIdx.x; p < s1; p += blockDim.x) acc += q[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void k_seg_offsets(int64_t *__restrict__ bsum, int32_t segs, int64_t *__restrict__ Q_end) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long run = 0;
        for (int b = 0; b < segs; ++b) {
            const long long v = bsum[b];
            bsum[b] = run;
            run += v;
        }
        *Q_end = run;
    }
}

__global__ void k_seg_scan(const int32_t *__restrict__ q, int64_t n, int64_t seg, const int64_t *__restrict__ boff,
                           int64_t *__restrict__ Q) {
    __shared__ long long tsum[256];
    const int64_t s0 = blockIdx.x * seg, s1 = min(n, s0 + seg);
    const int64_t per = (seg + blockDim.x - 1) / blockDim.x;
    const int64_t c0 = min(s1, s0 + threadIdx.x * per), c1 = min(s1, c0 + per);
    long long acc = 0;
    for (int64_t p = c0; p < c1; ++p) acc += q[p];
    tsum[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive scan of the thread sums (256 of them)
        long long run = boff[blockIdx.x];
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const long long v = tsum[t];
            tsum[t] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = tsum[threadIdx.x];
    for (int64_t p = c0; p < c1; ++p) {
        Q[p] = run;
        run += q[p];
    }
}

// reinit_thr < 0: every primitive takes its draw; else only those with
// sigmoid(nu_i) < reinit_thr (evaluated in FP64), whose Adam moments (if given) are
// cleared and which are counted in *count.
__global__ void k_sample(const float *__restrict__ image, int32_t H, int32_t W, int32_t N,
                         const double *__restrict__ u_pos, const double *__restrict__ u_theta,
                         const double *__restrict__ n_color, double s_min, double s_max, double sigma_c, double nu,
                         const double *__restrict__ nlv, const int64_t *__restrict__ Q, float *__restrict__ params,
                         double reinit_thr, float *__restrict__ adam_m, float *__restrict__ adam_v,
                         int32_t *__restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t n = (int64_t)H * W;
    const int64_t total = Q[n];
    if (total == 0) return;   // empty mask: nothing is drawn
    if (reinit_thr >= 0.0) {
        const double sig = 1.0 / (1.0 + exp(-(double)params[8 * (int64_t)i + 4]));
        if (!(sig < reinit_thr)) return;
        for (int j = 0; j < 8; ++j) {
            if (adam_m) adam_m[8 * (int64_t)i + j] = 0.0f;
            if (adam_v) adam_v[8 * (int64_t)i + j] = 0.0f;
        }
        if (count) atomicAdd(count, 1);
    }
    const int64_t t = (int64_t)floor(__dmul_rn(u_pos[i], (double)total));
    int64_t lo = 0, hi = n - 1;   // largest p with Q[p] <= t
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (Q[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int64_t p = lo;
    float *o = params + 8 * (int64_t)i;
    o[0] = (float)(p % W);
    o[1] = (float)(p / W);
    o[2] = (float)__dsub_rn(s_max, __dmul_rn(__dsub_rn(s_max, s_min), nlv[p]));
    o[3] = (float)__dmul_rn(6.283185307179586476925286766559, u_theta[i]);
    o[4] = (float)nu;
    for (int j = 0; j < 3; ++j) {
        double c = __dadd_rn((double)image[j * n + p], __dmul_rn(sigma_c, n_color[3 * (int64_t)i + j]));
        c = c < 1e-4 ? 1e-4 : (c > 1.0 - 1e-4 ? 1.0 - 1e-4 : c);
        o[5 + j] = (float)log(c / (1.0 - c));
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t structure_init_scratch(int64_t n) {
    return align256(sizeof(double) * n) + align256(sizeof(int32_t) * n) + align256(sizeof(int64_t) * (n + 1)) +
           align256(sizeof(int64_t) * kScanMaxSegs) + align256(2 * sizeof(unsigned long long));
}

cudaError_t launch_structure_init(const float *image, const float *mask, int32_t H, int32_t W, int32_t N,
                                  const double *u_pos, const double *u_theta, const double *n_color, double s_min,
                                  double s_max, double sigma_c, double nu, void *scratch, float *params,
                                  double *nlv_out, double reinit_thr, float *adam_m, float *adam_v,
                                  int32_t *count, cudaStream_t st) {
    const int64_t n = (int64_t)H * W;
    char *b = static_cast<char *>(scratch);
    double *lv = reinterpret_cast<double *>(b);
    b += align256(sizeof(double) * n);
    int32_t *q = reinterpret_cast<int32_t *>(b);
    b += align256(sizeof(int32_t) * n);
    int64_t *Q = reinterpret_cast<int64_t *>(b);
    b += align256(sizeof(int64_t) * (n + 1));
    int64_t *bsum = reinterpret_cast<int64_t *>(b);
    b += align256(sizeof(int64_t) * kScanMaxSegs);
    unsigned long long *minmax = reinterpret_cast<unsigned long long *>(b);
    k_minmax_reset<<<1, 1, 0, st>>>(minmax);
    const dim3 g((W + kLvTile - 1) / kLvTile, (H + kLvTile - 1) / kLvTile);
    k_lvar<<<g, dim3(kLvTile, kLvTile), 0, st>>>(image, H, W, lv, minmax);
    const int64_t qblocks = (n + 255) / 256;
    k_qweights<<<(int)(qblocks < 152 * 16 ? qblocks : 152 * 16), 256, 0, st>>>(lv, n, minmax, mask, q, nlv_out);
    const int64_t want = (n + 4095) / 4096;
    const int32_t segs = (int32_t)(want < 1 ? 1 : (want > kScanMaxSegs ? kScanMaxSegs : want));
    const int64_t seg = (n + segs - 1) / segs;
    k_seg_sum<<<segs, 256, 0, st>>>(q, n, seg, bsum);
    k_seg_offsets<<<1, 32, 0, st>>>(bsum, segs, Q + n);
    k_seg_scan<<<segs, 256, 0, st>>>(q, n, seg, bsum, Q);
    if (N > 0)
        k_sample<<<(N + 255) / 256, 256, 0, st>>>(image, H, W, N, u_pos, u_theta, n_color, s_min, s_max, sigma_c,
                                                  nu, lv, Q, params, reinit_thr, adam_m, adam_v, count);
    return cudaGetLastError();
}

}  // namespace dbmp
