// Atlas layout, MSE loss gradient and the Adam update (Tab. S1).
#include <cuda_runtime.h>
#include <math.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

// plane row b (H_b + 1) + v = bitmap b's row v for v < H_b, zero for v = H_b.
__global__ void k_plane(const float *__restrict__ tex, float *__restrict__ plane, int64_t pitch, int32_t n_bmp,
                        int32_t Hb, int32_t Wb) {
    const int64_t rows = (int64_t)n_bmp * (Hb + 1);
    const int64_t total = rows * Wb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / Wb;
        const int u = (int)(i - row * Wb);
        const int b = (int)(row / (Hb + 1)), v = (int)(row - (int64_t)b * (Hb + 1));
        plane[row * pitch + u] = v < Hb ? tex[((int64_t)b * Hb + v) * Wb + u] : 0.0f;
    }
}

// nzbox[b] = (u0, u1, v0, v1): the first and last column and row of bitmap b that
// hold a texel > 0, the box the binning specification sizes a primitive's tile
// rectangle from; (W_b, -1, H_b, -1) for an all-zero bitmap.  One CTA per bitmap.
__global__ void k_nzbox(const float *__restrict__ tex, int4 *__restrict__ nzbox, int32_t Hb, int32_t Wb) {
    __shared__ int u0, u1, v0, v1;
    if (threadIdx.x == 0) {
        u0 = Wb;
        u1 = -1;
        v0 = Hb;
        v1 = -1;
    }
    __syncthreads();
    const float *P = tex + (int64_t)blockIdx.x * Hb * Wb;
    int a0 = Wb, a1 = -1, b0 = Hb, b1 = -1;
    for (int64_t i = threadIdx.x; i < (int64_t)Hb * Wb; i += blockDim.x) {
        if (P[i] > 0.0f) {
            const int v = (int)(i / Wb), u = (int)(i - (int64_t)v * Wb);
            a0 = min(a0, u);
            a1 = max(a1, u);
            b0 = min(b0, v);
            b1 = max(b1, v);
        }
    }
    if (a1 >= 0) {
        atomicMin(&u0, a0);
        atomicMax(&u1, a1);
        atomicMin(&v0, b0);
        atomicMax(&v1, b1);
    }
    __syncthreads();
    if (threadIdx.x == 0) nzbox[blockIdx.x] = make_int4(u0, u1, v0, v1);
}

// sat[b][v][u] = number of texels P[v'][u'] > 0 with v' < v and u' < u
// (v in [0, H_b], u in [0, W_b]); one CTA per bitmap: row prefix sums, then columns.
__global__ void k_sat(const float *__restrict__ tex, int32_t *__restrict__ sat, int32_t Hb, int32_t Wb) {
    const int b = blockIdx.x;
    const float *P = tex + (int64_t)b * Hb * Wb;
    int32_t *S = sat + (int64_t)b * (Hb + 1) * (Wb + 1);
    for (int u = threadIdx.x; u <= Wb; u += blockDim.x) S[u] = 0;
    for (int v = threadIdx.x; v < Hb; v += blockDim.x) {
        int32_t run = 0;
        S[(int64_t)(v + 1) * (Wb + 1)] = 0;
        for (int u = 0; u < Wb; ++u) {
            run += P[(int64_t)v * Wb + u] > 0.0f ? 1 : 0;
            S[(int64_t)(v + 1) * (Wb + 1) + u + 1] = run;
        }
    }
    __syncthreads();
    for (int u = threadIdx.x; u <= Wb; u += blockDim.x) {
        int32_t run = 0;
        for (int v = 1; v <= Hb; ++v) {
            run += S[(int64_t)v * (Wb + 1) + u];
            S[(int64_t)v * (Wb + 1) + u] = run;
        }
    }
}

// dL/dI = 2 (I - I*) / n and the loss sum (I - I*)^2 / n.  The differences are
// formed in fp32 (the upstream gradient's precision), the squares summed per thread
// with acc_sq and across threads in FP64.  Four elements per thread and load when
// all pointers are 16-byte aligned; the tail and unaligned buffers take the scalar
// loop.
__global__ void k_mse(const float *__restrict__ I, const float *__restrict__ Tg, int64_t n,
                      float *__restrict__ dL, double *loss) {
    __shared__ double red[32];
    const float scale = (float)(2.0 / (double)n);
    float s = 0.0f, c = 0.0f;
    const bool vec = ((((uintptr_t)I) | ((uintptr_t)Tg) | ((uintptr_t)dL)) & 15) == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const float4 *I4 = reinterpret_cast<const float4 *>(I), *T4 = reinterpret_cast<const float4 *>(Tg);
    for (int64_t i0 = tid; i0 < n4; i0 += 2 * nth) {
        // two independent float4 pairs in flight per thread
        float4 a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = i0 + u * nth;
            if (i < n4) {
                a[u] = __ldg(I4 + i);
                b[u] = __ldg(T4 + i);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = i0 + u * nth;
            if (i >= n4) continue;
            const float4 d = make_float4(a[u].x - b[u].x, a[u].y - b[u].y, a[u].z - b[u].z, a[u].w - b[u].w);
            reinterpret_cast<float4 *>(dL)[i] = make_float4(scale * d.x, scale * d.y, scale * d.z, scale * d.w);
            acc_sq(d.x, s, c);
            acc_sq(d.y, s, c);
            acc_sq(d.z, s, c);
            acc_sq(d.w, s, c);
        }
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += nth) {
        const float d = I[i] - Tg[i];
        dL[i] = scale * d;
        acc_sq(d, s, c);
    }
    double acc = (double)s + (double)c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss, acc / (double)n);
    }
}

// Eq. 9 (Sec. 3.3.2), both squared norms read as means: over the pixels p (planar
// images of n1 pixels, n3 = 3 n1 values), m_p = [alpha*_p > 0],
//   L = sum m_p (I - I*)^2 / n3 + lam sum (I_alpha - alpha*)^2 / n1,  I_alpha = 1 - T_N,
//   dL/dI = 2 m_p (I - I*) / n3,  dL/dI_alpha = 2 lam (I_alpha - alpha*) / n1.
// Per-thread sums are compensated (acc_sq), cross-thread sums FP64.
// The rendered alpha channel I_alpha = 1 - T_N (Sec. 3.3.2) from the forward's T_final.
__global__ void k_alpha_from_T(const float *__restrict__ T, float *__restrict__ alpha, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        alpha[i] = 1.0f - T[i];
}

__global__ void k_alpha_loss(const float *__restrict__ I, const float *__restrict__ T, const float *__restrict__ It,
                             const float *__restrict__ at, int64_t n1, float lam, float *__restrict__ dI,
                             float *__restrict__ dA, double *loss) {
    __shared__ double red[32];
    const float s3 = (float)(2.0 / (3.0 * (double)n1)), s1 = (float)(2.0 * (double)lam / (double)n1);
    float c0 = 0.0f, e0 = 0.0f, c1 = 0.0f, e1 = 0.0f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n1; p += (int64_t)gridDim.x * blockDim.x) {
        const float a = at[p];
        const bool in = a > 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float d = in ? I[ch * n1 + p] - It[ch * n1 + p] : 0.0f;
            dI[ch * n1 + p] = s3 * d;
            acc_sq(d, c0, e0);
        }
        const float r = (1.0f - T[p]) - a;
        dA[p] = s1 * r;
        acc_sq(r, c1, e1);
    }
    double acc = ((double)c0 + (double)e0) / (3.0 * (double)n1) + (double)lam * ((double)c1 + (double)e1) / (double)n1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss, acc);
    }
}

struct AdamArgs {
    float lr, gamma, beta1, beta2, eps;
    float gains[8];
    int32_t zero_grad;
};

__global__ void k_adam(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, const int32_t *step, AdamArgs c) {
    pdl_wait();
    pdl_trigger();
    const int t = *step + 1;
    const float bc1 = 1.0f - powf(c.beta1, (float)t);
    const float bc2 = 1.0f - powf(c.beta2, (float)t);
    const float lr_t = c.lr * powf(c.gamma, (float)(t - 1));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        if (c.zero_grad) g[i] = 0.0f;
        const float mi = c.beta1 * m[i] + (1.0f - c.beta1) * gi;
        const float vi = c.beta2 * v[i] + (1.0f - c.beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        p[i] -= lr_t * c.gains[i & 7] * mh / (sqrtf(vh) + c.eps);
    }
}

// The same update, one primitive (eight columns, two 16-byte vectors per array) per
// thread, with the column gains in registers; for 16-byte aligned arrays.
__global__ void k_adam8(float4 *__restrict__ p, float4 *__restrict__ g, float4 *__restrict__ m,
                        float4 *__restrict__ v, int32_t N, const int32_t *step, AdamArgs c) {
    pdl_wait();
    pdl_trigger();
    const int t = *step + 1;
    const float bc1 = 1.0f - powf(c.beta1, (float)t);
    const float bc2 = 1.0f - powf(c.beta2, (float)t);
    const float lr_t = c.lr * powf(c.gamma, (float)(t - 1));
    // one float4 per thread: half (h) of primitive k / 2's eight parameters
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 2 * (int64_t)N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(k & 1);
        const float4 g4 = g[k], m4 = m[k], v4 = v[k], p4 = p[k];
        if (c.zero_grad) g[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float gi[4] = {g4.x, g4.y, g4.z, g4.w}, mo[4] = {m4.x, m4.y, m4.z, m4.w};
        const float vo[4] = {v4.x, v4.y, v4.z, v4.w}, po[4] = {p4.x, p4.y, p4.z, p4.w};
        float mn[4], vn[4], pn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            mn[e] = c.beta1 * mo[e] + (1.0f - c.beta1) * gi[e];
            vn[e] = c.beta2 * vo[e] + (1.0f - c.beta2) * gi[e] * gi[e];
            const float mh = mn[e] / bc1, vh = vn[e] / bc2;
            const float gain = h ? c.gains[4 + e] : c.gains[e];
            pn[e] = po[e] - lr_t * gain * mh / (sqrtf(vh) + c.eps);
        }
        m[k] = make_float4(mn[0], mn[1], mn[2], mn[3]);
        v[k] = make_float4(vn[0], vn[1], vn[2], vn[3]);
        p[k] = make_float4(pn[0], pn[1], pn[2], pn[3]);
    }
}

__global__ void k_step_inc(int32_t *step) {
    pdl_wait();
    *step += 1;
}

// Blocks for n work items of `threads` threads, at most `per_sm` resident blocks
// per SM (grid-stride loops take the rest).
int grid_for(int64_t n, int threads, int per_sm = 8) {
    const int sms = sm_count();
    const int64_t want = (n + threads - 1) / threads;
    return (int)(want < (int64_t)sms * per_sm ? (want > 0 ? want : 1) : (int64_t)sms * per_sm);
}

}  // namespace

int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 152;
    if (dev < 64) cached[dev] = n;   // the same value from any racing thread
    return n;
}

cudaError_t launch_atlas_build(const float *texels, float *plane, int64_t pitch, int32_t *sat, int4 *nzbox, int32_t n_bmp,
                               int32_t Hb, int32_t Wb, cudaStream_t st) {
    const int64_t total = (int64_t)n_bmp * (Hb + 1) * Wb;
    k_plane<<<grid_for(total, 256), 256, 0, st>>>(texels, plane, pitch, n_bmp, Hb, Wb);
    k_sat<<<n_bmp, 256, 0, st>>>(texels, sat, Hb, Wb);
    k_nzbox<<<n_bmp, 256, 0, st>>>(texels, nzbox, Hb, Wb);
    return cudaGetLastError();
}

size_t atlas_plane_pitch(int32_t Wb) { return ((size_t)Wb * sizeof(float) + 127) & ~(size_t)127; }

cudaError_t atlas_texture_fits(int32_t n_bmp, int32_t Hb, int32_t Wb, bool *fits) {
    int dev = 0, maxw = 0, maxh = 0, maxp = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLinearWidth, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLinearHeight, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxTexture2DLinearPitch, dev);
    if (e != cudaSuccess) return e;
    *fits = Wb <= maxw && (int64_t)n_bmp * (Hb + 1) <= maxh && atlas_plane_pitch(Wb) <= (size_t)maxp;
    return cudaSuccess;
}

cudaError_t atlas_texture_create(float *plane, size_t pitch_bytes, int32_t n_bmp, int32_t Hb, int32_t Wb,
                                 cudaTextureObject_t *out) {
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypePitch2D;
    rd.res.pitch2D.devPtr = plane;
    rd.res.pitch2D.desc = cudaCreateChannelDesc<float>();
    rd.res.pitch2D.width = (size_t)Wb;
    rd.res.pitch2D.height = (size_t)n_bmp * (Hb + 1);
    rd.res.pitch2D.pitchInBytes = pitch_bytes;
    cudaTextureDesc td{};
    td.addressMode[0] = cudaAddressModeBorder;
    td.addressMode[1] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;   // border colour: zero-initialised
    return cudaCreateTextureObject(out, &rd, &td, nullptr);
}

cudaError_t launch_mse_grad(const float *image, const float *target, int64_t n, float *dL,
                            double *loss, cudaStream_t st) {
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    // four resident blocks per SM: enough loads in flight for HBM with two float4
    // pairs per thread, and half the FP64 atomics of a full grid
    if (n > 0) k_mse<<<grid_for((n + 3) / 4, 256, 4), 256, 0, st>>>(image, target, n, dL, loss);
    return cudaGetLastError();
}

cudaError_t launch_alpha_from_T(const float *T_final, float *alpha, int64_t n, cudaStream_t st) {
    if (n > 0) k_alpha_from_T<<<grid_for(n, 256), 256, 0, st>>>(T_final, alpha, n);
    return cudaGetLastError();
}

cudaError_t launch_alpha_loss(const float *image, const float *T_final, const float *target,
                              const float *target_alpha, int64_t n_pix, float lam, float *dL_dimage,
                              float *dL_dalpha, double *loss, cudaStream_t st) {
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (n_pix > 0)
        k_alpha_loss<<<grid_for(n_pix, 256), 256, 0, st>>>(image, T_final, target, target_alpha, n_pix, lam,
                                                            dL_dimage, dL_dalpha, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *g, float *m, float *v, int32_t N, int32_t *step,
                        const DbmpAdamConfig &cfg, cudaStream_t st) {
    AdamArgs c;
    c.lr = cfg.lr;
    c.gamma = cfg.gamma;
    c.beta1 = cfg.beta1;
    c.beta2 = cfg.beta2;
    c.eps = cfg.eps;
    for (int j = 0; j < 8; ++j) c.gains[j] = cfg.gains[j];
    c.zero_grad = cfg.zero_grad;
    const int64_t n = (int64_t)N * 8;
    const bool aligned = ((((uintptr_t)p) | ((uintptr_t)g) | ((uintptr_t)m) | ((uintptr_t)v)) & 15) == 0;
    cudaError_t e = cudaSuccess;
    if (n > 0 && aligned)
        e = launch_pdl(k_adam8, dim3(grid_for(2 * (int64_t)N, 128)), dim3(128), 0, st, reinterpret_cast<float4 *>(p),
                       reinterpret_cast<float4 *>(g), reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), N,
                       static_cast<const int32_t *>(step), c);
    else if (n > 0)
        e = launch_pdl(k_adam, dim3(grid_for(n, 256)), dim3(256), 0, st, p, g, m, v, n,
                       static_cast<const int32_t *>(step), c);
    if (e == cudaSuccess) e = launch_pdl(k_step_inc, dim3(1), dim3(1), 0, st, step);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dbmp
