// Forward and backward compositors (Eqs. 1-5, 8; Algorithm 1; Eq. 6, Eqs. S4-S5).
//
// One CTA owns one tile of TILE x TILE pixels; each thread owns PPT pixels of it.
// The tile's list of primitive indices (front to back) is consumed in batches of
// BATCH records, gathered from the per-primitive record array into shared memory
// with cp.async (double-buffered: batch i+1 is in flight while batch i is
// composited).  Bitmaps are read through L1 as 16-byte tap quads (one 128-bit
// load per bilinear sample).  There is no per-layer state in global memory: the
// forward keeps only T_final and the position of the last contributing layer, and
// the backward walks the list back to front recovering T_k = T_{k+1} / (1 - a_k)
// with exactly the arithmetic the forward used (sample_bitmap).
#include <cuda_runtime.h>
#include <math.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr float kTFloor = 7.88860905e-31f;  // 2^-100: layers behind are never composited

__device__ __forceinline__ int find_canvas_tile(const CanvasDesc *cv, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cv[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Gathers records list[l0 .. l0+n) into dst[0 .. n) (3 x 16-byte async copies each).
template <int NT>
__device__ __forceinline__ void stage_records(PrimRec *dst, const PrimRec *__restrict__ rec,
                                              const int32_t *__restrict__ list, int64_t l0, int n) {
    for (int j = threadIdx.x; j < n; j += NT) {
        const PrimRec *src = rec + list[l0 + j];
        const char *s = reinterpret_cast<const char *>(src);
        char *d = reinterpret_cast<char *>(dst + j);
        cp_async16(d, s);
        cp_async16(d + 16, s + 16);
        cp_async16(d + 32, s + 32);
    }
    cp_async_commit();
}

struct TileGeom {
    CanvasDesc d;
    int tx, ty;
    int64_t start;
    int len;
};

__device__ __forceinline__ TileGeom tile_geom(const RenderArgs &a, int tile_id) {
    TileGeom g;
    const int c = find_canvas_tile(a.canvas, a.n_canvas, tile_id);
    g.d = a.canvas[c];
    const int lt = tile_id - g.d.tile_base;
    g.tx = lt % g.d.ntx;
    g.ty = lt / g.d.ntx;
    g.start = a.tile_off[tile_id];
    g.len = (int)(a.tile_off[tile_id + 1] - g.start);
    return g;
}

__device__ __forceinline__ float bg_at(const RenderArgs &a, const CanvasDesc &d, int ch, int64_t pix) {
    if (a.bg_mode == DBMP_BG_CONST) return ch == 0 ? a.bg0 : (ch == 1 ? a.bg1 : a.bg2);
    if (a.bg_mode == DBMP_BG_BUFFER)
        return a.bg_buf[3 * d.pix_base + (int64_t)ch * d.H * d.W + pix];
    return 0.0f;
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
template <int TILE, int PPT, int BATCH>
__device__ __forceinline__ void fwd_tile(const RenderArgs &a, int tile_id, PrimRec *sh) {
    constexpr int NT = TILE * TILE / PPT;
    constexpr int ROWS = NT / TILE;  // rows of the tile covered by one pass of the CTA
    const TileGeom g = tile_geom(a, tile_id);
    const int Wq = a.atlas.Wb + 1;
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    const float tstop = fmaxf(a.T_stop, kTFloor);

    int px[PPT], py[PPT];
    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    int last[PPT], evals[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        px[k] = g.tx * TILE + (threadIdx.x % TILE);
        py[k] = g.ty * TILE + (threadIdx.x / TILE) + k * ROWS;
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        last[k] = -1;
        const bool inside = px[k] < g.d.W && py[k] < g.d.H;
        done[k] = !inside;
        evals[k] = inside ? g.len : 0;
    }

    if (g.len > 0) {
        stage_records<NT>(sh, a.rec, a.list, g.start, min(BATCH, g.len));
        for (int b0 = 0, it = 0; b0 < g.len; b0 += BATCH, ++it) {
            const int n = min(BATCH, g.len - b0);
            PrimRec *cur = sh + (it & 1) * BATCH;
            if (b0 + BATCH < g.len)
                stage_records<NT>(sh + ((it + 1) & 1) * BATCH, a.rec, a.list, g.start + b0 + BATCH,
                                  min(BATCH, g.len - b0 - BATCH));
            else
                cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            bool warp_done = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) warp_done = warp_done && done[k];
            if (!__all_sync(0xffffffffu, warp_done)) {
                for (int j = 0; j < n; ++j) {
                    const PrimRec r = cur[j];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (done[k]) continue;
                        if (T[k] < tstop) {
                            done[k] = true;
                            evals[k] = b0 + j;
                            continue;
                        }
                        Sample s;
                        if (sample_bitmap(r, a.atlas.quad, Wq, kw, kv, Wbf, Hbf, (float)px[k],
                                          (float)py[k], s) &&
                            s.M > 0.0f) {
                            const float al = __fmul_rn(r.a, s.M);
                            const float q = __fsub_rn(1.0f, al);
                            const float w = __fmul_rn(T[k], al);
                            C0[k] = __fmaf_rn(w, r.cr, C0[k]);
                            C1[k] = __fmaf_rn(w, r.cg, C1[k]);
                            C2[k] = __fmaf_rn(w, r.cb, C2[k]);
                            T[k] = __fmul_rn(T[k], q);
                            last[k] = b0 + j;
                        }
                    }
                }
            }
            bool all = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) all = all && (done[k] || T[k] < tstop);
            if (__syncthreads_and(all)) {
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (!done[k]) {
                        done[k] = true;
                        evals[k] = b0 + n;
                    }
                break;
            }
        }
        cp_async_wait<0>();
        __syncthreads();
    }

    int64_t ev = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (px[k] >= g.d.W || py[k] >= g.d.H) continue;
        ev += evals[k];
        const int64_t pix = (int64_t)py[k] * g.d.W + px[k];
        const int64_t HW = (int64_t)g.d.H * g.d.W;
        float *img = a.image + 3 * g.d.pix_base;
        img[pix] = __fmaf_rn(T[k], bg_at(a, g.d, 0, pix), C0[k]);
        img[HW + pix] = __fmaf_rn(T[k], bg_at(a, g.d, 1, pix), C1[k]);
        img[2 * HW + pix] = __fmaf_rn(T[k], bg_at(a, g.d, 2, pix), C2[k]);
        a.T_final[g.d.pix_base + pix] = T[k];
        a.n_last[g.d.pix_base + pix] = last[k];
    }
    // one counter update per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd((unsigned long long *)&a.status->pairs_eval_fwd,
                                                 (unsigned long long)ev);
}

template <int TILE, int PPT, int BATCH>
__global__ void __launch_bounds__(TILE * TILE / PPT) k_fwd(RenderArgs a) {
    __shared__ PrimRec sh[2 * BATCH];
    if (a.status->lists_valid == 0) return;
    fwd_tile<TILE, PPT, BATCH>(a, blockIdx.x, sh);
}

template <int TILE, int PPT, int BATCH>
__global__ void __launch_bounds__(TILE * TILE / PPT) k_fwd_persistent(RenderArgs a) {
    __shared__ PrimRec sh[2 * BATCH];
    __shared__ int item;
    if (a.status->lists_valid == 0) return;
    for (;;) {
        if (threadIdx.x == 0) item = (int)atomicAdd(&a.status->queue[0], 1u);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= a.n_tiles) break;
        fwd_tile<TILE, PPT, BATCH>(a, a.tile_order ? a.tile_order[it] : it, sh);
    }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// Sums v[0..7] over the 32 lanes of the warp (transpose reduction: 9 shuffles)
// and adds the eight totals to dst[0..7] (lanes 0, 4, ..., 28 each add one).
__device__ __forceinline__ void warp_reduce8_add(const float v[8], float *dst) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float k1[4];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float keep = up ? v[4 + i] : v[i];
            const float send = up ? v[i] : v[4 + i];
            k1[i] = keep + __shfl_xor_sync(FULL, send, 16);
        }
    }
    float k2[2];
    {
        const bool up = lane & 8;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float keep = up ? k1[2 + i] : k1[i];
            const float send = up ? k1[i] : k1[2 + i];
            k2[i] = keep + __shfl_xor_sync(FULL, send, 8);
        }
    }
    float k3;
    {
        const bool up = lane & 4;
        const float keep = up ? k2[1] : k2[0];
        const float send = up ? k2[0] : k2[1];
        k3 = keep + __shfl_xor_sync(FULL, send, 4);
    }
    k3 += __shfl_xor_sync(FULL, k3, 2);
    k3 += __shfl_xor_sync(FULL, k3, 1);
    if ((lane & 3) == 0) {
        const int vid = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (k3 != 0.0f) atomicAdd(dst + vid, k3);
    }
}

// Transmittance in front of list position `upto` for one pixel, by a forward
// re-walk (used only when the last contributing layer was exactly opaque, so
// that dividing by (1 - alpha) = 0 cannot recover it).
__device__ float rewalk_T(const RenderArgs &a, const TileGeom &g, int upto, float px, float py) {
    const int Wq = a.atlas.Wb + 1;
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    float T = 1.0f;
    for (int j = 0; j < upto; ++j) {
        const PrimRec r = a.rec[a.list[g.start + j]];
        Sample s;
        if (sample_bitmap(r, a.atlas.quad, Wq, kw, kv, Wbf, Hbf, px, py, s) && s.M > 0.0f)
            T = __fmul_rn(T, __fsub_rn(1.0f, __fmul_rn(r.a, s.M)));
    }
    return T;
}

template <int TILE, int PPT, int BATCH>
__device__ __forceinline__ void bwd_tile(const RenderArgs &a, int tile_id, PrimRec *sh, int *sh_max) {
    constexpr int NT = TILE * TILE / PPT;
    constexpr int ROWS = NT / TILE;
    const TileGeom g = tile_geom(a, tile_id);
    const int Wq = a.atlas.Wb + 1;
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    const float rho = kw / kv, irho = kv / kw;

    int px[PPT], py[PPT], last[PPT];
    float T[PPT], Y[PPT], g0[PPT], g1[PPT], g2[PPT];
    int my_max = -1;
    int64_t ev = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        px[k] = g.tx * TILE + (threadIdx.x % TILE);
        py[k] = g.ty * TILE + (threadIdx.x / TILE) + k * ROWS;
        last[k] = -1;
        T[k] = Y[k] = g0[k] = g1[k] = g2[k] = 0.0f;
        if (px[k] < g.d.W && py[k] < g.d.H) {
            const int64_t pix = (int64_t)py[k] * g.d.W + px[k];
            const int64_t HW = (int64_t)g.d.H * g.d.W;
            last[k] = min(a.n_last[g.d.pix_base + pix], g.len - 1);
            T[k] = a.T_final[g.d.pix_base + pix];
            const float *gI = a.dL_dimage + 3 * g.d.pix_base;
            g0[k] = gI[pix];
            g1[k] = gI[HW + pix];
            g2[k] = gI[2 * HW + pix];
            const float gA = a.dL_dalpha ? a.dL_dalpha[g.d.pix_base + pix] : 0.0f;
            // Y = g . R - gA B, with R = b and B = 1 behind the last layer
            Y[k] = g0[k] * bg_at(a, g.d, 0, pix) + g1[k] * bg_at(a, g.d, 1, pix) +
                   g2[k] * bg_at(a, g.d, 2, pix) - gA;
            my_max = max(my_max, last[k]);
            ev += last[k] + 1;
        }
    }
    if (threadIdx.x == 0) *sh_max = -1;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
    if ((threadIdx.x & 31) == 0) atomicMax(sh_max, my_max);
    __syncthreads();
    const int jmax = *sh_max;
    __syncthreads();

    if (jmax >= 0) {
        // batches [lo, hi) from the back
        int hi = jmax + 1;
        int lo = max(0, hi - BATCH);
        stage_records<NT>(sh, a.rec, a.list, g.start + lo, hi - lo);
        for (int it = 0; hi > 0; ++it) {
            const int nlo = max(0, lo - BATCH);
            PrimRec *cur = sh + (it & 1) * BATCH;
            if (lo > 0)
                stage_records<NT>(sh + ((it + 1) & 1) * BATCH, a.rec, a.list, g.start + nlo, lo - nlo);
            else
                cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            for (int j = hi - 1; j >= lo; --j) {
                const PrimRec r = cur[j - lo];
                float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (j > last[k]) continue;
                    Sample s;
                    if (!sample_bitmap(r, a.atlas.quad, Wq, kw, kv, Wbf, Hbf, (float)px[k],
                                       (float)py[k], s) ||
                        !(s.M > 0.0f))
                        continue;
                    any = true;
                    const float al = __fmul_rn(r.a, s.M);
                    const float q = __fsub_rn(1.0f, al);
                    float Tk;
                    if (q > 0.0f) {
                        Tk = __fdividef(T[k], q);
                    } else {
                        Tk = rewalk_T(a, g, j, (float)px[k], (float)py[k]);
                    }
                    T[k] = Tk;
                    const float gc = g0[k] * r.cr + g1[k] * r.cg + g2[k] * r.cb;
                    const float dA = Tk * (gc - Y[k]);          // dL/dalpha_k
                    const float w = Tk * al;
                    const float dM = dA * r.a;                  // dL/dM
                    const float dMdU = fmaf(s.wv, s.d1 - s.d0, s.d0);
                    const float dMdV = s.m1 - s.m0;
                    const float gU = dM * dMdU, gV = dM * dMdV;
                    v[0] += gU;
                    v[1] += gV;
                    v[2] += gU * s.Up + gV * s.Vp;
                    v[3] += rho * gU * s.Vp - irho * gV * s.Up;
                    v[4] += dA * al;
                    v[5] += g0[k] * w;
                    v[6] += g1[k] * w;
                    v[7] += g2[k] * w;
                    Y[k] = fmaf(q, Y[k], al * gc);
                }
                if (__any_sync(0xffffffffu, any)) warp_reduce8_add(v, a.graw + 8 * (int64_t)r.index);
            }
            __syncthreads();
            hi = lo;
            lo = nlo;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd((unsigned long long *)&a.status->pairs_eval_bwd,
                                                 (unsigned long long)ev);
}

template <int TILE, int PPT, int BATCH>
__global__ void __launch_bounds__(TILE * TILE / PPT) k_bwd(RenderArgs a) {
    __shared__ PrimRec sh[2 * BATCH];
    __shared__ int sh_max;
    if (a.status->lists_valid == 0) return;
    bwd_tile<TILE, PPT, BATCH>(a, blockIdx.x, sh, &sh_max);
}

template <int TILE, int PPT, int BATCH>
__global__ void __launch_bounds__(TILE * TILE / PPT) k_bwd_persistent(RenderArgs a) {
    __shared__ PrimRec sh[2 * BATCH];
    __shared__ int sh_max;
    __shared__ int item;
    if (a.status->lists_valid == 0) return;
    for (;;) {
        if (threadIdx.x == 0) item = (int)atomicAdd(&a.status->queue[1], 1u);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= a.n_tiles) break;
        bwd_tile<TILE, PPT, BATCH>(a, a.tile_order ? a.tile_order[it] : it, sh, &sh_max);
    }
}

// Per-primitive chain rule from the eight reduced sums to the raw parameters:
//   x: -(A S0 + C S1)    y: -(B S0 + D S1)    s: -S2 / s    theta: S3
//   nu: S4 (1 - sigmoid(nu))    c_j: S_{5+j} chat_j (1 - chat_j)
__global__ void k_finalize(const float *__restrict__ params, const PrimRec *__restrict__ rec,
                           const float *__restrict__ graw, float *__restrict__ dparams, int32_t N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const PrimRec r = rec[i];
    const float *S = graw + 8 * (size_t)i;
    const float *p = params + 8 * (size_t)i;
    float *o = dparams + 8 * (size_t)i;
    const float s = p[2];
    const float sig_nu = 1.0f / (1.0f + expf(-p[4]));
    o[0] += -(r.A * S[0] + r.C * S[1]);
    o[1] += -(r.B * S[0] + r.D * S[1]);
    o[2] += -S[2] / s;
    o[3] += S[3];
    o[4] += S[4] * (1.0f - sig_nu);
    o[5] += S[5] * r.cr * (1.0f - r.cr);
    o[6] += S[6] * r.cg * (1.0f - r.cg);
    o[7] += S[7] * r.cb * (1.0f - r.cb);
}

int persistent_grid(const void *kernel, int threads, cudaStream_t) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    return sms * (per > 0 ? per : 1);
}

template <int TILE, int PPT, int BATCH>
cudaError_t launch_fwd_t(const RenderArgs &a, bool persistent, cudaStream_t st) {
    constexpr int NT = TILE * TILE / PPT;
    if (persistent) {
        const int grid = persistent_grid((const void *)k_fwd_persistent<TILE, PPT, BATCH>, NT, st);
        k_fwd_persistent<TILE, PPT, BATCH><<<grid, NT, 0, st>>>(a);
    } else {
        k_fwd<TILE, PPT, BATCH><<<a.n_tiles, NT, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int TILE, int PPT, int BATCH>
cudaError_t launch_bwd_t(const RenderArgs &a, bool persistent, cudaStream_t st) {
    constexpr int NT = TILE * TILE / PPT;
    if (persistent) {
        const int grid = persistent_grid((const void *)k_bwd_persistent<TILE, PPT, BATCH>, NT, st);
        k_bwd_persistent<TILE, PPT, BATCH><<<grid, NT, 0, st>>>(a);
    } else {
        k_bwd<TILE, PPT, BATCH><<<a.n_tiles, NT, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// (tile, batch) -> instantiation.  Pixels per thread: tile 8 -> 1 (64 threads),
// tile 16 -> 2 (128 threads), tile 32 -> 4 (256 threads).
template <bool FWD>
cudaError_t dispatch(const RenderArgs &a, const RenderCfg &cfg, bool persistent, cudaStream_t st) {
#define DBMP_CASE(T, P, B)                                                                  \
    if (cfg.tile == T && cfg.batch == B)                                                    \
        return FWD ? launch_fwd_t<T, P, B>(a, persistent, st) : launch_bwd_t<T, P, B>(a, persistent, st);
    DBMP_CASE(8, 1, 32) DBMP_CASE(8, 1, 64) DBMP_CASE(8, 1, 128) DBMP_CASE(8, 1, 256)
    DBMP_CASE(16, 2, 32) DBMP_CASE(16, 2, 64) DBMP_CASE(16, 2, 128) DBMP_CASE(16, 2, 256)
    DBMP_CASE(32, 4, 32) DBMP_CASE(32, 4, 64) DBMP_CASE(32, 4, 128) DBMP_CASE(32, 4, 256)
#undef DBMP_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fwd(const RenderArgs &a, const RenderCfg &cfg, bool persistent, cudaStream_t st) {
    if (persistent) cudaMemsetAsync(&a.status->queue[0], 0, sizeof(uint32_t), st);
    return dispatch<true>(a, cfg, persistent, st);
}

cudaError_t launch_bwd(const RenderArgs &a, const RenderCfg &cfg, bool persistent, cudaStream_t st) {
    if (persistent) cudaMemsetAsync(&a.status->queue[1], 0, sizeof(uint32_t), st);
    return dispatch<false>(a, cfg, persistent, st);
}

cudaError_t launch_grad_finalize(const float *params, const PrimRec *rec, const float *graw,
                                 float *dparams, int32_t N, float, int32_t, int32_t, cudaStream_t st) {
    if (N > 0) k_finalize<<<(N + 255) / 256, 256, 0, st>>>(params, rec, graw, dparams, N);
    return cudaGetLastError();
}

}  // namespace dbmp
