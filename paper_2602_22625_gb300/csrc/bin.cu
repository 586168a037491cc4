// Tile binning (Sec. 3.1.1 "Parallelization", Sec. S1.3) on the GPU.
//
// The paper bins on the CPU.  Here every step runs on the device:
//   k_prep     per primitive: FP64 transform coefficients rounded to a 48-byte record
//              (Eqs. 1-3 folded), and the fp32 bounding-box rectangle of tiles;
//   k_count    per (chunk of primitives, slab of tile rows): per-tile hit counts from
//              column and row bit masks (a tile's mask is their AND);
//   k_colscan  per tile: exclusive scan over chunks  -> each chunk's base in the tile;
//   k_tilescan exclusive scan over tiles             -> tile offsets, K = sum_t d_t;
//   k_scatter  per (chunk, slab), one warp per tile: the set bits of the tile's mask,
//              in index order, written as one contiguous run at the chunk's base.
// Together this is a stable counting sort keyed on the tile id.  Because each run
// holds its primitives in index order, each list comes out sorted front to back, which is
// exactly the order of the keys (tile << 32 | index): no 64-bit keys are formed and
// no radix passes over them are needed.
#include <cuda_runtime.h>
#include <math.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {


__device__ __forceinline__ int find_canvas_by(const CanvasDesc *cv, int n, int value, int which) {
    // largest c with base(c) <= value; which: 0 = prim_base, 1 = chunk_base, 2 = tile_base
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int b = which == 0 ? cv[mid].prim_base : (which == 1 ? cv[mid].chunk_base : cv[mid].tile_base);
        if (b <= value) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// sin, cos of the binning specification: Cody-Waite reduction by pi/2 with a
// three-part constant, Taylor polynomials of degree 9 (sin) and 8 (cos) on
// [-pi/4, pi/4], the quadrant's signs.  Every operation rounds once (explicit
// intrinsics).  False (and 1, 1) for |th| > 65536, outside the reduction's range.
__device__ __forceinline__ bool spec_sincos(float th, float &sn, float &cs) {
    if (!(fabsf(th) <= 65536.0f)) {
        sn = 1.0f;
        cs = 1.0f;
        return false;
    }
    const float two_over_pi = 0.636619772367581343f;
    const float C1 = 1.5703125f;
    const float C2 = 4.83751296997070312e-4f;
    const float C3 = 7.54978995489188e-8f;
    const float k = rintf(__fmul_rn(th, two_over_pi));
    float r = __fsub_rn(th, __fmul_rn(k, C1));
    r = __fsub_rn(r, __fmul_rn(k, C2));
    r = __fsub_rn(r, __fmul_rn(k, C3));
    const float r2 = __fmul_rn(r, r);
    float sp = 1.0f / 362880.0f;
    sp = __fadd_rn(__fmul_rn(sp, r2), -1.0f / 5040.0f);
    sp = __fadd_rn(__fmul_rn(sp, r2), 1.0f / 120.0f);
    sp = __fadd_rn(__fmul_rn(sp, r2), -1.0f / 6.0f);
    const float sr = __fadd_rn(r, __fmul_rn(__fmul_rn(r, r2), sp));
    float cp = 1.0f / 40320.0f;
    cp = __fadd_rn(__fmul_rn(cp, r2), -1.0f / 720.0f);
    cp = __fadd_rn(__fmul_rn(cp, r2), 1.0f / 24.0f);
    cp = __fadd_rn(__fmul_rn(cp, r2), -0.5f);
    const float cr = __fadd_rn(1.0f, __fmul_rn(r2, cp));
    const int q = (((int)k % 4) + 4) % 4;   // quadrant: th = k pi/2 + r
    sn = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
    cs = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
    return true;
}

__device__ __forceinline__ void spec_abs_sincos(float th, float &as, float &ac) {
    float sn, cs;
    spec_sincos(th, sn, cs);
    as = fabsf(sn);
    ac = fabsf(cs);
}

__device__ __forceinline__ bool all_finite8(const float *p) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) ok = ok && isfinite(p[j]);
    return ok;
}

// Half-extents of the padded box of the bitmap's whole support with its zero-padding
// ring (e_u = 1 + 2/(W_b-1), e_v likewise) rotated by theta and scaled by |s|, one
// IEEE operation at a time: the footprint A_i = (2 hx + 2)(2 hy + 2) of the scaling
// statistics (Sec. S4).
__device__ __forceinline__ void spec_halfext(float s_raw, float theta, int32_t Hb, int32_t Wb, float &hx, float &hy) {
    const float eu = __fadd_rn(1.0f, __fdiv_rn(2.0f, (float)(Wb - 1)));
    const float ev = __fadd_rn(1.0f, __fdiv_rn(2.0f, (float)(Hb - 1)));
    float as, ac;
    spec_abs_sincos(theta, as, ac);
    const float s = fabsf(s_raw);
    hx = __fmul_rn(s, __fadd_rn(__fmul_rn(ac, eu), __fmul_rn(as, ev)));
    hy = __fmul_rn(s, __fadd_rn(__fmul_rn(as, eu), __fmul_rn(ac, ev)));
}

__global__ void k_prep(const float *__restrict__ params, const int32_t *__restrict__ bitmap_id,
                       const CanvasDesc *__restrict__ cv, int32_t n_canvas, int32_t N,
                       AtlasView atlas, float alpha_max, int32_t tile, PrimRec *__restrict__ rec,
                       int4 *__restrict__ rect, DevStatus *status) {
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = find_canvas_by(cv, n_canvas, i, 0);
    const CanvasDesc d = cv[c];
    float p[8];
    const float4 *p4 = reinterpret_cast<const float4 *>(params + 8 * (size_t)i);
    const float4 lo = p4[0], hi = p4[1];
    p[0] = lo.x; p[1] = lo.y; p[2] = lo.z; p[3] = lo.w;
    p[4] = hi.x; p[5] = hi.y; p[6] = hi.z; p[7] = hi.w;

    // ---- record: transform coefficients in FP64, rounded once ----
    const double kw = 0.5 * (double)(atlas.Wb - 1), kv = 0.5 * (double)(atlas.Hb - 1);
    double sn, cs;
    sincos((double)p[3], &sn, &cs);
    const double inv_s = 1.0 / (double)p[2];
    PrimRec r;
    r.x = p[0];
    r.y = p[1];
    r.A = (float)(kw * cs * inv_s);
    r.B = (float)(kw * sn * inv_s);
    r.C = (float)(-kv * sn * inv_s);
    r.D = (float)(kv * cs * inv_s);
    // opacity and colour sigmoids in fp32 (a few ulps; they enter the image linearly)
    r.a = alpha_max / (1.0f + expf(-p[4]));
    r.bmp_row = bitmap_id[i] * (atlas.Hb + 1);  // checked below
    r.cr = 1.0f / (1.0f + expf(-p[5]));
    r.cg = 1.0f / (1.0f + expf(-p[6]));
    r.cb = 1.0f / (1.0f + expf(-p[7]));
    r.index = i;
    const int32_t bid = bitmap_id[i];
    const bool bid_ok = bid >= 0 && bid < atlas.n_bmp;
    if (!bid_ok) {
        r.bmp_row = 0;
        atomicAdd(&status->n_degenerate, 1);
    }
    const bool valid = bid_ok && all_finite8(p) && p[2] != 0.0f;
    // |A|, |B|, |C|, |D| <= 2^100 keeps every bitmap coordinate a compositor forms
    // for a pixel the primitive's tile rectangle covers finite in float32.
    const float kMaxCoef = 1.2676506e30f;   // 2^100
    if (valid && !(fabsf(r.A) <= kMaxCoef && fabsf(r.B) <= kMaxCoef && fabsf(r.C) <= kMaxCoef &&
                   fabsf(r.D) <= kMaxCoef)) {
        // |s| below ~1e-28 of the bitmap's half-width: the primitive is drawn with
        // zero opacity and counted.
        r.a = 0.0f;
        r.A = r.B = r.C = r.D = 0.0f;
        atomicAdd(&status->n_degenerate, 1);
    }
    rec[i] = r;

    // ---- tile rectangle: the fp32 binning specification ----
    // The box holds every pixel where M can be non-zero: its bitmap coordinates lie
    // within one texel of the bitmap's non-zero box [u0, u1] x [v0, v1] (zero padding,
    // Sec. S1.1).  That texel box (centre (cu, cv), half-extents (hu, hv) from the
    // bitmap centre, exact) maps to a rotated box of centre s (cos uc - sin vc,
    // sin uc + cos vc) and axis-aligned half-extents |s| (|cos| eu + |sin| ev),
    // |s| (|sin| eu + |cos| ev) in normalised coordinates (Eq. 1), widened by the
    // margin m = 1 + |s| 2^-19 pixels, which exceeds the rounding of these steps and of
    // the compositors' transform.  An all-zero bitmap lists the primitive nowhere.
    int4 rc = make_int4(0, 0, -1, -1);
    const int4 nz = bid_ok ? atlas.nzbox[bid] : make_int4(1, 0, 1, 0);
    if (valid && nz.x <= nz.y) {
        const float kw = __fmul_rn((float)(atlas.Wb - 1), 0.5f), kv = __fmul_rn((float)(atlas.Hb - 1), 0.5f);
        const float cu = __fmul_rn(__fsub_rn((float)(nz.x + nz.y), (float)(atlas.Wb - 1)), 0.5f);
        const float hu = __fmul_rn((float)(nz.y - nz.x + 2), 0.5f);
        const float cv = __fmul_rn(__fsub_rn((float)(nz.z + nz.w), (float)(atlas.Hb - 1)), 0.5f);
        const float hv = __fmul_rn((float)(nz.w - nz.z + 2), 0.5f);
        const float uc = __fdiv_rn(cu, kw), eu = __fdiv_rn(hu, kw);
        const float vc = __fdiv_rn(cv, kv), ev = __fdiv_rn(hv, kv);
        const float s = p[2], as = fabsf(p[2]);
        float sn, cs, dxc, dyc, hx, hy;
        if (spec_sincos(p[3], sn, cs)) {
            dxc = __fmul_rn(s, __fsub_rn(__fmul_rn(cs, uc), __fmul_rn(sn, vc)));
            dyc = __fmul_rn(s, __fadd_rn(__fmul_rn(sn, uc), __fmul_rn(cs, vc)));
            hx = __fmul_rn(as, __fadd_rn(__fmul_rn(fabsf(cs), eu), __fmul_rn(fabsf(sn), ev)));
            hy = __fmul_rn(as, __fadd_rn(__fmul_rn(fabsf(sn), eu), __fmul_rn(fabsf(cs), ev)));
        } else {   // rotation unknown: a box about (x, y) that holds every rotation
            dxc = 0.0f;
            dyc = 0.0f;
            hx = __fmul_rn(as, __fadd_rn(__fadd_rn(__fadd_rn(fabsf(uc), eu), fabsf(vc)), ev));
            hy = hx;
        }
        const float m = __fadd_rn(1.0f, __fmul_rn(as, 1.9073486328125e-06f));   // 1 + |s| 2^-19
        const float cx = __fadd_rn(p[0], dxc), cy = __fadd_rn(p[1], dyc);
        const float inv_t = __fdiv_rn(1.0f, (float)tile);
        const float fx0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(cx, hx), m), inv_t));
        const float fx1 = floorf(__fmul_rn(__fadd_rn(__fadd_rn(cx, hx), m), inv_t));
        const float fy0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(cy, hy), m), inv_t));
        const float fy1 = floorf(__fmul_rn(__fadd_rn(__fadd_rn(cy, hy), m), inv_t));
        const float mx = (float)(d.ntx - 1), my = (float)(d.nty - 1);
        if (fx1 >= 0.0f && fy1 >= 0.0f && fx0 <= mx && fy0 <= my) {
            rc.x = fx0 < 0.0f ? 0 : (int)fx0;
            rc.y = fy0 < 0.0f ? 0 : (int)fy0;
            rc.z = fx1 > mx ? d.ntx - 1 : (int)fx1;
            rc.w = fy1 > my ? d.nty - 1 : (int)fy1;
        }
    }
    rect[i] = rc;
}

// Binning work unit: one CTA per (chunk of 2^chunk_log2 primitives, slab of tile
// rows), taking the chunk in passes of blockDim.x primitives, one warp per 32.
// A primitive's tiles form a rectangle, so primitive (w, q) of a pass overlaps tile
// (tx, ty) iff bit q is set in both colw[tx][w] (tx0 <= tx <= tx1) and
// roww[ty][w] (ty0 <= ty <= ty1): the CTA keeps (columns + slab rows) x warps
// words instead of a mask per tile, and a tile's mask is their AND.
struct SlabWork {
    int local, p0, p1, sy0, sy1, rows, slab_tiles, ntiles, nw;
    uint32_t *colw, *roww;   // [ntx][nw], [rows][nw] words in shared memory
};

__device__ __forceinline__ bool slab_work(const CanvasDesc &d, uint32_t *smem, SlabWork &s) {
    if ((int)blockIdx.y >= d.n_slabs) return false;
    s.ntiles = d.ntx * d.nty;
    s.nw = blockDim.x >> 5;
    s.local = (int)blockIdx.x - d.chunk_base;
    s.p0 = d.prim_base + (s.local << d.chunk_log2);
    s.p1 = d.prim_base + (int)min((int64_t)d.N, ((int64_t)s.local + 1) << d.chunk_log2);
    s.sy0 = blockIdx.y * d.slab_rows;
    s.sy1 = min(s.sy0 + d.slab_rows, d.nty);
    s.rows = s.sy1 - s.sy0;
    s.slab_tiles = s.rows * d.ntx;
    s.colw = smem;
    s.roww = smem + d.ntx * s.nw;
    return true;
}

// Bits [lo, hi] of the 32 positions [p0, p0 + 32) covered by the inclusive run [a, b].
__device__ __forceinline__ uint32_t run_bits(int a, int b, int p0) {
    if (b < p0 || a > p0 + 31) return 0u;
    const int lo = max(a - p0, 0), hi = min(b - p0, 31);
    return (0xffffffffu >> (31 - hi)) & (0xffffffffu << lo);
}

// Transposes the warp's 32 x 32 bit matrix held one row per lane (bit c of lane q)
// into one column per lane (bit q of lane c): five butterfly stages, stage j
// exchanging the off-diagonal j x j blocks between lanes l and l ^ j.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t lowmask[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const uint32_t m = lowmask[s];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Builds colw / roww for the pass starting at primitive q0: lane q of warp w takes
// the rectangle of primitive q0 + 32 w + q, forms its run of covered columns (rows)
// in each group of 32 as a row of bits, and a warp transpose turns the 32 rows
// into the group's 32 column (row) words.  No atomics: every word has one writer.
__device__ __forceinline__ void build_masks(const int4 *__restrict__ rect, int q0, const SlabWork &s, int ntx) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // readers of the previous pass' words are done
    const int p = q0 + warp * 32 + lane;
    int4 r = make_int4(0, 0, -1, -1);
    if (p < s.p1) r = rect[p];
    for (int c0 = 0; c0 < ntx; c0 += 32) {
        const uint32_t word = transpose32(run_bits(r.x, r.z, c0), lane);
        if (c0 + lane < ntx) s.colw[(c0 + lane) * s.nw + warp] = word;
    }
    for (int y0 = 0; y0 < s.rows; y0 += 32) {
        const uint32_t word = transpose32(run_bits(r.y, r.w, s.sy0 + y0), lane);
        if (y0 + lane < s.rows) s.roww[(y0 + lane) * s.nw + warp] = word;
    }
    __syncthreads();
}

// Number of the pass' primitives overlapping slab tile t (nw is a multiple of 4,
// the word arrays 16-byte aligned).
__device__ __forceinline__ int tile_count(const SlabWork &s, int tx, int ty) {
    const uint4 *cw = reinterpret_cast<const uint4 *>(s.colw + tx * s.nw);
    const uint4 *rw = reinterpret_cast<const uint4 *>(s.roww + ty * s.nw);
    int n = 0;
    for (int i = 0; i < (s.nw >> 2); ++i) {
        const uint4 a = cw[i], b = rw[i];
        n += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
    }
    return n;
}

__global__ void k_count(const int4 *__restrict__ rect, const CanvasDesc *__restrict__ cv,
                        int32_t n_canvas, int32_t *__restrict__ hist) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint32_t smem[];
    const CanvasDesc d = cv[find_canvas_by(cv, n_canvas, blockIdx.x, 1)];
    SlabWork s;
    if (!slab_work(d, smem, s)) return;
    int32_t *row = hist + d.hist_base + (int64_t)s.local * s.ntiles + s.sy0 * d.ntx;
    for (int q0 = s.p0; q0 < s.p1; q0 += blockDim.x) {
        build_masks(rect, q0, s, d.ntx);
        // (tx, ty) of tile t, advanced by (blockDim % ntx, blockDim / ntx) per step
        const int dtx = (int)blockDim.x % d.ntx, dty = (int)blockDim.x / d.ntx;
        int tx = (int)threadIdx.x % d.ntx, ty = (int)threadIdx.x / d.ntx;
        for (int t = threadIdx.x; t < s.slab_tiles; t += blockDim.x) {
            row[t] = (q0 == s.p0 ? 0 : row[t]) + tile_count(s, tx, ty);
            tx += dtx;
            ty += dty;
            if (tx >= d.ntx) tx -= d.ntx, ++ty;
        }
    }
}

// Per tile: exclusive scan of the chunk counts down the tile's column.  A CTA covers
// 32 tiles (x) with 8 groups (y) that each scan one eighth of the chunks, so the
// dependent chain per thread is an eighth of the column.
__global__ void k_colscan(const CanvasDesc *__restrict__ cv, int32_t n_canvas, int32_t n_tiles,
                          int32_t *__restrict__ hist, int64_t *__restrict__ tile_cnt) {
    pdl_wait();
    pdl_trigger();
    __shared__ int32_t part[8][33];
    const int t = blockIdx.x * 32 + threadIdx.x;
    const int g = threadIdx.y;
    int32_t run = 0;
    int ntiles = 0, k0 = 0, k1 = 0;
    int32_t *col = nullptr;
    if (t < n_tiles) {
        const CanvasDesc d = cv[find_canvas_by(cv, n_canvas, t, 2)];
        ntiles = d.ntx * d.nty;
        const int per = (d.n_chunks + 7) / 8;
        k0 = min(g * per, d.n_chunks);
        k1 = min(k0 + per, d.n_chunks);
        col = hist + d.hist_base + (t - d.tile_base);
        for (int k = k0; k < k1; ++k) run += col[(int64_t)k * ntiles];
    }
    part[g][threadIdx.x] = run;
    __syncthreads();
    if (t < n_tiles) {
        int32_t base = 0;
        for (int h = 0; h < g; ++h) base += part[h][threadIdx.x];
        for (int k = k0; k < k1; ++k) {
            const int32_t v = col[(int64_t)k * ntiles];
            col[(int64_t)k * ntiles] = base;
            base += v;
        }
        if (g == 7) tile_cnt[t] = base;
    }
}

// Longest-list-first ordering key of a tile: 0 for the longest lists ... 63 for empty
// (power-of-two buckets of the list length).
__device__ __forceinline__ int len_bucket(int64_t len) {
    return len <= 0 ? 63 : 62 - (63 - __clzll((unsigned long long)len));
}

// Exclusive scan of n tile counts in place (single CTA of 1024 threads), writes
// off[n] = K and the capacity verdict.  With `order` non-null it then lists the tiles
// longest list first (a counting sort on len_bucket; ties in any order) for the
// persistent compositors.
__global__ void __launch_bounds__(1024) k_tilescan(int64_t *__restrict__ off, int32_t n,
                                                   int64_t cap, DevStatus *status, int32_t *__restrict__ order,
                                                   int32_t reset_fwd) {
    pdl_wait();
    pdl_trigger();
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    __shared__ int32_t bucket[64];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    if (tid < 64) bucket[tid] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024 * 4) {
        int64_t v[4];
        int64_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = base + tid * 4 + k;
            v[k] = i < n ? off[i] : 0;
            s += v[k];
            if (order && i < n) atomicAdd(&bucket[len_bucket(v[k])], 1);
        }
        int64_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = warp_sums[lane];
            int64_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_sums[lane] = wi - w;  // exclusive warp offsets
        }
        __syncthreads();
        int64_t run = carry + warp_sums[warp] + incl - s;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = base + tid * 4 + k;
            if (i < n) off[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) carry = run;
        __syncthreads();
    }
    if (tid == 0) {
        const int64_t K = carry;
        off[n] = K;
        if (reset_fwd) {   // the forward's status group, for a forward launched as a dependent
            status->pairs_eval_fwd = 0;
            status->pairs_contrib = 0;
            status->warp_steps_fwd = 0;
            status->survivors_fwd = 0;
            status->queue_fwd = 0u;
            status->pad_fwd = 0u;
        }
        status->pairs_required = K;
        status->lists_valid = K <= cap ? 1 : 0;
        if (K > cap) status->code = (int32_t)DBMP_ERR_CAPACITY;
    }
    if (!order) return;
    if (warp == 0) {   // bucket counts -> exclusive cursors (64 buckets, two per lane)
        const int c0 = bucket[2 * lane], c1 = bucket[2 * lane + 1];
        int incl = c0 + c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        bucket[2 * lane] = incl - c0 - c1;
        bucket[2 * lane + 1] = incl - c1;
    }
    __syncthreads();   // also orders the offsets written above before the reads below
    for (int i = tid; i < n; i += 1024) {
        const int64_t len = (i + 1 < n ? off[i + 1] : carry) - off[i];
        order[atomicAdd(&bucket[len_bucket(len)], 1)] = i;
    }
}

// Writes the entries of one (chunk, slab), one warp per tile: lane l owns the nw
// consecutive bits [l nw, (l + 1) nw) of the tile's 32 nw-bit mask (primitives
// q0 + l nw + j), a warp scan of the lanes' bit counts places them, and the run of
// the tile's entries from this pass is written contiguously at
//   tile_off[t] + (entries of earlier chunks) + (entries of earlier passes),
// so each list comes out in index (front-to-back) order.
__global__ void k_scatter(const int4 *__restrict__ rect, const CanvasDesc *__restrict__ cv,
                          int32_t n_canvas, const int32_t *__restrict__ hist,
                          const int64_t *__restrict__ tile_off, int32_t *__restrict__ list,
                          const DevStatus *status) {
    pdl_wait();
    extern __shared__ __align__(16) uint32_t smem[];
    if (status->lists_valid == 0) return;
    const CanvasDesc d = cv[find_canvas_by(cv, n_canvas, blockIdx.x, 1)];
    SlabWork s;
    if (!slab_work(d, smem, s)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *done = reinterpret_cast<int32_t *>(s.roww + s.rows * s.nw);   // entries of earlier passes
    const int32_t *row = hist + d.hist_base + (int64_t)s.local * s.ntiles + s.sy0 * d.ntx;
    const int64_t *toff = tile_off + d.tile_base + s.sy0 * d.ntx;
    const int bit0 = lane * s.nw;              // first bit of this lane
    const int wi = bit0 >> 5, sh = bit0 & 31;  // its word and offset (nw divides 32)
    const uint32_t keep = s.nw == 32 ? 0xffffffffu : ((1u << s.nw) - 1u);
    for (int q0 = s.p0; q0 < s.p1; q0 += blockDim.x) {
        build_masks(rect, q0, s, d.ntx);
        const bool first = q0 == s.p0, last = q0 + (int)blockDim.x >= s.p1;
        // lane l fetches the list base (tile offset + earlier chunks) of the warp's
        // tile 32 i + l ahead of time; tile i takes it from lane i % 32
        int64_t base_ahead = 0;
        // (tx, ty) of tile t, advanced by (nw % ntx, nw / ntx) per step without divisions
        const int dtx = s.nw % d.ntx, dty = s.nw / d.ntx;
        int tx = warp % d.ntx, ty = warp / d.ntx;
        for (int t = warp, it = 0; t < s.slab_tiles; t += s.nw, ++it) {
            if (it > 0) {
                tx += dtx;
                ty += dty;
                if (tx >= d.ntx) tx -= d.ntx, ++ty;
            }
            if ((it & 31) == 0) {
                const int tl = t + lane * s.nw;
                base_ahead = tl < s.slab_tiles ? toff[tl] + row[tl] : 0;
            }
            const int64_t tile_base = __shfl_sync(0xffffffffu, base_ahead, it & 31);
            uint32_t v = (s.colw[tx * s.nw + wi] & s.roww[ty * s.nw + wi]) >> sh & keep;
            const int c = __popc(v);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) {
                if (first && !last && lane == 0) done[t] = 0;
                continue;
            }
            const int prev = first ? 0 : done[t];
            int64_t pos = tile_base + prev + (incl - c);
            const int pbase = q0 + bit0;
            while (v) {
                const int j = __ffs(v) - 1;
                if (DBMP_CHECKED && (pos < 0 || pos >= status->pairs_required))
                    flag_bad(const_cast<DevStatus *>(status), BAD_LIST_WRITE, pos);
                else
                    list[pos] = pbase + j;
                ++pos;
                v &= v - 1u;
            }
            if (!last && lane == 0) done[t] = prev + total;
        }
    }
}


// ---- scaling statistics of a binning (Sec. S4) ----
// st: [0] listed primitives, [1] sum tau, [2] max tau, [3] max d, [4] tiles,
// [5] empty tiles, [8 + b] tau histogram, [40 + b] d histogram, [72 + b] footprint
// histogram (b = 0..31, see DbmpBinStats).
__global__ void k_stats_prims(const int4 *__restrict__ rect, const float *__restrict__ params,
                              const CanvasDesc *__restrict__ cv, int32_t n_canvas, int32_t N, int32_t Hb, int32_t Wb,
                              unsigned long long *st) {
    __shared__ unsigned long long h[64];
    __shared__ unsigned long long listed, pairs, tmax;
    if (threadIdx.x < 64) h[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) listed = pairs = tmax = 0ull;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int4 r = rect[i];
        if (r.z < r.x || r.w < r.y) continue;
        const unsigned long long tau = (unsigned long long)(r.z - r.x + 1) * (unsigned long long)(r.w - r.y + 1);
        atomicAdd(&listed, 1ull);
        atomicAdd(&pairs, tau);
        atomicMax(&tmax, tau);
        atomicAdd(&h[63 - __clzll(tau)], 1ull);
        float hx, hy;
        const float *p = params + 8 * (int64_t)i;
        spec_halfext(p[2], p[3], Hb, Wb, hx, hy);
        const double area = __dmul_rn(__dadd_rn(__dmul_rn(2.0, (double)hx), 2.0),
                                      __dadd_rn(__dmul_rn(2.0, (double)hy), 2.0));
        const CanvasDesc d = cv[find_canvas_by(cv, n_canvas, i, 0)];
        int e;
        frexp(__ddiv_rn(area, (double)d.H * (double)d.W), &e);   // ratio in [2^(e-1), 2^e)
        atomicAdd(&h[32 + min(31, max(0, -e))], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        if (h[threadIdx.x]) atomicAdd(&st[8 + threadIdx.x], h[threadIdx.x]);
        if (h[32 + threadIdx.x]) atomicAdd(&st[72 + threadIdx.x], h[32 + threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&st[0], listed);
        atomicAdd(&st[1], pairs);
        atomicMax(&st[2], tmax);
    }
}

__global__ void k_stats_tiles(const int64_t *__restrict__ off, int32_t n, unsigned long long *st) {
    __shared__ unsigned long long h[32];
    __shared__ unsigned long long empty, dmax;
    if (threadIdx.x < 32) h[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) empty = dmax = 0ull;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const unsigned long long d = (unsigned long long)(off[t + 1] - off[t]);
        if (d == 0) {
            atomicAdd(&empty, 1ull);
            continue;
        }
        atomicMax(&dmax, d);
        atomicAdd(&h[63 - __clzll(d)], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&st[40 + threadIdx.x], h[threadIdx.x]);
    if (threadIdx.x == 0) {
        atomicAdd(&st[5], empty);
        atomicMax(&st[3], dmax);
        if (blockIdx.x == 0) atomicAdd(&st[4], (unsigned long long)n);
    }
}

}  // namespace

cudaError_t launch_bin_stats(const BinBuffers &b, const float *params, int32_t Hb, int32_t Wb,
                             unsigned long long *st, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(unsigned long long) * kBinStatsWords, s);
    if (e != cudaSuccess) return e;
    if (b.N > 0)
        k_stats_prims<<<min(1216, (b.N + 255) / 256), 256, 0, s>>>(b.rect, params, b.canvas, b.n_canvas, b.N, Hb,
                                                                   Wb, st);
    if (b.n_tiles > 0) k_stats_tiles<<<min(1216, (b.n_tiles + 255) / 256), 256, 0, s>>>(b.tile_off, b.n_tiles, st);
    return cudaGetLastError();
}

cudaError_t init_bin_kernels(int32_t) {
    cudaError_t e = cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSmemCap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSmemCap);
    return e;
}

cudaError_t launch_bin(const BinBuffers &b, const float *params, const int32_t *bitmap_id,
                       const AtlasView &atlas, float alpha_max, int32_t tile, cudaStream_t st, bool reset_fwd) {
    if (b.N > 0) {
        k_prep<<<(b.N + 255) / 256, 256, 0, st>>>(params, bitmap_id, b.canvas, b.n_canvas, b.N, atlas,
                                                   alpha_max, tile, b.rec, b.rect, b.status);
    }
    const int chunk_threads = bin_threads(b.chunk_log2);
    const dim3 grid_cs(b.n_chunks, b.max_slabs);
    if (b.n_chunks > 0) {
        cudaError_t e = launch_pdl(k_count, grid_cs, dim3(chunk_threads), b.smem_count, st, b.rect, b.canvas,
                                   b.n_canvas, b.hist);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_pdl(k_colscan, dim3((b.n_tiles + 31) / 32), dim3(32, 8), 0, st, b.canvas, b.n_canvas,
                               b.n_tiles, b.hist, b.tile_off);
    if (e == cudaSuccess)
        e = launch_pdl(k_tilescan, dim3(1), dim3(1024), 0, st, b.tile_off, b.n_tiles, b.cap, b.status,
                       b.tile_order, (int32_t)(reset_fwd ? 1 : 0));
    if (e == cudaSuccess && b.n_chunks > 0)
        e = launch_pdl(k_scatter, grid_cs, dim3(chunk_threads), b.smem_scatter, st, b.rect, b.canvas, b.n_canvas,
                       b.hist, b.tile_off, b.list, b.status);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dbmp
