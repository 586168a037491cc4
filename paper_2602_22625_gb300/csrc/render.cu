// Forward and backward compositors (Eqs. 1-5, 8; Algorithm 1; Eq. 6, Eqs. S4-S5).
//
// Work decomposition: a tile of TILE x TILE pixels is split into regions of
// 32 * PPT pixels (RW = min(TILE, 16) columns, 32 * PPT / RW rows); one warp
// composites one region, each lane owning PPT pixels of one column.  Warps are independent
// workers: each pulls (tile, region) items from a global atomic queue (tiles in
// longest-list-first order when the binning produced one), gathers the tile's
// primitive records into registers one batch ahead, keeps those whose bitmap is
// non-empty over the region in its own shared-memory slice, walks them, and stops
// as soon as all of its own pixels are saturated (T < T_stop).  There is no
// CTA-wide barrier, so a region that saturates early frees its warp for the next
// item instead of idling until the slowest pixel of the tile is done.
//
// Bitmaps are read through the texture path: one gather fetches the four taps of a
// bilinear sample from the stacked texel plane.  Every pixel runs the same
// straight-line blend for every record (a pixel that does not composite it has
// M = 0, which makes each update an exact no-op).  The forward keeps no per-layer
// state: it writes T_final and the list position of the last contributing layer;
// the backward walks each region's list back to front from the region's largest
// n_last, recovering T_k = T_{k+1} / (1 - alpha_k) with exactly the arithmetic the
// forward used (col_xf, tap_issue, tap_M), reduces the eight per-primitive sums
// across the warp with shuffles and adds them with one atomic per primitive per
// warp.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr float kTFloor = 7.88860905e-31f;  // 2^-100: layers behind are never composited
constexpr int kWarpsPerBlock = 4;

// Resident CTAs per SM each compositor instantiation is compiled for (register
// budget 65536 / (128 x blocks)).  Both kernels hide the latency of their tap
// loads with warps, so occupancy beats registers; these are the largest counts
// at which ptxas spills at most a few words.
constexpr int fwd_blocks(int ppt, int batch) { return ppt == 4 ? 5 : (ppt == 2 && batch == 64 ? 7 : 8); }
constexpr int bwd_blocks(int ppt, int batch) {
    return ppt == 1 ? (batch == 32 ? 6 : 5) : (ppt == 2 ? (batch == 32 ? 5 : 4) : (batch == 32 ? 4 : 3));
}
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int find_canvas_tile(const CanvasDesc *cv, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cv[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Records of one batch held in registers: lane l holds entries l, l + 32, ...
template <int RPL>
struct Prefetch {
    float4 q0[RPL], q1[RPL], q2[RPL];
    int pos[RPL];              // list positions (survivor record only)
    unsigned bad;              // checked build: bit r set for an out-of-range list entry
};

// Issues the loads of list entries [l0, l0 + n) (lane l: entries l + 32 r).  The
// loads are consumed by the next compaction, so their latency overlaps with the
// compositing of the previous batch.
template <int RPL>
__device__ __forceinline__ void prefetch(Prefetch<RPL> &pf, const RenderArgs &a, int64_t l0, int n, int lane) {
    pf.bad = 0u;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int j = lane + 32 * r;
        if (j < n) {
            int32_t idx = __ldg(a.list + l0 + j);
            if (DBMP_CHECKED && (idx < 0 || idx >= a.n_prims)) {
                flag_bad(a.status, BAD_LIST_ENTRY, l0 + j);
                pf.bad |= 1u << r;
                idx = 0;
            }
            const float4 *p = reinterpret_cast<const float4 *>(a.rec + idx);
            pf.q0[r] = __ldg(p);
            pf.q1[r] = __ldg(p + 1);
            pf.q2[r] = __ldg(p + 2);
        }
    }
}

__device__ __forceinline__ PrimRec as_rec(float4 a, float4 b, float4 c) {
    PrimRec r;
    r.x = a.x; r.y = a.y; r.A = a.z; r.B = a.w;
    r.C = b.x; r.D = b.y; r.a = b.z; r.bmp_row = __float_as_int(b.w);
    r.cr = c.x; r.cg = c.y; r.cb = c.z; r.index = __float_as_int(c.w);
    return r;
}

// Can primitive r be non-zero anywhere in the pixel rectangle [x0, x0+w] x [y0, y0+h]?
// U and V are affine in (x, y), so the rectangle maps to a parallelogram whose
// bounding box, widened by one texel (plus the bilinear neighbour), contains every
// tap any of its pixels reads; the bitmap's summed-area table of non-zero texels
// says whether that box holds a non-zero texel.  Never false for a primitive that
// is non-zero at one of the pixels, so culling with it changes no result.
// The bounds carry fp32 rounding errors of a few 2^-24 (|A| (|dx| + w) + |B| (|dy| + h))
// texels (likewise for V).  The region lies in a tile the primitive's box reaches, so
// |A dx| is at most about 2 kw + |A| x (tile + margin), and while |A| + |B| + |C| + |D|
// <= 2^12 the errors stay far below the one texel by which the box is widened.  A larger
// transform (a half-extent below a few hundredths of a pixel) can lose the bitmap's
// offset kw to cancellation in U0 + A w, so such a primitive is never culled.
__device__ __forceinline__ bool region_hits(const PrimRec &r, const AtlasView &at, float x0, float y0,
                                            float w, float h, float kw, float kv) {
    if (fabsf(r.A) + fabsf(r.B) + fabsf(r.C) + fabsf(r.D) > 4096.0f) return true;
    const float dx = x0 - r.x, dy = y0 - r.y;
    const float U0 = fmaf(r.A, dx, r.B * dy) + kw;
    const float V0 = fmaf(r.C, dx, r.D * dy) + kv;
    const float aw = r.A * w, bh = r.B * h, cw = r.C * w, dh = r.D * h;
    const float umin = U0 + fminf(aw, 0.0f) + fminf(bh, 0.0f);
    const float umax = U0 + fmaxf(aw, 0.0f) + fmaxf(bh, 0.0f);
    const float vmin = V0 + fminf(cw, 0.0f) + fminf(dh, 0.0f);
    const float vmax = V0 + fmaxf(dh, 0.0f) + fmaxf(cw, 0.0f);
    const float Wm = (float)(at.Wb - 1), Hm = (float)(at.Hb - 1);
    // texels [floor(umin) - 1, floor(umax) + 2] x [floor(vmin) - 1, floor(vmax) + 2]
    const float fu0 = floorf(umin) - 1.0f, fu1 = floorf(umax) + 2.0f;
    const float fv0 = floorf(vmin) - 1.0f, fv1 = floorf(vmax) + 2.0f;
    if (!(fu1 >= 0.0f && fv1 >= 0.0f && fu0 <= Wm && fv0 <= Hm)) return false;
    const int u0 = (int)fmaxf(fu0, 0.0f), u1 = (int)fminf(fu1, Wm);
    const int v0 = (int)fmaxf(fv0, 0.0f), v1 = (int)fminf(fv1, Hm);
    const int Ws = at.Wb + 1;
    const int32_t *S = at.sat + r.bmp_row * Ws;
    // L2-only loads: a region's four corners are rarely read again from this SM
    const int32_t n = __ldcg(S + (v1 + 1) * Ws + u1 + 1) - __ldcg(S + v0 * Ws + u1 + 1) -
                      __ldcg(S + (v1 + 1) * Ws + u0) + __ldcg(S + v0 * Ws + u0);
    return n > 0;
}

// Tests the prefetched records of list entries [e0, e0 + n) against the warp's
// region and writes the survivors, in list order, to sh[0 .. m) with their list
// positions in pos[]; returns m (same on every lane).
template <int RPL>
__device__ __forceinline__ int compact(const Prefetch<RPL> &pf, int e0, int n, PrimRec *sh, int *pos,
                                       const RenderArgs &a, float x0, float y0, float w, float h,
                                       float kw, float kv, int lane) {
    int base = 0;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int j = lane + 32 * r;
        bool keep = false;
        PrimRec rc;
        if (j < n) {
            rc = as_rec(pf.q0[r], pf.q1[r], pf.q2[r]);
            bool ok = !((pf.bad >> r) & 1u);
            if (DBMP_CHECKED && ok) {
                const int stride = a.atlas.Hb + 1;
                if (rc.bmp_row < 0 || rc.bmp_row > (a.atlas.n_bmp - 1) * stride || rc.bmp_row % stride != 0) {
                    flag_bad(a.status, BAD_BITMAP_ROW, rc.index);
                    ok = false;
                }
            }
            keep = ok && region_hits(rc, a.atlas, x0, y0, w, h, kw, kv);
        }
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) {
            const int slot = base + __popc(m & lt);
            float4 *d = reinterpret_cast<float4 *>(sh + slot);
            d[0] = pf.q0[r];
            d[1] = pf.q1[r];
            d[2] = pf.q2[r];
            pos[slot] = e0 + j;
        }
        base += __popc(m);
    }
    __syncwarp();
    return base;
}

// Issues the loads of survivor-record entries [e0, e0 + n) and of their primitives'
// records (lane l: entries l + 32 r).
template <int RPL>
__device__ __forceinline__ void prefetch_rec(Prefetch<RPL> &pf, const RenderArgs &a, int64_t e0, int n, int lane) {
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int j = lane + 32 * r;
        if (j < n) {
            const int2 e = __ldg(a.surv + e0 + j);
            pf.pos[r] = e.y;
            const float4 *p = reinterpret_cast<const float4 *>(a.rec + e.x);
            pf.q0[r] = __ldg(p);
            pf.q1[r] = __ldg(p + 1);
            pf.q2[r] = __ldg(p + 2);
        }
    }
}

// Writes n prefetched survivor records to sh[0 .. n) with their list positions and
// returns how many of them lie at list positions <= limit: a batch's positions
// increase, so those are the first ones (same on every lane).
template <int RPL>
__device__ __forceinline__ int place(const Prefetch<RPL> &pf, int n, PrimRec *sh, int *pos, int limit, int lane) {
    int m = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int j = lane + 32 * r;
        if (j < n) {
            float4 *d = reinterpret_cast<float4 *>(sh + j);
            d[0] = pf.q0[r];
            d[1] = pf.q1[r];
            d[2] = pf.q2[r];
            pos[j] = pf.pos[r];
        }
        m += __popc(__ballot_sync(FULL, j < n && pf.pos[r] <= limit));
    }
    __syncwarp();
    return m;
}

// Bucket of a region cost c >= 1 for the longest-first order: four per octave,
// 4 floor(log2 c) + the two bits below the leading one (0 .. 127, increasing with c).
__device__ __forceinline__ int cost_bucket(int c) {
    const int e = 31 - __clz(c);
    const int sub = e >= 2 ? (c >> (e - 2)) & 3 : (c << (2 - e)) & 3;
    return 4 * e + sub;
}

struct Region {
    int raw;          // region id: tile * R + region within the tile
    CanvasDesc d;
    int x0, y0;       // canvas coordinates of the region's top-left pixel
    int64_t start;    // first list entry of the tile
    int len;          // tile list length
};

// Width of a warp's region: the tile's width up to 16 pixels, so that a 32-pixel
// tile (shorter lists in total, cheaper binning) still gives each warp a compact
// 16-pixel-wide region to cull against.
__host__ __device__ constexpr int region_w(int tile) { return tile < 16 ? tile : 16; }

template <int TILE, int PPT>
__device__ __forceinline__ Region region_of(const RenderArgs &a, int item) {
    constexpr int RW = region_w(TILE);            // columns per region
    constexpr int RH = 32 * PPT / RW;             // rows per region
    constexpr int RX = TILE / RW;                 // regions across a tile
    constexpr int R = RX * (TILE / RH);           // regions per tile
    int raw;
    if (a.item_order) {
        raw = a.item_order[item];
    } else {
        const int ti = item / R;
        raw = (a.tile_order ? a.tile_order[ti] : ti) * R + (item - ti * R);
    }
    const int tile_id = raw / R, r = raw - tile_id * R;
    Region g;
    g.raw = raw;
    const int c = find_canvas_tile(a.canvas, a.n_canvas, tile_id);
    g.d = a.canvas[c];
    const int lt = tile_id - g.d.tile_base;
    g.x0 = (lt % g.d.ntx) * TILE + (r % RX) * RW;
    g.y0 = (lt / g.d.ntx) * TILE + (r / RX) * RH;
    g.start = a.tile_off[tile_id];
    g.len = (int)(a.tile_off[tile_id + 1] - g.start);
    if (DBMP_CHECKED) {
        const int64_t K = a.status->pairs_required, end = a.tile_off[tile_id + 1];
        if (g.start < 0 || end < g.start || end > K) {
            flag_bad(a.status, BAD_TILE_RANGE, tile_id);
            g.len = g.start < 0 || g.start > K ? 0 : (int)(min(max(end, g.start), K) - g.start);
        }
    }
    return g;
}

__device__ __forceinline__ float bg_at(const RenderArgs &a, const CanvasDesc &d, int ch, int64_t pix) {
    if (a.bg_mode == DBMP_BG_CONST) return ch == 0 ? a.bg0 : (ch == 1 ? a.bg1 : a.bg2);
    if (a.bg_mode == DBMP_BG_BUFFER) return a.bg_buf[3 * d.pix_base + (int64_t)ch * d.H * d.W + pix];
    return 0.0f;
}

// Work counters of one warp, kept in shared memory rather than registers (the
// compositors are register-limited): per item each lane's counts are summed over
// the warp and lane 0 adds them here; flushed to the status block at exit.
struct WarpStats {
    unsigned long long v[4];
};

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Next work item for this warp (lane 0 pulls, all lanes get it).
__device__ __forceinline__ int next_item(uint32_t *queue, int lane) {
    int it = 0;
    if (lane == 0) it = (int)atomicAdd(queue, 1u);
    return __shfl_sync(FULL, it, 0);
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
// COUNT: also count the contributing pairs (layers with M > 0 composited while
// T >= T_stop) into the status block; a per-pixel increment that costs about a tenth
// of the forward's time, so it is compiled in only when asked for.
template <int TILE, int PPT, int BATCH, bool COUNT>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, fwd_blocks(PPT, BATCH)) k_fwd(RenderArgs a, int32_t n_items) {
    pdl_wait();   // launched as a programmatic dependent of the binning when its status group is reset there
    constexpr int RPL = BATCH / 32;   // records per lane per batch
    constexpr int RW = region_w(TILE);
    constexpr int LROWS = 32 / RW;    // rows covered by the 32 lanes in one pass
    constexpr int RH = LROWS * PPT;   // rows of a region
    __shared__ PrimRec sh_all[kWarpsPerBlock][BATCH];
    __shared__ int pos_all[kWarpsPerBlock][BATCH];
    if (a.status->lists_valid == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    PrimRec *sh = sh_all[warp];
    int *pos = pos_all[warp];
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    const float tstop = fmaxf(a.T_stop, kTFloor);
    __shared__ WarpStats stats_all[kWarpsPerBlock];
    WarpStats &stats = stats_all[warp];   // pairs evaluated, contributing, walked, survivors
    if (lane < 4) stats.v[lane] = 0ull;
    __syncwarp();
    float mse_s = 0.0f, mse_c = 0.0f;     // this lane's compensated sum of (I - I*)^2
    // this warp's segment of the survivor record and its fill
    const int64_t sbase = (int64_t)(blockIdx.x * kWarpsPerBlock + warp) * a.surv_wcap;
    int sfill = 0;

    const int row1 = a.row1 > 0 ? a.row1 : 0x7fffffff;
    for (int item = next_item(&a.status->queue_fwd, lane); item < n_items;
         item = next_item(&a.status->queue_fwd, lane)) {
        const Region g = region_of<TILE, PPT>(a, item);
        if (g.y0 < a.row0 || g.y0 >= row1) {   // outside the row window
            if (lane == 0) {
                if (a.item_cost) {
                    a.item_cost[g.raw] = 1;
                    atomicAdd(a.item_hist, 1);
                }
                if (a.surv) a.surv_tab[g.raw] = make_int4(0, -1, 0, 0);
            }
            continue;
        }
        const int sfirst = sfill;   // the region's first entry in the segment
        bool srec = a.surv != nullptr;
        int tested = 0;             // end of the list range compacted
        const int x = g.x0 + lane % RW;
        const float px = (float)x;
        float py[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
        int last[PPT];
        bool inside[PPT];
        Tap tp[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int y = g.y0 + lane / RW + k * LROWS;
            inside[k] = x < g.d.W && y < g.d.H;
            py[k] = (float)y;
            T[k] = inside[k] ? 1.0f : 0.0f;   // pixels off the canvas never composite
            C0[k] = C1[k] = C2[k] = 0.0f;
            last[k] = -1;
            tp[k].q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        const float rx0 = (float)g.x0, ry0 = (float)g.y0;
        const float rw = (float)(RW - 1), rh = (float)(RH - 1);
        int walked = g.len, sv_it = 0, ct_it = 0;
        if (g.len > 0) {
            Prefetch<RPL> pf;
            prefetch<RPL>(pf, a, g.start, min(BATCH, g.len), lane);
            bool alive = __any_sync(FULL, T[0] >= tstop || (PPT > 1 && T[PPT - 1] >= tstop));
            for (int b0 = 0; b0 < g.len && alive; b0 += BATCH) {
                const int n = min(BATCH, g.len - b0);
                const int m = compact<RPL>(pf, b0, n, sh, pos, a, rx0, ry0, rw, rh, kw, kv, lane);
                sv_it += m;
                tested = b0 + n;
                if (srec) {   // append the batch's survivors to the record
                    if (sfill + m <= a.surv_wcap) {
#pragma unroll
                        for (int r = 0; r < RPL; ++r)
                            if (lane + 32 * r < m)
                                a.surv[sbase + sfill + lane + 32 * r] =
                                    make_int2(sh[lane + 32 * r].index, pos[lane + 32 * r]);
                        sfill += m;
                    } else {
                        srec = false;
                    }
                }
                if (b0 + BATCH < g.len)
                    prefetch<RPL>(pf, a, g.start + b0 + BATCH, min(BATCH, g.len - b0 - BATCH), lane);
                for (int t = 0; t < m; ++t) {
                    const PrimRec r = sh[t];
                    const int j = pos[t];
                    const ColXf cx = col_xf(r, kw, kv, px);
                    if constexpr (PPT % 2 == 0) {
#pragma unroll
                        for (int k = 0; k < PPT; k += 2)
                            tap_issue2(r, cx, a.atlas.tex, Wbf, Hbf, make_float2(py[k], py[k + 1]), T[k] >= tstop,
                                       T[k + 1] >= tstop, tp[k], tp[k + 1]);
                    } else {
#pragma unroll
                        for (int k = 0; k < PPT; ++k)
                            tap_issue(r, cx, a.atlas.tex, Wbf, Hbf, py[k], T[k] >= tstop, tp[k]);
                    }
                    // Branch-free per pixel: a pixel that does not composite this layer
                    // has M = 0, so alpha = 0, q = 1 and every update below is an exact
                    // no-op (T * 1 = T, fma(0, c, C) = C).
                    bool any = false;
                    float M[PPT];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) M[k] = tap_M(tp[k]);
                    if constexpr (PPT % 2 == 0) {
                        // two pixels per packed FP32x2 instruction (lane-wise the same
                        // rounding as the scalar form below)
                        const float2 a2 = make_float2(r.a, r.a), na2 = make_float2(-r.a, -r.a);
                        const float2 one2 = make_float2(1.0f, 1.0f);
                        const float2 cr2 = make_float2(r.cr, r.cr), cg2 = make_float2(r.cg, r.cg),
                                     cb2 = make_float2(r.cb, r.cb);
#pragma unroll
                        for (int k = 0; k < PPT; k += 2) {
                            const float2 M2 = make_float2(M[k], M[k + 1]);
                            float2 T2 = make_float2(T[k], T[k + 1]);
                            const float2 w = __fmul2_rn(T2, __fmul2_rn(a2, M2));
                            T2 = __fmul2_rn(T2, __ffma2_rn(na2, M2, one2));
                            const float2 c0 = __ffma2_rn(w, cr2, make_float2(C0[k], C0[k + 1]));
                            const float2 c1 = __ffma2_rn(w, cg2, make_float2(C1[k], C1[k + 1]));
                            const float2 c2 = __ffma2_rn(w, cb2, make_float2(C2[k], C2[k + 1]));
                            T[k] = T2.x; T[k + 1] = T2.y;
                            C0[k] = c0.x; C0[k + 1] = c0.y;
                            C1[k] = c1.x; C1[k + 1] = c1.y;
                            C2[k] = c2.x; C2[k + 1] = c2.y;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            const float w = __fmul_rn(T[k], __fmul_rn(r.a, M[k]));
                            C0[k] = __fmaf_rn(w, r.cr, C0[k]);
                            C1[k] = __fmaf_rn(w, r.cg, C1[k]);
                            C2[k] = __fmaf_rn(w, r.cb, C2[k]);
                            T[k] = __fmul_rn(T[k], __fmaf_rn(-r.a, M[k], 1.0f));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const bool c = M[k] > 0.0f;
                        last[k] = c ? j : last[k];
                        if (COUNT) ct_it += c ? 1 : 0;
                        any = any || T[k] >= tstop;
                    }
                    if (!__any_sync(FULL, any)) {
                        alive = false;
                        walked = j + 1;
                        break;
                    }
                }
                __syncwarp();
            }
        }
        const int64_t HW = (int64_t)g.d.H * g.d.W;
        int ev_it = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (!inside[k]) continue;
            // a pixel evaluates entries up to its last layer, then finds T < T_stop
            ev_it += T[k] < tstop ? last[k] + 1 : g.len;
            const int64_t pix = (int64_t)py[k] * g.d.W + x;
            float *img = a.image + 3 * g.d.pix_base;
            const float I0 = __fmaf_rn(T[k], bg_at(a, g.d, 0, pix), C0[k]);
            const float I1 = __fmaf_rn(T[k], bg_at(a, g.d, 1, pix), C1[k]);
            const float I2 = __fmaf_rn(T[k], bg_at(a, g.d, 2, pix), C2[k]);
            img[pix] = I0;
            img[HW + pix] = I1;
            img[2 * HW + pix] = I2;
            a.T_final[g.d.pix_base + pix] = T[k];
            a.n_last[g.d.pix_base + pix] = last[k];
            if (a.mse_target) {   // the loss of the pixel (the same arithmetic as k_mse)
                const float *tg = a.mse_target + 3 * g.d.pix_base;
                float *dl = a.mse_dL + 3 * g.d.pix_base;
                const float d0 = I0 - tg[pix], d1 = I1 - tg[HW + pix], d2 = I2 - tg[2 * HW + pix];
                dl[pix] = a.mse_scale * d0;
                dl[HW + pix] = a.mse_scale * d1;
                dl[2 * HW + pix] = a.mse_scale * d2;
                acc_sq(d0, mse_s, mse_c);
                acc_sq(d1, mse_s, mse_c);
                acc_sq(d2, mse_s, mse_c);
            }
        }
        // per item each lane's counts fit 32 bits (<= PPT x list length)
        ev_it = warp_sum(ev_it);
        if (COUNT) ct_it = warp_sum(ct_it);
        if (lane == 0) {
            stats.v[0] += (unsigned)ev_it;
            stats.v[1] += (unsigned)ct_it;
            stats.v[2] += (unsigned)walked;
            stats.v[3] += (unsigned)sv_it;
            if (a.item_cost) {   // the region's cost, for the next pass' order
                const int c = sv_it + 1;
                a.item_cost[g.raw] = c;
                atomicAdd(a.item_hist + cost_bucket(c), 1);
            }
            if (a.surv)
                a.surv_tab[g.raw] = srec ? make_int4((int)(sbase + sfirst), sfill - sfirst, tested, 0)
                                         : make_int4(0, -1, 0, 0);
        }
        if (!srec) sfill = sfirst;   // a region not recorded leaves no entries
    }
    __syncwarp();
    if (a.mse_target) {
        double acc = (double)mse_s + (double)mse_c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0 && acc != 0.0) atomicAdd(a.mse_loss, acc * a.mse_inv_n);
    }
    if (lane == 0) {
        if (stats.v[0]) {
            atomicAdd((unsigned long long *)&a.status->pairs_eval_fwd, stats.v[0]);
            atomicAdd((unsigned long long *)&a.status->pairs_contrib, stats.v[1]);
        }
        if (stats.v[2]) atomicAdd((unsigned long long *)&a.status->warp_steps_fwd, stats.v[2]);
        if (stats.v[3]) atomicAdd((unsigned long long *)&a.status->survivors_fwd, stats.v[3]);
    }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// Sums v[0..7] over the 32 lanes of the warp (transpose reduction: 9 shuffles)
// and adds the eight totals to dst[0..7] (lanes 0, 4, ..., 28 each add one).
__device__ __forceinline__ void warp_reduce8_add(const float v[8], float *dst, int lane) {
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
// re-walk (used only when the last contributing layer was exactly opaque, so that
// dividing by (1 - alpha) = 0 cannot recover it).
__device__ float rewalk_T(const RenderArgs &a, const Region &g, int upto, float px, float py) {
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    float T = 1.0f;
    Tap tp;
    tp.q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int j = 0; j < upto; ++j) {
        const int32_t idx = a.list[g.start + j];
        if (DBMP_CHECKED && (idx < 0 || idx >= a.n_prims)) {
            flag_bad(a.status, BAD_LIST_ENTRY, g.start + j);
            continue;
        }
        const PrimRec r = a.rec[idx];
        tap_issue(r, col_xf(r, kw, kv, px), a.atlas.tex, Wbf, Hbf, py, true, tp);
        T = __fmul_rn(T, __fmaf_rn(-r.a, tap_M(tp), 1.0f));
    }
    return T;
}

template <int TILE, int PPT, int BATCH>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, bwd_blocks(PPT, BATCH)) k_bwd(RenderArgs a, int32_t n_items) {
    pdl_wait();   // launched as a programmatic dependent of the region sort when its status group is reset there
    constexpr int RPL = BATCH / 32;
    constexpr int RW = region_w(TILE);
    constexpr int LROWS = 32 / RW;
    constexpr int RH = LROWS * PPT;
    __shared__ PrimRec sh_all[kWarpsPerBlock][BATCH];
    __shared__ int pos_all[kWarpsPerBlock][BATCH];
    if (a.status->lists_valid == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    PrimRec *sh = sh_all[warp];
    int *pos = pos_all[warp];
    const float kw = 0.5f * (float)(a.atlas.Wb - 1), kv = 0.5f * (float)(a.atlas.Hb - 1);
    const float Wbf = (float)a.atlas.Wb, Hbf = (float)a.atlas.Hb;
    const float rho = kw / kv, irho = kv / kw;
    __shared__ WarpStats stats_all[kWarpsPerBlock];
    WarpStats &stats = stats_all[warp];   // pairs evaluated, -, walked, survivors
    // the region's largest last layer, kept in shared memory: the walk over recorded
    // survivors reads it once per batch, and a register held across the walk costs spills
    __shared__ int last_max_all[kWarpsPerBlock];
    if (lane < 4) stats.v[lane] = 0ull;
    __syncwarp();

    const int row1 = a.row1 > 0 ? a.row1 : 0x7fffffff;
    for (int item = next_item(&a.status->queue_bwd, lane); item < n_items;
         item = next_item(&a.status->queue_bwd, lane)) {
        const Region g = region_of<TILE, PPT>(a, item);
        if (g.y0 < a.row0 || g.y0 >= row1) continue;   // outside the row window
        const int x = g.x0 + lane % RW;
        const float px = (float)x;
        float py[PPT], T[PPT], Y[PPT], g0[PPT], g1[PPT], g2[PPT];
        int last[PPT];
        Tap tp[PPT];
        int my_max = -1, ev_it = 0, sv_it = 0;
        const int64_t HW = (int64_t)g.d.H * g.d.W;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int y = g.y0 + lane / RW + k * LROWS;
            py[k] = (float)y;
            last[k] = -1;
            T[k] = Y[k] = g0[k] = g1[k] = g2[k] = 0.0f;
            tp[k].q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (x < g.d.W && y < g.d.H) {
                const int64_t pix = (int64_t)y * g.d.W + x;
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
                ev_it += last[k] + 1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(FULL, my_max, o));
        ev_it = warp_sum(ev_it);
        if (lane == 0) {
            stats.v[0] += (unsigned)ev_it;
            stats.v[2] += (unsigned)(my_max + 1);
        }
        if (my_max < 0) continue;
        if (lane == 0) last_max_all[warp] = my_max;
        __syncwarp();
        const float rx0 = (float)g.x0, ry0 = (float)g.y0;
        const float rw = (float)(RW - 1), rh = (float)(RH - 1);

        // The forward's survivors of this region, when it recorded them up to beyond
        // every pixel's last layer: the walk then reads them in batches from the back
        // (entries behind the last layer are skipped) and tests nothing.  Otherwise
        // batches [lo, hi) of list positions from the back of the region's walk.
        int4 rec = make_int4(0, -1, 0, 0);
        if (a.surv_use) rec = a.surv_tab[g.raw];
        const bool use_rec = rec.y >= 0 && my_max < rec.z;
        int hi = use_rec ? rec.y : my_max + 1;
        int lo = max(0, hi - BATCH);
        Prefetch<RPL> pf;
        if (use_rec)
            prefetch_rec<RPL>(pf, a, rec.x + lo, hi - lo, lane);
        else
            prefetch<RPL>(pf, a, g.start + lo, hi - lo, lane);
        while (hi > 0) {
            int m;
            if (use_rec) {   // the entries behind every pixel's last layer are left out
                m = place<RPL>(pf, hi - lo, sh, pos, last_max_all[warp], lane);
            } else {
                m = compact<RPL>(pf, lo, hi - lo, sh, pos, a, rx0, ry0, rw, rh, kw, kv, lane);
            }
            sv_it += m;
            const int nlo = max(0, lo - BATCH);
            if (lo > 0) {
                if (use_rec)
                    prefetch_rec<RPL>(pf, a, rec.x + nlo, lo - nlo, lane);
                else
                    prefetch<RPL>(pf, a, g.start + nlo, lo - nlo, lane);
            }
            for (int t = m - 1; t >= 0; --t) {
                const int j = pos[t];
                const PrimRec r = sh[t];
                const ColXf cx = col_xf(r, kw, kv, px);
                if constexpr (PPT % 2 == 0) {
#pragma unroll
                    for (int k = 0; k < PPT; k += 2)
                        tap_issue2<true>(r, cx, a.atlas.tex, Wbf, Hbf, make_float2(py[k], py[k + 1]), j <= last[k],
                                         j <= last[k + 1], tp[k], tp[k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) tap_issue(r, cx, a.atlas.tex, Wbf, Hbf, py[k], j <= last[k], tp[k]);
                }
                // Phase 1: alpha and the recovered transmittance in front of the layer.
                // A pixel that does not composite this layer (behind its last layer,
                // outside the bitmap, zero texels) has M = 0 and keeps T and Y.  The
                // packed form keeps nal = -alpha; q = 1 - a M is rounded once (fma), as
                // in the forward, so T_{k+1} = T_k q is undone by the same q.
                const float2 na2 = make_float2(-r.a, -r.a);
                float M[PPT], nal[PPT], q[PPT], Tk[PPT];
                bool redo = false, any = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) M[k] = tap_M(tp[k]);
                if constexpr (PPT % 2 == 0) {
#pragma unroll
                    for (int k = 0; k < PPT; k += 2) {
                        const float2 M2 = make_float2(M[k], M[k + 1]);
                        const float2 n2 = __fmul2_rn(na2, M2);
                        const float2 q2 = __ffma2_rn(na2, M2, make_float2(1.0f, 1.0f));
                        nal[k] = n2.x; nal[k + 1] = n2.y;
                        q[k] = q2.x; q[k + 1] = q2.y;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        nal[k] = __fmul_rn(-r.a, M[k]);
                        q[k] = __fmaf_rn(-r.a, M[k], 1.0f);
                    }
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    Tk[k] = M[k] > 0.0f ? __fdividef(T[k], q[k]) : T[k];
                    // alpha rounds below 1 only if a M < 1 - 2^-25, and then q > 0
                    redo = redo || nal[k] <= -1.0f;
                    any = any || M[k] > 0.0f;
                }
                // no pixel of the warp composites this layer: T, Y and the sums are unchanged
                if (!__any_sync(FULL, any)) continue;
                if (__any_sync(FULL, redo)) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k)
                        if (nal[k] <= -1.0f) Tk[k] = rewalk_T(a, g, j, px, py[k]);
                }
                // Phase 2: the eight per-primitive sums.  The factor a (opacity) common
                // to the geometric sums is applied once per primitive, and the
                // centring of U, V (Up = U - kw, Vp = V - kv) is undone on the sums:
                //   sum dM dMdU Up  = a (sum dA dMdU U - kw sum dA dMdU), and so on.
                // The packed form accumulates the negated sums (with -dL/dalpha and
                // -T alpha) and applies the sign with the factor -a and in s5..s7.
                float s0, s1, s2, s3u, s3v, s4, s5, s6, s7, ra;
                if constexpr (PPT % 2 == 0) {
                    const float2 ncr = make_float2(-r.cr, -r.cr), ncg = make_float2(-r.cg, -r.cg),
                                 ncb = make_float2(-r.cb, -r.cb);
                    float2 S0, S1, S2, S3u, S3v, S4, S5, S6, S7;
#pragma unroll
                    for (int k = 0; k < PPT; k += 2) {
                        float du0, dv0, du1, dv1;
                        tap_M(tp[k], du0, dv0);
                        tap_M(tp[k + 1], du1, dv1);
                        T[k] = Tk[k];
                        T[k + 1] = Tk[k + 1];
                        const float2 G0 = make_float2(g0[k], g0[k + 1]), G1 = make_float2(g1[k], g1[k + 1]),
                                     G2 = make_float2(g2[k], g2[k + 1]);
                        float2 ngc = __fmul2_rn(G0, ncr);                  // -g . c
                        ngc = __ffma2_rn(G1, ncg, ngc);
                        ngc = __ffma2_rn(G2, ncb, ngc);
                        const float2 Tk2 = make_float2(Tk[k], Tk[k + 1]);
                        const float2 Y2 = make_float2(Y[k], Y[k + 1]);
                        float2 ndA = __fmul2_rn(Tk2, __fadd2_rn(ngc, Y2));  // -dL/dalpha_k
                        ndA.x = M[k] > 0.0f ? ndA.x : 0.0f;
                        ndA.y = M[k + 1] > 0.0f ? ndA.y : 0.0f;
                        const float2 gU = __fmul2_rn(ndA, make_float2(du0, du1));
                        const float2 gV = __fmul2_rn(ndA, make_float2(dv0, dv1));
                        const float2 U2 = make_float2(tp[k].U, tp[k + 1].U), V2 = make_float2(tp[k].V, tp[k + 1].V);
                        const float2 M2 = make_float2(M[k], M[k + 1]);
                        const float2 nal2 = make_float2(nal[k], nal[k + 1]);
                        const float2 nw = __fmul2_rn(Tk2, nal2);            // -T_k alpha_k
                        if (k == 0) {
                            S0 = gU;
                            S1 = gV;
                            S2 = __fmul2_rn(gU, U2);
                            S3u = __fmul2_rn(gU, V2);
                            S3v = __fmul2_rn(gV, U2);
                            S4 = __fmul2_rn(ndA, M2);
                            S5 = __fmul2_rn(G0, nw);
                            S6 = __fmul2_rn(G1, nw);
                            S7 = __fmul2_rn(G2, nw);
                        } else {
                            S0 = __fadd2_rn(S0, gU);
                            S1 = __fadd2_rn(S1, gV);
                            S2 = __ffma2_rn(gU, U2, S2);
                            S3u = __ffma2_rn(gU, V2, S3u);
                            S3v = __ffma2_rn(gV, U2, S3v);
                            S4 = __ffma2_rn(ndA, M2, S4);
                            S5 = __ffma2_rn(G0, nw, S5);
                            S6 = __ffma2_rn(G1, nw, S6);
                            S7 = __ffma2_rn(G2, nw, S7);
                        }
                        S2 = __ffma2_rn(gV, V2, S2);
                        // Y = q Y + alpha (g . c), with alpha (g . c) = (-alpha)(-g . c)
                        const float2 Yn = __ffma2_rn(make_float2(q[k], q[k + 1]), Y2, __fmul2_rn(nal2, ngc));
                        Y[k] = Yn.x;
                        Y[k + 1] = Yn.y;
                    }
                    s0 = -S0.x - S0.y;
                    s1 = -S1.x - S1.y;
                    s2 = -S2.x - S2.y;
                    s3u = -S3u.x - S3u.y;
                    s3v = -S3v.x - S3v.y;
                    s4 = -S4.x - S4.y;
                    s5 = -S5.x - S5.y;
                    s6 = -S6.x - S6.y;
                    s7 = -S7.x - S7.y;
                    ra = -r.a;
                } else {
                    s0 = s1 = s2 = s3u = s3v = s4 = s5 = s6 = s7 = 0.0f;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        float dMdU, dMdV;
                        tap_M(tp[k], dMdU, dMdV);
                        const bool c = M[k] > 0.0f;
                        T[k] = Tk[k];
                        const float al = -nal[k];
                        const float gc = g0[k] * r.cr + g1[k] * r.cg + g2[k] * r.cb;
                        const float dA = c ? Tk[k] * (gc - Y[k]) : 0.0f;   // dL/dalpha_k
                        const float gU = dA * dMdU, gV = dA * dMdV;        // / a
                        s0 += gU;
                        s1 += gV;
                        s2 = fmaf(gU, tp[k].U, s2);
                        s2 = fmaf(gV, tp[k].V, s2);
                        s3u = fmaf(gU, tp[k].V, s3u);
                        s3v = fmaf(gV, tp[k].U, s3v);
                        s4 = fmaf(dA, M[k], s4);                           // / a
                        const float w = Tk[k] * al;
                        s5 = fmaf(g0[k], w, s5);
                        s6 = fmaf(g1[k], w, s6);
                        s7 = fmaf(g2[k], w, s7);
                        Y[k] = fmaf(q[k], Y[k], al * gc);
                    }
                    ra = r.a;
                }
                {
                    float v[8];
                    (void)ra;
                    v[0] = s0;
                    v[1] = s1;
                    v[2] = s2;
                    v[3] = fmaf(rho, s3u, -irho * s3v);
                    v[4] = s4;
                    v[5] = s5;
                    v[6] = s6;
                    v[7] = s7;
                    warp_reduce8_add(v, a.graw + 8 * (int64_t)r.index, lane);
                }
            }
            __syncwarp();
            hi = lo;
            lo = nlo;
        }
        if (lane == 0) stats.v[3] += (unsigned)sv_it;
    }
    __syncwarp();
    if (lane == 0) {
        if (stats.v[0]) atomicAdd((unsigned long long *)&a.status->pairs_eval_bwd, stats.v[0]);
        if (stats.v[2]) atomicAdd((unsigned long long *)&a.status->warp_steps_bwd, stats.v[2]);
        if (stats.v[3]) atomicAdd((unsigned long long *)&a.status->survivors_bwd, stats.v[3]);
    }
}

// Regions sorted by decreasing cost (longest first): a counting sort over the
// forward's cost buckets (four per octave, cost_bucket).  Within a bucket the order is
// whatever the atomics give; any order renders the same pixels.  hist[128..255] (the
// cursors) start at zero.  If the buckets do not count every region (a forward that
// stopped early, e.g. on a tile-list capacity overflow), the order is the identity, so
// that it always holds every region exactly once.  The counts come in two halves used
// by alternate forwards: this kernel clears the other half (next_hist) for the next
// forward, so no separate reset is queued.  Launched as a programmatic dependent of the
// forward, with 256 threads per block.  With reset_bwd set it also resets the backward's
// status group, so that the backward can follow as its programmatic dependent with no
// memset in between.
__global__ void k_item_order(const int32_t *__restrict__ cost, int32_t *__restrict__ hist,
                             int32_t *__restrict__ next_hist, int32_t *__restrict__ order, int32_t n,
                             DevStatus *reset_bwd) {
    pdl_wait();
    pdl_trigger();
    __shared__ int32_t base[128];
    __shared__ int32_t total;
    if (blockIdx.x == 0) next_hist[threadIdx.x] = 0;
    // the backward's status group (counters and work queue), reset for the next backward
    if (reset_bwd && blockIdx.x == 0 && threadIdx.x == 0) {
        reset_bwd->pairs_eval_bwd = 0;
        reset_bwd->warp_steps_bwd = 0;
        reset_bwd->survivors_bwd = 0;
        reset_bwd->queue_bwd = 0u;
        reset_bwd->pad_bwd = 0u;
    }
    if (threadIdx.x < 32) {
        // lane l holds buckets 127 - 4 l ... 124 - 4 l (costliest first): an inclusive
        // scan over the lanes counts the regions of all costlier buckets
        const int l = threadIdx.x;
        int c[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c[k] = hist[127 - 4 * l - k];
            sum += c[k];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, o);
            if (l >= o) incl += u;
        }
        int run = incl - sum;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            base[127 - 4 * l - k] = run;
            run += c[k];
        }
        if (l == 31) total = incl;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (total != n) {
        if (i < n) order[i] = i;
        return;
    }
    // one atomic per bucket per warp: the lanes of a bucket take consecutive slots
    const int b = i < n ? cost_bucket(max(cost[i], 1)) : -1;
    const unsigned same = __match_any_sync(FULL, b);
    const int lead = __ffs(same) - 1;
    const int lane = threadIdx.x & 31;
    int slot = 0;
    if (b >= 0 && lane == lead) slot = atomicAdd(hist + 128 + b, __popc(same));
    slot = __shfl_sync(FULL, slot, lead) + __popc(same & ((1u << lane) - 1u));
    if (b >= 0) order[base[b] + slot] = i;
}

// Per-primitive chain rule from the eight reduced sums to the raw parameters:
//   x: -(A S0 + C S1)    y: -(B S0 + D S1)    s: -S2 / s    theta: S3
//   nu: S4 (1 - sigmoid(nu))    c_j: S_{5+j} chat_j (1 - chat_j)
// The sums are read and then zeroed, so graw is zero again for the next backward.
__global__ void k_finalize(const float *__restrict__ params, const PrimRec *__restrict__ rec,
                           float *__restrict__ graw, float *__restrict__ dparams, int32_t N, float kw, float kv) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const PrimRec r = rec[i];
    float4 *g4 = reinterpret_cast<float4 *>(graw + 8 * (size_t)i);
    const float4 lo = g4[0], hi = g4[1];
    g4[0] = g4[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float a = r.a;
    const float S[8] = {a * lo.x, a * lo.y, a * fmaf(-kv, lo.y, fmaf(-kw, lo.x, lo.z)),
                        a * fmaf(kv, lo.y, fmaf(-kw, lo.x, lo.w)), a * hi.x, hi.y, hi.z, hi.w};
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

// Resident CTAs per SM of each instantiation and the SM count, queried once per
// device (init_render_kernels, with that device current) so that launches inside a
// CUDA-graph capture make no occupancy queries.  Each device's table is filled
// under its own std::call_once, so concurrent first callers do not race.
constexpr int kMaxDevices = 64;
constexpr int kMaxOcc = 64;
struct OccEntry {
    const void *fn;
    int per_sm;
};
struct DeviceKernels {
    int sms;
    int n_occ;
    OccEntry occ[kMaxOcc];
    cudaError_t err;
};
DeviceKernels g_dk[kMaxDevices];
std::once_flag g_dk_once[kMaxDevices];

// The current device's table (nullptr for a device ordinal beyond the table).
const DeviceKernels *device_kernels() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    return &g_dk[dev];
}

int resident_ctas(const DeviceKernels *dk, const void *fn) {
    if (dk)
        for (int i = 0; i < dk->n_occ; ++i)
            if (dk->occ[i].fn == fn) return dk->occ[i].per_sm;
    return 1;
}

int persistent_grid(const void *kernel, int32_t n_items) {
    const DeviceKernels *dk = device_kernels();
    const int sms = dk && dk->sms > 0 ? dk->sms : 1;
    const int full = sms * resident_ctas(dk, kernel);
    const int need = (n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return need < full ? (need > 0 ? need : 1) : full;
}

template <int TILE, int PPT, int BATCH>
void register_occupancy(DeviceKernels &dk) {
    const void *fns[3] = {(const void *)k_fwd<TILE, PPT, BATCH, false>, (const void *)k_fwd<TILE, PPT, BATCH, true>,
                          (const void *)k_bwd<TILE, PPT, BATCH>};
    for (const void *fn : fns) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 32 * kWarpsPerBlock, 0);
        // the smallest shared-memory carve-out that keeps this occupancy, leaving the
        // rest of the SM's on-chip memory to L1 (the texel gathers' cache)
        for (int pct = 0; pct <= 100; pct += 2) {
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            int p2 = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, fn, 32 * kWarpsPerBlock, 0);
            if (p2 >= per) break;
        }
        if (dk.n_occ < kMaxOcc) dk.occ[dk.n_occ++] = OccEntry{fn, per > 0 ? per : 1};
    }
}

template <int TILE, int PPT, int BATCH>
cudaError_t launch_t(const RenderArgs &a, bool fwd, bool pdl, cudaStream_t st) {
    constexpr int R = TILE * TILE / (32 * PPT);   // regions per tile (any region shape)
    const int32_t n_items = a.n_tiles * R;
    if (fwd) {
        const void *fn = a.count_pairs ? (const void *)k_fwd<TILE, PPT, BATCH, true>
                                       : (const void *)k_fwd<TILE, PPT, BATCH, false>;
        const int grid = persistent_grid(fn, n_items);
        RenderArgs b = a;
        if (b.surv) {   // the survivor record's entries, divided among the grid's warps
            const int64_t w = b.surv_cap / ((int64_t)grid * kWarpsPerBlock);
            b.surv_wcap = (int32_t)(w < 0x7fffffff ? w : 0x7fffffff);
            if (b.surv_wcap < 1) b.surv = nullptr;
        }
        if (pdl) {
            const cudaError_t e =
                a.count_pairs ? launch_pdl(k_fwd<TILE, PPT, BATCH, true>, dim3(grid), dim3(32 * kWarpsPerBlock), 0, st, b, n_items)
                              : launch_pdl(k_fwd<TILE, PPT, BATCH, false>, dim3(grid), dim3(32 * kWarpsPerBlock), 0, st, b, n_items);
            if (e != cudaSuccess) return e;
        } else if (a.count_pairs) {
            k_fwd<TILE, PPT, BATCH, true><<<grid, 32 * kWarpsPerBlock, 0, st>>>(b, n_items);
        } else {
            k_fwd<TILE, PPT, BATCH, false><<<grid, 32 * kWarpsPerBlock, 0, st>>>(b, n_items);
        }
    } else {
        const int grid = persistent_grid((const void *)k_bwd<TILE, PPT, BATCH>, n_items);
        if (pdl) {
            const cudaError_t e = launch_pdl(k_bwd<TILE, PPT, BATCH>, dim3(grid), dim3(32 * kWarpsPerBlock), 0, st, a, n_items);
            if (e != cudaSuccess) return e;
        } else {
            k_bwd<TILE, PPT, BATCH><<<grid, 32 * kWarpsPerBlock, 0, st>>>(a, n_items);
        }
    }
    return cudaGetLastError();
}

cudaError_t dispatch(const RenderArgs &a, const RenderCfg &cfg, bool fwd, bool pdl, cudaStream_t st) {
#define DBMP_CASE(T, P, B) \
    if (cfg.tile == T && cfg.ppt == P && cfg.batch == B) return launch_t<T, P, B>(a, fwd, pdl, st);
    DBMP_CASE(8, 1, 32) DBMP_CASE(8, 2, 32) DBMP_CASE(8, 1, 64) DBMP_CASE(8, 2, 64)
    DBMP_CASE(16, 1, 32) DBMP_CASE(16, 2, 32) DBMP_CASE(16, 4, 32)
    DBMP_CASE(16, 1, 64) DBMP_CASE(16, 2, 64) DBMP_CASE(16, 4, 64)
    DBMP_CASE(32, 1, 32) DBMP_CASE(32, 2, 32) DBMP_CASE(32, 4, 32)
    DBMP_CASE(32, 1, 64) DBMP_CASE(32, 2, 64) DBMP_CASE(32, 4, 64)
#undef DBMP_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t init_render_kernels() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_dk_once[dev], [dev]() {
        DeviceKernels &dk = g_dk[dev];
        dk.n_occ = 0;
        dk.err = cudaDeviceGetAttribute(&dk.sms, cudaDevAttrMultiProcessorCount, dev);
        if (dk.err != cudaSuccess) return;
        register_occupancy<8, 1, 32>(dk); register_occupancy<8, 2, 32>(dk);
        register_occupancy<8, 1, 64>(dk); register_occupancy<8, 2, 64>(dk);
        register_occupancy<16, 1, 32>(dk); register_occupancy<16, 2, 32>(dk); register_occupancy<16, 4, 32>(dk);
        register_occupancy<16, 1, 64>(dk); register_occupancy<16, 2, 64>(dk); register_occupancy<16, 4, 64>(dk);
        register_occupancy<32, 1, 32>(dk); register_occupancy<32, 2, 32>(dk); register_occupancy<32, 4, 32>(dk);
        register_occupancy<32, 1, 64>(dk); register_occupancy<32, 2, 64>(dk); register_occupancy<32, 4, 64>(dk);
        dk.err = cudaGetLastError();
    });
    return g_dk[dev].err;
}

bool render_cfg_supported(const RenderCfg &cfg) {
    const bool tile_ok = cfg.tile == 8 || cfg.tile == 16 || cfg.tile == 32;
    auto ppt_ok = [&](int p) { return p == 1 || p == 2 || (p == 4 && cfg.tile >= 16); };
    return tile_ok && ppt_ok(cfg.ppt) && ppt_ok(cfg.bwd_ppt()) && (cfg.batch == 32 || cfg.batch == 64);
}

// The status block's forward (backward) group, work queue included, must be zero at
// the launch: reset by a memset the caller queues, or by the previous kernel of the
// stream, which the launch then follows as a programmatic dependent (pdl).
cudaError_t launch_fwd(const RenderArgs &a, const RenderCfg &cfg, cudaStream_t st, bool pdl) {
    return dispatch(a, cfg, true, pdl, st);
}

cudaError_t launch_bwd(const RenderArgs &a, const RenderCfg &cfg, cudaStream_t st, bool pdl) {
    RenderCfg b = cfg;
    b.ppt = cfg.bwd_ppt();
    return dispatch(a, b, false, pdl, st);
}

int32_t render_items(const RenderCfg &cfg, int32_t n_tiles, bool bwd) {
    const int ppt = bwd ? cfg.bwd_ppt() : cfg.ppt;
    return n_tiles * (cfg.tile * cfg.tile / (32 * ppt));
}

cudaError_t launch_item_order(const int32_t *cost, int32_t *hist, int32_t *next_hist, int32_t *order,
                              int32_t n_items, DevStatus *reset_bwd, cudaStream_t st) {
    if (n_items > 0) {
        const cudaError_t e = launch_pdl(k_item_order, dim3((n_items + 255) / 256), dim3(256), 0, st, cost, hist,
                                         next_hist, order, n_items, reset_bwd);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const float *params, const PrimRec *rec, float *graw,
                                 float *dparams, int32_t N, float kw, float kv, cudaStream_t st) {
    if (N > 0) {
        const cudaError_t e = launch_pdl(k_finalize, dim3((N + 255) / 256), dim3(256), 0, st, params, rec, graw,
                                         dparams, N, kw, kv);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace dbmp
