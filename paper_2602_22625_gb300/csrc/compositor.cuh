// Definitions the compositor kernels are built from (records, canvases, status block,
// atlas view, launch arguments, the bilinear sample and the small device helpers).
// Included by dbmp_internal.cuh; kept apart from the host-side declarations so that
// the kernels' source is exactly render.cu plus this file.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/dbmp.h"

namespace dbmp {

// Per-primitive record staged in shared memory by the compositors (48 bytes).
// U = A (x - x_i) + B (y - y_i) + kw,  V = C (x - x_i) + D (y - y_i) + kv  (Eqs. 1-2
// folded: A = kw cos/s, B = kw sin/s, C = -kv sin/s, D = kv cos/s, kw = (W_b-1)/2,
// kv = (H_b-1)/2), computed in FP64 and rounded once.
struct __align__(16) PrimRec {
    float x, y, A, B;
    float C, D, a;       // a = alpha_max sigmoid(nu)  (Eq. 3 without M)
    int32_t bmp_row;     // first row of the primitive's bitmap in the texel plane: id x (H_b + 1)
    float cr, cg, cb;    // sigmoid(c)
    int32_t index;       // primitive index (row of params / dparams)
};
static_assert(sizeof(PrimRec) == 48, "PrimRec layout");

// One canvas of a (possibly single-canvas) batch.
struct CanvasDesc {
    int32_t H, W, ntx, nty;
    int32_t tile_base;   // first global tile id of this canvas
    int32_t prim_base;   // first primitive of this canvas
    int32_t N;           // primitives of this canvas
    int32_t chunk_base;  // first global binning chunk of this canvas
    int32_t n_chunks;
    int32_t chunk_log2;  // primitives per binning chunk = 1 << chunk_log2
    int64_t pix_base;    // first pixel of this canvas in concatenated per-pixel maps
    int64_t hist_base;   // offset of this canvas' chunk x tile histogram
    int32_t slab_rows;   // tile rows per binning slab
    int32_t n_slabs;     // ceil(nty / slab_rows)
};

// Device status block (mirrors DbmpDeviceStatus, plus internal flags).
struct DevStatus {
    int32_t code;
    int32_t n_degenerate;
    int64_t pairs_required;
    int32_t lists_valid;    // 1 after a binning that fit its capacity
    int32_t pad;
    // first out-of-range index an index-checked build met (BadIndexKind, 0: none)
    int32_t bad_kind;
    int32_t pad_bad;
    int64_t bad_index;
    // forward counters and work queue, reset together before each forward
    int64_t pairs_eval_fwd;
    int64_t pairs_contrib;  // (pixel, layer) pairs with alpha > 0 composited by the last fwd (when counted)
    int64_t warp_steps_fwd; // list entries walked, summed over warps (last fwd)
    int64_t survivors_fwd;  // records that passed the region test (last fwd)
    uint32_t queue_fwd;     // persistent-kernel work counter
    uint32_t pad_fwd;
    // backward counters and work queue, reset together before each backward
    int64_t pairs_eval_bwd;
    int64_t warp_steps_bwd; // same for the last bwd
    int64_t survivors_bwd;  // same for the last bwd
    uint32_t queue_bwd;
    uint32_t pad_bwd;
};
// Byte lengths of the two groups, each reset by one memset from its first field.
constexpr size_t kFwdGroupBytes = offsetof(DevStatus, pairs_eval_bwd) - offsetof(DevStatus, pairs_eval_fwd);
constexpr size_t kBwdGroupBytes = sizeof(DevStatus) - offsetof(DevStatus, pairs_eval_bwd);
static_assert(kFwdGroupBytes == 4 * sizeof(int64_t) + 2 * sizeof(uint32_t), "forward group layout");
static_assert(kBwdGroupBytes == 3 * sizeof(int64_t) + 2 * sizeof(uint32_t), "backward group layout");

// Index checks, compiled into the checked build of the library only (DBMP_CHECKED=1):
// a kernel that meets a tile range, a list entry, a bitmap row or a list position
// outside its valid range records the first one in the status block and skips the
// access (the tile counts as empty, the entry as culled) instead of trapping, so the
// context stays usable and the status says what was wrong.  The kinds are the ABI's
// DBMP_BAD_* values.
#ifndef DBMP_CHECKED
#define DBMP_CHECKED 0
#endif
enum BadIndexKind : int32_t {
    BAD_NONE = 0,
    BAD_TILE_RANGE = 1,   // tile offsets outside [0, sum_t d_t]: index = tile id
    BAD_LIST_ENTRY = 2,   // primitive index outside [0, N): index = list position
    BAD_BITMAP_ROW = 3,   // record's bitmap row not the start of a bitmap: index = primitive
    BAD_LIST_WRITE = 4,   // binning write outside [0, sum_t d_t): index = list position
};

__device__ __forceinline__ void flag_bad(DevStatus *st, int32_t kind, int64_t index) {
    if (atomicCAS(&st->bad_kind, 0, kind) == 0) st->bad_index = index;
}

// The bitmap atlas as the kernels see it.  The texels of all bitmaps are stacked in
// one pitch-linear float plane, bitmap b in rows b (H_b + 1) .. b (H_b + 1) + H_b - 1
// followed by one zero row, read through a 2-D texture object (border address mode,
// border value 0; point sampling, unnormalised coordinates).  A bilinear sample
// fetches its four taps with one gather, so taps outside the bitmap read 0 (zero
// padding, Sec. S1.1) from the border or the zero row.
struct AtlasView {
    cudaTextureObject_t tex;  // texel plane
    const int32_t *sat;       // [n_bmp][H_b+1][W_b+1] summed-area table of (texel > 0)
    int32_t n_bmp, Hb, Wb;
    const int4 *nzbox;        // [n_bmp] first/last column and row holding a texel > 0:
                              // (u0, u1, v0, v1); (W_b, -1, H_b, -1) for an all-zero bitmap
};

// Tile size, records per warp staging batch, pixels per lane of the forward and
// of the backward (0: same as the forward).
struct RenderCfg {
    int32_t tile;
    int32_t batch;
    int32_t ppt;
    int32_t ppt_bwd;
    int32_t bwd_ppt() const { return ppt_bwd ? ppt_bwd : ppt; }
};

// ---------------------------------------------------------------------------
// The one bilinear sample every compositor uses (Eq. 2, Eqs. S1-S3).  Every
// operation is explicitly rounded (no contraction decided by the compiler), so
// the forward, the backward and the backward's re-walk compute bit-identical M
// and alpha for the same (pixel, primitive).
//
// The transform is split by what it depends on.  Its column part depends on the
// primitive and the pixel's x only, so a lane that owns several pixels of one
// column evaluates it once per primitive:
//     dx = px - x,   au = A dx + kw,   cv = C dx + kv            (col_xf)
// and each pixel adds its row part:
//     dy = py - y,   U = B dy + au,    V = D dy + cv             (tap_issue)
// (U, V) outside (-1, W_b) x (-1, H_b) reads only zero taps; there, and for a
// pixel that no longer composites, no load is issued and tap_M returns 0 (the
// backward's tap_issue2<true> issues the load when only U is outside: the texture's
// border then supplies the zero taps, and M is 0 all the same).
// ---------------------------------------------------------------------------
struct ColXf {
    float au, cv;              // A dx + kw, C dx + kv
    float row;                 // bmp_row + 1: gather y of the bitmap's row -1
};

__device__ __forceinline__ ColXf col_xf(const PrimRec &r, float kw, float kv, float px) {
    const float dx = __fsub_rn(px, r.x);
    ColXf c;
    c.au = __fmaf_rn(r.A, dx, kw);
    c.cv = __fmaf_rn(r.C, dx, kv);
    c.row = (float)(r.bmp_row + 1);
    return c;
}

// The per-pixel half of a sample.  tap_issue transforms the pixel, tests the range
// and issues the texture gather of the four taps; tap_M blends.  Splitting them lets
// a lane have the gathers of all its pixels in flight before it blends.  q keeps its
// previous contents when no gather is issued (ok false); tap_M then returns 0
// without reading it, and every other quantity computed from q stays finite.
struct Tap {
    float4 q;                  // (p00, p01, p10, p11)
    float U, V, wu, wv;        // bitmap coordinates and their fractional parts
    bool ok;
};

__device__ __forceinline__ void tap_issue(const PrimRec &r, const ColXf &c, cudaTextureObject_t tex, float Wbf,
                                          float Hbf, float py, bool live, Tap &t) {
    const float dy = __fsub_rn(py, r.y);
    t.U = __fmaf_rn(r.B, dy, c.au);
    t.V = __fmaf_rn(r.D, dy, c.cv);
    t.ok = live && t.U >= -1.0f && t.U < Wbf && t.V >= -1.0f && t.V < Hbf;
    const float fu = floorf(t.U), fv = floorf(t.V);
    t.wu = __fsub_rn(t.U, fu);
    t.wv = __fsub_rn(t.V, fv);
    if (t.ok) {
        // Texel centres sit at half-integers, so a gather at (fu + 1, row + fv) has
        // its 2 x 2 footprint at texels fu, fu + 1 of plane rows bmp_row + fv,
        // bmp_row + fv + 1 with no rounding to decide: exact integers, fu, fv in
        // [-1, W_b-1] x [-1, H_b-1].  Gather order: (u0,v1), (u1,v1), (u1,v0), (u0,v0).
        const float4 g = tex2Dgather<float4>(tex, __fadd_rn(fu, 1.0f), __fadd_rn(fv, c.row), 0);
        t.q = make_float4(g.w, g.z, g.x, g.y);
    }
}

// tap_issue for two pixels of one column (rows py2.x, py2.y), with the transform and
// the fractional parts in packed FP32x2 instructions.  Lane-wise the roundings are
// those of tap_issue: a - b is computed as fma(b, -1, a), which rounds a - b once.
// V_ONLY tests only V's range: for U outside [-1, W_b) the gather's 2 x 2 footprint
// lies in columns < 0 or >= W_b, where the texture's border gives zeros, so M and both
// derivatives are exactly 0 as when no gather is issued (the backward's choice: it
// then issues gathers for pixels beside the bitmap, but tests less).
template <bool V_ONLY = false>
__device__ __forceinline__ void tap_issue2(const PrimRec &r, const ColXf &c, cudaTextureObject_t tex, float Wbf,
                                           float Hbf, float2 py2, bool live0, bool live1, Tap &t0, Tap &t1) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 dy = __ffma2_rn(make_float2(r.y, r.y), m1, py2);
    const float2 U = __ffma2_rn(make_float2(r.B, r.B), dy, make_float2(c.au, c.au));
    const float2 V = __ffma2_rn(make_float2(r.D, r.D), dy, make_float2(c.cv, c.cv));
    const float2 fu = make_float2(floorf(U.x), floorf(U.y)), fv = make_float2(floorf(V.x), floorf(V.y));
    const float2 wu = __ffma2_rn(fu, m1, U), wv = __ffma2_rn(fv, m1, V);
    t0.U = U.x; t0.V = V.x; t0.wu = wu.x; t0.wv = wv.x;
    t1.U = U.y; t1.V = V.y; t1.wu = wu.y; t1.wv = wv.y;
    if (V_ONLY) {
        t0.ok = live0 && V.x >= -1.0f && V.x < Hbf;
        t1.ok = live1 && V.y >= -1.0f && V.y < Hbf;
    } else {
        t0.ok = live0 && U.x >= -1.0f && U.x < Wbf && V.x >= -1.0f && V.x < Hbf;
        t1.ok = live1 && U.y >= -1.0f && U.y < Wbf && V.y >= -1.0f && V.y < Hbf;
    }
    if (t0.ok) {
        const float4 g = tex2Dgather<float4>(tex, __fadd_rn(fu.x, 1.0f), __fadd_rn(fv.x, c.row), 0);
        t0.q = make_float4(g.w, g.z, g.x, g.y);
    }
    if (t1.ok) {
        const float4 g = tex2Dgather<float4>(tex, __fadd_rn(fu.y, 1.0f), __fadd_rn(fv.y, c.row), 0);
        t1.q = make_float4(g.w, g.z, g.x, g.y);
    }
}

// Bilinear value M (0 when !ok) and the two tap differences the backward needs:
// dMdU = d0 + wv (d1 - d0), dMdV = m1 - m0.  M >= 0 whenever the texels are.
__device__ __forceinline__ float tap_M(const Tap &t, float &dMdU, float &dMdV) {
    const float d0 = __fsub_rn(t.q.y, t.q.x);          // p01 - p00
    const float d1 = __fsub_rn(t.q.w, t.q.z);          // p11 - p10
    const float m0 = __fmaf_rn(t.wu, d0, t.q.x);
    const float m1 = __fmaf_rn(t.wu, d1, t.q.z);
    dMdV = __fsub_rn(m1, m0);
    dMdU = __fmaf_rn(t.wv, __fsub_rn(d1, d0), d0);
    const float M = __fmaf_rn(t.wv, dMdV, m0);
    return t.ok ? M : 0.0f;
}

__device__ __forceinline__ float tap_M(const Tap &t) {
    float du, dv;
    return tap_M(t, du, dv);
}

// Adds d^2 to the compensated sum (s, c) with error-free transformations (the
// exact product d^2 = p + pe by one FMA, the exact sum s + p = t + se by TwoSum),
// as in Ogita, Rump and Oishi's compensated dot product: s + c carries about twice
// fp32 precision, so the loss needs no FP64 arithmetic per element (FP64 throughput
// is a small fraction of FP32 on this GPU).  Explicitly rounded operations keep the
// compiler from contracting or reassociating the transformations.
__device__ __forceinline__ void acc_sq(float d, float &s, float &c) {
    const float p = __fmul_rn(d, d);
    const float pe = __fmaf_rn(d, d, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(se, pe));
}

// Programmatic dependent launch (PDL).  A kernel launched with launch_pdl may start
// while the previous kernel of the stream is still running; pdl_wait(), its first
// statement, returns once that kernel has completed and its writes are visible
// (hardware-managed, no spin of ours).  pdl_trigger() lets the next kernel launch
// as soon as every CTA of this one has issued it, instead of after the last exits.
// A kernel launched without the attribute passes pdl_wait() at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


struct RenderArgs {
    const PrimRec *rec;
    const int64_t *tile_off;
    const int32_t *list;
    const int32_t *tile_order;  // nullptr: tile id = work item
    const CanvasDesc *canvas;
    int32_t n_canvas;
    int32_t n_tiles;
    DevStatus *status;
    AtlasView atlas;
    int32_t bg_mode;
    float bg0, bg1, bg2;
    const float *bg_buf;
    float T_stop;
    // forward outputs / backward inputs
    float *image;
    float *T_final;
    int32_t *n_last;
    const float *dL_dimage;
    const float *dL_dalpha;
    float *graw;                // [N][8] raw per-primitive sums (backward; zero between calls)
    // rows [row0, row1) of every canvas are composited, regions outside are skipped
    // (row1 <= 0: all rows); both multiples of the tile size, so that no region
    // straddles the window
    int32_t row0, row1;
    int32_t n_prims;            // primitives of the plan (list entries index [0, n_prims))
    // Region scheduling.  A region's id is tile * R + r (R regions per tile).  With
    // item_order set, queue position q takes region item_order[q]; otherwise the
    // regions of tile_order's tiles in turn.  With item_cost set, the forward records
    // each region's cost (surviving records + 1) there and counts it into
    // item_hist[cost_bucket(cost)] (four buckets per octave), from which k_item_order
    // sorts the regions by decreasing cost for the next pass.
    const int32_t *item_order;
    int32_t *item_cost;
    int32_t *item_hist;         // [128] counts by cost bucket, then [128] cursors
    // forward with the MSE loss fused (null target: off): dL/dI = mse_scale (I - I*)
    // into mse_dL, and L = sum (I - I*)^2 / n added into *mse_loss (zeroed by the caller)
    const float *mse_target;
    float *mse_dL;
    double *mse_loss;
    float mse_scale;            // float(2 / n)
    double mse_inv_n;           // 1 / n, n = 3 x pixels of all canvases
    // Survivor record (null: off).  Forward: warp w of the grid appends every batch's
    // records that passed the region test, as (primitive, list position), to its own
    // segment surv[w surv_wcap, (w + 1) surv_wcap), and describes region i in
    // surv_tab[i] = (first entry, count, end of the list range it tested, 0), count -1
    // when not recorded (segment full, region outside the row window).  Backward
    // (surv_use): a recorded region whose range covers the pixels' last layers walks its
    // survivors instead of re-reading and re-testing its tile's list.
    int2 *surv;
    int4 *surv_tab;
    int64_t surv_cap;           // entries of surv (the launch divides them among its warps)
    int32_t surv_wcap;          // entries per warp (set by the launch)
    int32_t surv_use;
    int32_t count_pairs;        // forward: count the contributing pairs (status pairs_contrib)
};

}  // namespace dbmp
