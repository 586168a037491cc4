// BF16 GEMM on the sm_103a tensor cores (tcgen05 + TMEM + TMA), FP32 accumulation.
//
//   C[m][n] (op)= sum_k A[m][k] * B[n][k]      A: M x K, B: N x K, both K-contiguous BF16
//
// A persistent CTA per SM computes 128 x BN tiles (BN = 32 ... 256) in turn, with
// three warp roles:
//   warp 0      producer: one thread issues the TMA tensor copies of the A and B
//               K-slabs (64 wide) into a ring of shared-memory stages, each stage
//               announced on its `full` mbarrier with the bytes it expects;
//   warp 1      allocates NACC BN TMEM columns (NACC accumulators, 2 or 4); one
//               thread issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction)
//               for each stage and commits it to the stage's `empty` mbarrier, which
//               returns the slot to the producer; a commit after a tile's last stage
//               marks its accumulator full;
//   warps 2-5   epilogue (and warps 6-9 for tiles of BN <= 64, taking every other
//               tile): each reads the TMEM lane quarter it may access
//               (32 (warp % 4) ...) with tcgen05.ld and applies the mode.  When C's
//               rows are 16-byte aligned, each warp writes 128-byte row pieces of its
//               32 rows into a double-buffered shared-memory box in the 128-byte
//               swizzled layout and one lane issues a TMA tensor store of the box (a
//               TMA reduce-add for split-K); otherwise every lane stores its own row.
// TMA writes each stage with the 128-byte swizzle, whose eight-row atoms of 1024
// bytes the shared-memory matrix descriptors describe (layout type SWIZZLE_128B):
//   K-major operand   one box of 64 (K) x rows: 128-byte rows along K, atoms 1024
//                     bytes apart along M/N; an MMA's K step of 16 advances the
//                     start address by 32 bytes;
//   MN-major operand  boxes of 64 (M/N) x 64 (K), 8 KB each: 128-byte rows along
//                     M/N, atoms 1024 bytes apart along K (stride byte offset),
//                     boxes 8 KB apart along M/N (leading byte offset); a K step of
//                     16 advances the start address by 2048 bytes.
// Rows past M or N are zero-filled by the tensor copy; K must be a multiple of 64.
// Split-K adds partial tiles into C (TMA reduce-add, or fp32 atomics).
//
// Every mbarrier wait is bounded.  A wait that gives up sets the status flag and every
// role stops at its next check; the producer still waits (bounded) for the copies it
// issued, the MMA thread for the MMAs it issued, and TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;   // a wait gives up after 2 s

// Epilogue staging: per epilogue warp two boxes of 32 rows x 128 bytes.
constexpr int kStageBox = 32 * 128;
constexpr int kSmemMax = 232448;                 // 227 KB of dynamic shared memory per block

// Per tile width: narrow tiles (BN <= 64) have two epilogue warpgroups taking
// alternate tiles and four TMEM accumulators, since their epilogue is as long as
// their MMAs and copies; wider tiles one warpgroup and two accumulators.
template <int BN>
struct TileCfg {
    static constexpr int EPI_GROUPS = BN <= 64 ? 2 : 1;
    static constexpr int NACC = 2 * EPI_GROUPS;                // accumulators (NACC BN TMEM columns)
    static constexpr int THREADS = 64 + 128 * EPI_GROUPS;
    static constexpr int EPI_BYTES = EPI_GROUPS * 4 * 2 * kStageBox;
    static constexpr int A_BYTES = kBM * kBK * 2;   // 16 KB
    static constexpr int B_BYTES = BN * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int FIT = (kSmemMax - 1024 - EPI_BYTES) / STAGE;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT;                  // with the staging boxes
    static constexpr int FIT_ALL = (kSmemMax - 1024) / STAGE;
    static constexpr int STAGES_MAX = FIT_ALL > 12 ? 12 : FIT_ALL;    // without them
    static constexpr int SMEM_EPI = STAGES * STAGE + EPI_BYTES + 1024;   // + alignment slack
    static constexpr int SMEM_NOEPI = STAGES_MAX * STAGE + 1024;
    static constexpr int SMEM = SMEM_EPI > SMEM_NOEPI ? SMEM_EPI : SMEM_NOEPI;
    static_assert(SMEM <= kSmemMax && STAGES >= 3, "shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Waits for the phase of parity `parity` to complete; false if it gave up after
// kWaitNs of the global timer.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 63) == 0) {
            const unsigned long long t = global_ns();
            if (i == 0) t0 = t;
            else if (t - t0 > kWaitNs) return false;
        }
    }
}

// 2-D tensor copy global -> shared (coordinates: x along K, y along rows),
// completing `bar`'s transaction count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 4-D tensor copy global -> shared (coordinates innermost first), completing `bar`'s
// transaction count.  Coordinates outside the tensor read zeros.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Coordinates of the 4-D copy of a conv operand: channel index `chan` (a multiple of
// 64: tap chan / conv_chan, channels chan % conv_chan ...) and first pixel row `row`
// (the box covers whole output rows of the Ho x Ho grid), for parity group grp.
// conv_chan and Ho are powers of two (lc, lh their log2): shifts and masks only, since
// one thread issues every copy and its arithmetic sits on the copy pipeline's path.
__device__ __forceinline__ void conv_coords(int kind, int lc, int lh, int chan, int row, int grp, int &c0, int &c1,
                                            int &c2, int &c3) {
    const int tap = chan >> lc;
    const int dy = tap >> 1, dx = tap & 1;
    const int oy = (row >> lh) & ((1 << lh) - 1);
    c0 = chan & ((1 << lc) - 1);
    c3 = row >> (2 * lh);
    if (kind == CONV_BLOCKED) {
        c1 = dx;
        c2 = oy + dy;
    } else {   // CONV_DGRAD: rows and columns one block up and left per parity
        c1 = 1 - (grp & 1) - dx;
        c2 = oy + 1 - (grp >> 1) - dy;
    }
}

// Column of the weight gradient's canonical (ky, kx, c) order for column n of the
// blocked tap order (GemmArgs::col_remap); runs of C columns stay contiguous.
__device__ __forceinline__ int remap_col(int n, int C) {
    if (C == 0) return n;
    const int tap = n / (4 * C), r = n - tap * 4 * C;
    const int s = r / C, c = r - s * C;
    const int ky = 2 * (tap >> 1) + (s >> 1), kx = 2 * (tap & 1) + (s & 1);
    return (ky * 4 + kx) * C + c;
}

// Element offset of output row `row` (column 0) and of its mask row (OUT_DGRAD).
__device__ __forceinline__ size_t out_row_offset(const GemmArgs &g, int row, int grp, size_t &moff) {
    moff = 0;
    if (g.out_kind == OUT_PLAIN) return (size_t)row * g.ldc;
    const int S = g.out_side, ls = 31 - __clz(S);   // S a power of two
    const int xj = row & (S - 1), t = row >> ls;
    const int yi = t & (S - 1), b = t >> ls;
    const size_t N = (size_t)g.N;
    if (g.out_kind == OUT_BLOCKED) {
        const int hb = S / 2 + 1;
        return (((size_t)b * hb + ((yi + 1) >> 1)) * hb + ((xj + 1) >> 1)) * 4 * N +
               (size_t)((((yi + 1) & 1) << 1) + ((xj + 1) & 1)) * N;
    }
    const int sy = grp >> 1, sx = grp & 1;
    const int H = 2 * S, y = 2 * yi + 1 - sy, x = 2 * xj + 1 - sx;
    moff = (((size_t)b * (S + 1) + yi + 1 - sy) * (S + 1) + xj + 1 - sx) * 4 * N + (size_t)grp * N;
    return (((size_t)b * H + y) * H + x) * N;
}

// 2-D tensor store / reduce-add shared -> global of one box (bulk async-group).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// at most one of this thread's bulk groups still reading shared memory
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory"); }
// all of this thread's bulk groups complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor (sm_100 family) with the 128-byte swizzle:
// stride byte offset 1024 (eight-row atoms); the leading byte offset is the
// distance between 64-element M/N boxes of an MN-major operand (not used by a
// swizzled K-major operand, which gets one 16-byte unit).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // leading byte offset
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 1024 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // layout: 128-byte swizzle
    return d;
}

// Descriptor of an unswizzled operand (layout type 0): core matrices of eight
// 16-byte rows, 128 contiguous bytes each.  K-major: lbo = distance between core
// matrices along K, sbo = along M/N; MN-major: lbo = along K, sbo = along M/N.
__device__ __forceinline__ uint64_t plain_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, M = 128, N = BN; bits 15
// and 16 mark A / B as MN-major.
template <int BN>
__device__ __forceinline__ uint32_t instr_desc(bool a_mn, bool b_mn) {
    return (1u << 4)                 // D format: f32
           | (1u << 7)               // A format: bf16
           | (1u << 10)              // B format: bf16
           | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16)
           | ((uint32_t)(BN >> 3) << 17)
           | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// The CTA's tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... as mixed-radix digits
// (tm, tn, sp, grp) of radices (tiles_m, tiles_n, split, groups), stepped by adding the
// digits of gridDim.x with carries: no division per tile on the roles' issue paths.
struct TileWalk {
    int rm, rn, rs;               // radices (the last digit needs none)
    int dm, dn, ds, dg;           // digits of the stride
    int tm, tn, sp, grp, t;       // the current tile
    __device__ TileWalk(int tiles_m, int tiles_n, int split) : rm(tiles_m), rn(tiles_n), rs(split) {
        digits(gridDim.x, dm, dn, ds, dg);
        digits(blockIdx.x, tm, tn, sp, grp);
        t = blockIdx.x;
    }
    __device__ void digits(int v, int &a, int &b, int &c, int &d) const {
        a = v % rm;
        v /= rm;
        b = v % rn;
        v /= rn;
        c = v % rs;
        d = v / rs;
    }
    __device__ void next() {
        t += gridDim.x;
        tm += dm;
        int c = tm >= rm;
        tm -= c ? rm : 0;
        tn += dn + c;
        c = tn >= rn;
        tn -= c ? rn : 0;
        sp += ds + c;
        c = sp >= rs;
        sp -= c ? rs : 0;
        grp += dg + c;
    }
};

// Persistent kernel: CTA c takes tiles c, c + gridDim.x, ... of the tiles_m x tiles_n
// x split schedule (m fastest, so that concurrent CTAs share the B tile).  The stage
// ring runs across tile boundaries, and the accumulator is double-buffered in TMEM
// (NACC BN columns): the MMA thread fills buffer lt % NACC of the CTA's tile lt while the
// epilogue warps drain the other.
//   acc_full[b]   completed by the MMA commit after a tile's last K step;
//   acc_empty[b]  completed when the four epilogue warps have read the buffer.
// Tiles of a split with no K steps are skipped by every role alike.
template <int BN>
__global__ void __launch_bounds__(TileCfg<BN>::THREADS, 1)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, GemmArgs g) {
    using C = TileCfg<BN>;
    // ring stages: fewer when the epilogue's TMA staging boxes share the shared memory
    const int S = g.tma_c ? C::STAGES : C::STAGES_MAX;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int NACC = C::NACC;
    __shared__ __align__(8) uint64_t full[C::STAGES_MAX], empty[C::STAGES_MAX], acc_full[NACC], acc_empty[NACC], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (g.M + kBM - 1) / kBM, tiles_n = (g.N + BN - 1) / BN;
    const int kt_total = g.K / kBK;
    const int kt_per = (kt_total + g.split - 1) / g.split;
    const int n_tiles = tiles_m * tiles_n * g.split * g.groups;
    // tile -> output origin (m0, n0), K steps [kt0, kt0 + T) and group grp
    auto decode = [&](const TileWalk &w, int &m0, int &n0, int &kt0, int &T, int &grp) {
        m0 = w.tm * kBM;
        n0 = w.tn * BN;
        kt0 = w.sp * kt_per;
        grp = w.grp;
        T = max(0, min(kt_per, kt_total - kt0));
    };

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 4);
        }
        mbar_init(smem_u32(&drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        if (g.tma_c) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)(NACC * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        const int lc = g.conv_chan ? __ffs(g.conv_chan) - 1 : 0, lh = g.conv_side ? __ffs(g.conv_side) - 1 : 0;
        uint32_t u = 0;   // stage uses issued: slot u % S, its (u / S)-th use
        int s = 0;
        uint32_t ph = 0;
        for (TileWalk w(tiles_m, tiles_n, g.split); w.t < n_tiles; w.next()) {
            int m0, n0, kt0, T, grp;
            decode(w, m0, n0, kt0, T, grp);
            for (int i = 0; i < T && !g.stall; ++i) {
                if (u >= (uint32_t)S && !mbar_wait(smem_u32(&empty[s]), ph ^ 1)) abort_flag = 1;
                if (*(volatile int *)&abort_flag) break;
                const uint32_t sa = sbase + s * C::STAGE, fb = smem_u32(&full[s]);
                const int k = (kt0 + i) * kBK;
                mbar_expect_tx(fb, C::STAGE);
                if (g.a_conv == CONV_PAIRS) {
                    // chunk kc = (ky, p) of every row: 128 rows x 16 B, 2 KB apart
                    const int b = m0 >> (2 * lh), oy = (m0 >> lh) & ((1 << lh) - 1), ox = m0 & ((1 << lh) - 1);
                    for (int kc = 0; kc < 8; ++kc)
                        tma_load_4d(sa + kc * 2048, &tmA, 0, ox + (kc & 1), 2 * oy - 1 + (kc >> 1), b, fb);
                } else if (g.a_conv) {
                    int c0, c1, c2, c3;
                    conv_coords(g.a_conv, lc, lh, k, m0, grp, c0, c1, c2, c3);
                    tma_load_4d(sa, &tmA, c0, c1, c2, c3, fb);
                } else if (g.a_mn) {
                    for (int j = 0; j < kBM / 64; ++j) tma_load_2d(sa + j * 8192, &tmA, m0 + 64 * j, k, fb);
                } else {
                    tma_load_2d(sa, &tmA, k, m0, fb);
                }
                if (g.b_conv == CONV_PAIRS) {
                    // MN-major: chunk kc = (ky, p) of 64 pixel rows, 64 x 16 B, 1 KB apart
                    const int b = k >> (2 * lh), oy = (k >> lh) & ((1 << lh) - 1), ox = k & ((1 << lh) - 1);
                    for (int kc = 0; kc < 8; ++kc)
                        tma_load_4d(sa + C::A_BYTES + kc * 1024, &tmB, 0, ox + (kc & 1), 2 * oy - 1 + (kc >> 1), b, fb);
                } else if (g.b_conv) {   // MN-major: 64 channels x 64 pixel rows per box
                    for (int j = 0; j < BN / 64; ++j) {
                        int c0, c1, c2, c3;
                        conv_coords(g.b_conv, lc, lh, n0 + 64 * j, k, grp, c0, c1, c2, c3);
                        tma_load_4d(sa + C::A_BYTES + j * 8192, &tmB, c0, c1, c2, c3, fb);
                    }
                } else if (g.b_mn) {
                    for (int j = 0; j < BN / 64; ++j)
                        tma_load_2d(sa + C::A_BYTES + j * 8192, &tmB, n0 + 64 * j, k, fb);
                } else {
                    tma_load_2d(sa + C::A_BYTES, &tmB, k, grp * g.N + n0, fb);
                }
                ++u;
                if (++s == S) s = 0, ph ^= 1;
            }
            if (*(volatile int *)&abort_flag) break;
        }
        // every issued copy lands before the CTA can exit
        for (uint32_t v = u > (uint32_t)S ? u - S : 0; v < u; ++v)
            if (!mbar_wait(smem_u32(&full[v % S]), (v / S) & 1)) abort_flag = 1;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const uint32_t idesc = instr_desc<BN>(g.a_mn != 0, g.b_mn != 0);
        // per K step of 16: +32 B (K-major) or +2048 B (MN-major); leading byte offsets
        const uint32_t a_step = g.a_conv == CONV_PAIRS ? 4096u : g.a_mn ? 2048u : 32u;
        const uint32_t b_step = g.b_conv == CONV_PAIRS ? 256u : g.b_mn ? 2048u : 32u;
        const uint32_t a_lbo = g.a_mn ? 8192u : 16u, b_lbo = g.b_mn ? 8192u : 16u;
        // pixel-pair operands are unswizzled: A (K-major) 16-byte chunks 2 KB apart along
        // K, eight-row groups 128 B apart along M; B (MN-major) eight-pixel groups 128 B
        // apart along K, 16-byte chunks 1 KB apart along N
        const bool a_plain = g.a_conv == CONV_PAIRS, b_plain = g.b_conv == CONV_PAIRS;
        int s = 0, lt = 0;
        uint32_t ph = 0;
        for (TileWalk w(tiles_m, tiles_n, g.split); w.t < n_tiles; w.next()) {
            int m0, n0, kt0, T, grp;
            decode(w, m0, n0, kt0, T, grp);
            if (T == 0) continue;
            const int b = lt % NACC;
            if (lt >= NACC && !mbar_wait(smem_u32(&acc_empty[b]), ((lt / NACC) & 1) ^ 1)) abort_flag = 1;
            if (*(volatile int *)&abort_flag) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * BN);
            for (int i = 0; i < T; ++i) {
                if (!mbar_wait(smem_u32(&full[s]), ph)) abort_flag = 1;
                if (*(volatile int *)&abort_flag) break;
                tc_fence_after();
                const uint32_t sa = sbase + s * C::STAGE, sb = sa + C::A_BYTES;
                // a K step of 16 moves the start address field (address >> 4, below
                // 2^14 for any shared-memory address) without a carry into the rest
                const uint64_t da = a_plain ? plain_desc(sa, 2048u, 128u) : sw128_desc(sa, a_lbo);
                const uint64_t db = b_plain ? plain_desc(sb, 128u, 1024u) : sw128_desc(sb, b_lbo);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(d, da + (uint64_t)((kk * a_step) >> 4), db + (uint64_t)((kk * b_step) >> 4), idesc,
                             (i > 0 || kk > 0) ? 1u : 0u);
                mma_commit(smem_u32(&empty[s]));
                if (++s == S) s = 0, ph ^= 1;
            }
            if (*(volatile int *)&abort_flag) break;
            mma_commit(smem_u32(&acc_full[b]));   // arrives once the tile's MMAs have completed
            ++lt;
        }
        mma_commit(smem_u32(&drain));             // every MMA issued by this thread
        if (!mbar_wait(smem_u32(&drain), 0)) abort_flag = 1;
    } else if (warp >= 2) {
        // ---- epilogue ----
        const int q = warp & 3;                   // TMEM lanes 32 q .. 32 q + 31
        const int eg = (warp - 2) >> 2;           // epilogue group: tiles lt with lt % EPI_GROUPS == eg
        const bool bf = g.mode == GEMM_BIAS_RELU_BF16 || g.mode == GEMM_STORE_BF16;
        const bool relu = g.mode == GEMM_BIAS_RELU_BF16;
        const int ecols = bf ? 64 : 32;           // columns of a 128-byte row piece
        const uint32_t box0 = sbase + S * C::STAGE + (uint32_t)((warp - 2) * 2 * kStageBox);
        unsigned char *box0p = smem + S * C::STAGE + (warp - 2) * 2 * kStageBox;
        int buf = 0, lt = 0;
        for (TileWalk w(tiles_m, tiles_n, g.split); w.t < n_tiles; w.next()) {
            int m0, n0, kt0, T, grp;
            decode(w, m0, n0, kt0, T, grp);
            if (T == 0) continue;
            if (lt % C::EPI_GROUPS != eg) {       // the other group's tile
                ++lt;
                continue;
            }
            const int b = lt % NACC;
            // the per-lane path's row placement and, for OUT_DGRAD tiles of BN <= 64, the
            // row's mask: loaded before the accumulator wait so that the mask's memory
            // latency overlaps the tile's MMAs
            const int row = m0 + q * 32 + lane;
            size_t moff = 0;
            const size_t ooff = (!g.tma_c && row < g.M) ? out_row_offset(g, row, grp, moff) : 0;
            constexpr int MKN = BN <= 64 ? BN / 8 : 1;
            uint4 mk[MKN];
            if (BN <= 64 && g.mask && row < g.M) {
#pragma unroll
                for (int j = 0; j < MKN; ++j)
                    if (n0 + 8 * j + 8 <= g.N) mk[j] = __ldg(reinterpret_cast<const uint4 *>(g.mask + moff + n0) + j);
            }
            bool ok = mbar_wait(smem_u32(&acc_full[b]), (lt / NACC) & 1);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) abort_flag = 1;
            ok = ok && !*(volatile int *)&abort_flag;
            ok = __all_sync(0xffffffffu, ok);     // tcgen05.ld below is warp-collective
            if (!ok) break;
            tc_fence_after();
            const uint32_t trow = tmem + (uint32_t)(b * BN) + ((uint32_t)(q * 32) << 16);
            if (g.tma_c) {
                // Row `lane` of a staging box holds its eight 16-byte chunks at
                // chunk ^ (lane % 8) (128-byte swizzle: conflict-free for the warp,
                // the layout the tensor map's swizzle reads).
                for (int c0 = 0; c0 < BN; c0 += ecols, buf ^= 1) {
                    uint32_t w[32];   // this lane's 128 bytes of the piece
                    for (int h = 0; h < ecols; h += 16) {
                        float v[16];
                        if (c0 + h < BN) {   // a 64-column bf16 piece of a 32-wide tile: the rest is
                            tmem_ld16(trow + c0 + h, v);   // past N (the store clips it) and never read
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[i] = 0.0f;
                        }
                        const int nb = n0 + c0 + h;
                        if (g.mode == GEMM_BIAS_F32 || g.mode == GEMM_BIAS_RELU_BF16) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[i] += nb + i < g.N ? g.bias[nb + i] : 0.0f;
                        }
                        if (relu) {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                w[h / 2 + i] = pack_bf16x2(fmaxf(v[2 * i], 0.0f), fmaxf(v[2 * i + 1], 0.0f));
                        } else if (bf) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) w[h / 2 + i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) w[h + i] = __float_as_uint(v[i]);
                        }
                    }
                    if (lane == 0) bulk_wait_read1();   // the store issued from this buffer two pieces ago
                    __syncwarp();
                    unsigned char *rowp = box0p + buf * kStageBox + lane * 128;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<uint4 *>(rowp + ((j ^ (lane & 7)) << 4)) =
                            make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        const uint32_t src = box0 + (uint32_t)(buf * kStageBox);
                        const int x = remap_col(n0 + c0, g.col_remap);
                        if (g.mode == GEMM_ATOMIC_F32)
                            tma_reduce_add_2d(&tmC, x, m0 + q * 32, src);
                        else
                            tma_store_2d(&tmC, x, m0 + q * 32, src);
                        bulk_commit();
                    }
                }
            } else {
#pragma unroll(BN <= 64 ? BN / 16 : 1)
                for (int c0 = 0; c0 < BN; c0 += 16) {
                    float v[16];
                    tmem_ld16(trow + c0, v);
                    if (row >= g.M) continue;
                    const int nb = n0 + c0;
                    const bool full16 = nb + 16 <= g.N;
                    if (g.mode == GEMM_STORE_F32 || g.mode == GEMM_BIAS_F32) {
                        float *out = g.Cf + ooff + nb;
                        if (g.mode == GEMM_BIAS_F32) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[i] += nb + i < g.N ? g.bias[nb + i] : 0.0f;
                        }
                        if (full16 && ((g.ldc & 3) == 0) && ((nb & 3) == 0)) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                reinterpret_cast<float4 *>(out)[i] =
                                    make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (nb + i < g.N) out[i] = v[i];
                        }
                    } else if (g.mode == GEMM_ATOMIC_F32) {
                        float *out = g.Cf + ooff + remap_col(nb, g.col_remap);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (nb + i < g.N) atomicAdd(out + i, v[i]);
                    } else {  // GEMM_BIAS_RELU_BF16, GEMM_STORE_BF16
                        __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(g.Cb) + ooff + nb;
                        __align__(16) __nv_bfloat16 h[16];
                        if (relu) {
                            float bb[16];
                            if (full16 && (((uintptr_t)(g.bias + nb) & 15) == 0)) {
#pragma unroll
                                for (int i = 0; i < 4; ++i)
                                    *reinterpret_cast<float4 *>(bb + 4 * i) =
                                        __ldg(reinterpret_cast<const float4 *>(g.bias + nb) + i);
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i) bb[i] = nb + i < g.N ? g.bias[nb + i] : 0.0f;
                            }
#pragma unroll
                            for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(fmaxf(v[i] + bb[i], 0.0f));
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(v[i]);
                        }
                        if (g.mask) {   // OUT_DGRAD: N is a multiple of 16, rows 16-byte aligned
                            __align__(16) uint16_t m16[16];
                            if (BN <= 64) {
                                reinterpret_cast<uint4 *>(m16)[0] = mk[(c0 >> 3) % MKN];
                                reinterpret_cast<uint4 *>(m16)[1] = mk[((c0 >> 3) + 1) % MKN];
                            } else {
                                const uint4 *mp = reinterpret_cast<const uint4 *>(g.mask + moff + nb);
                                reinterpret_cast<uint4 *>(m16)[0] = mp[0];
                                reinterpret_cast<uint4 *>(m16)[1] = mp[1];
                            }
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (!(__bfloat162float(__ushort_as_bfloat16(m16[i])) > 0.0f)) h[i] = __float2bfloat16_rn(0.0f);
                        }
                        if (full16 && (((ooff + nb) & 7) == 0)) {
                            reinterpret_cast<uint4 *>(out)[0] = reinterpret_cast<const uint4 *>(h)[0];
                            reinterpret_cast<uint4 *>(out)[1] = reinterpret_cast<const uint4 *>(h)[1];
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (nb + i < g.N) out[i] = h[i];
                        }
                    }
                }
            }
            // this warp's reads of buffer b are complete: release it to the MMA thread
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
            ++lt;
        }
        if (lane == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag && g.status) atomicExch(g.status, (int)DBMP_ERR_TIMEOUT);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)(NACC * BN))
                     : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Tensor map of a row-major bf16 matrix with `inner` contiguous elements per row and
// `outer` rows (row stride ld elements), copied in boxes of 64 (inner) x box_outer
// with the 128-byte swizzle; out-of-range elements read 0.  K-major operands have
// inner = K, MN-major operands inner = M (or N).
bool make_map(CUtensorMap *m, const uint16_t *base, int outer, int inner, int ld, int box_outer) {
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D tensor map of a conv operand's source [nb][side][side][chan] (bf16, channels
// contiguous), copied in boxes of 64 channels x `rows` pixel rows of the Ho x Ho output
// grid (whole rows: Ho columns, rows / Ho grid rows, or whole Ho x Ho images), with the
// 128-byte swizzle: each pixel row is one 128-byte row of the box, as in a 2-D copy of
// the equivalent matrix.  Out-of-range coordinates read 0.
bool make_map_conv(CUtensorMap *m, const uint16_t *base, int chan, int side, int nb, int ho, int rows) {
    const int bw = ho < rows ? ho : rows;
    const int bh = ho < rows / bw ? ho : rows / bw;
    const int bb = rows / (bw * bh);
    if (bw * bh * bb != rows || bb > nb || chan % 64 != 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)chan, (cuuint64_t)side, (cuuint64_t)side, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {(cuuint64_t)chan * 2, (cuuint64_t)side * chan * 2,
                                   (cuuint64_t)side * side * chan * 2};
    const cuuint32_t box[4] = {64u, (cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bb};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D tensor map of the first conv's padded input [nb][2 Ho][2 Ho + 2][4] (bf16, one
// zero pixel on each side of a row) as pixel pairs: [nb][2 Ho][Ho + 1][8], pair j =
// padded pixels 2j, 2j + 1.  Boxes of 8 elements (16 bytes) x `rows` pairs of one row,
// unswizzled: for output pixel ox, tap row ky and pair p = kx / 2, pair ox + p holds
// taps kx = 2p, 2p + 1 of the 4 x 4 window, so a box starting at pair ox0 + p of row
// 2 oy - 1 + ky is one 16-byte K chunk of `rows` consecutive output pixels.
bool make_map_pairs(CUtensorMap *m, const uint16_t *base, int ho, int nb, int rows) {
    const cuuint64_t pairs = (cuuint64_t)ho + 1, H = 2 * (cuuint64_t)ho, row_bytes = (2 * (cuuint64_t)ho + 2) * 8;
    const cuuint64_t dims[4] = {8, pairs, H, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {16, row_bytes, H * row_bytes};
    const cuuint32_t box[4] = {8u, (cuuint32_t)rows, 1u, 1u};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the output C (M rows of N elements, row stride ldc) for the
// epilogue's TMA stores: boxes of 128 bytes (32 fp32 or 64 bf16) x 32 rows, 128-byte
// swizzle.  False when C's base or row stride is not 16-byte aligned, and for rows of
// under 256 bytes: there one lane per row already stores a warp's rows contiguously,
// and the staging buffers would only cost resident CTAs.
bool make_map_c(CUtensorMap *m, const GemmArgs &g) {
    const bool bf = g.mode == GEMM_BIAS_RELU_BF16 || g.mode == GEMM_STORE_BF16;
    const void *base = bf ? (const void *)g.Cb : (const void *)g.Cf;
    const size_t esz = bf ? 2 : 4;
    if (!base || ((uintptr_t)base & 15) || (((size_t)g.ldc * esz) & 15) || g.ldc < g.N) return false;
    if ((size_t)g.ldc * esz < 256 || g.out_kind != OUT_PLAIN) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
    const cuuint64_t strides[1] = {(cuuint64_t)g.ldc * esz};
    const cuuint32_t box[2] = {bf ? 64u : 32u, 32u};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(m, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_gemm_t(const GemmArgs &g0, int split_k, int sms, cudaStream_t st) {
    CUtensorMap ta, tb, tc;
    GemmArgs g = g0;
    auto conv_map = [&](CUtensorMap *m, const uint16_t *base, int kind, int rows) {
        if (kind == CONV_PAIRS) return make_map_pairs(m, base, g.conv_side, g.conv_batch, rows);
        const int side = kind == CONV_BLOCKED ? g.conv_side + 1 : g.conv_side;
        return make_map_conv(m, base, g.conv_chan, side, g.conv_batch, g.conv_side, rows);
    };
    const bool ok_a = g.a_conv ? conv_map(&ta, g.A, g.a_conv, kBM)
                      : g.a_mn ? make_map(&ta, g.A, g.K, g.M, g.lda, kBK)
                               : make_map(&ta, g.A, g.M, g.K, g.lda, kBM);
    const bool ok_b = g.b_conv ? conv_map(&tb, g.B, g.b_conv, kBK)
                      : g.b_mn ? make_map(&tb, g.B, g.K, g.N, g.ldb, kBK)
                               : make_map(&tb, g.B, g.N * g.groups, g.K, g.ldb, BN);
    if (!ok_a || !ok_b) return cudaErrorInvalidValue;
    memset(&tc, 0, sizeof tc);
    g.tma_c = make_map_c(&tc, g) ? 1 : 0;
    g.split = split_k;
    const int64_t tiles = (int64_t)((g.M + kBM - 1) / kBM) * ((g.N + BN - 1) / BN) * split_k * g.groups;
    if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
    // One CTA per SM: the ring and the staging boxes take most of the SM's shared
    // memory, the accumulators NACC BN of its 512 TMEM columns.  The ring
    // runs across tiles, so a short-K product still has several tiles' operands in flight.
    const int smem = g.tma_c ? TileCfg<BN>::SMEM_EPI : TileCfg<BN>::SMEM_NOEPI;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_gemm_tma<BN><<<grid, TileCfg<BN>::THREADS, smem, st>>>(ta, tb, tc, g);
    return cudaGetLastError();
}

template <int BN>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_gemm_tma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<BN>::SMEM);
}

}  // namespace

// The driver's tensor-map encoder is looked up once per process; the kernels'
// shared-memory limits are raised once per device (each under its own
// std::call_once, with that device current), so repeated and concurrent callers
// neither race nor repeat the attribute calls.
cudaError_t init_gemm_kernels() {
    static std::once_flag encode_once;
    static cudaError_t encode_err = cudaSuccess;
    std::call_once(encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (encode_err == cudaSuccess && (q != cudaDriverEntryPointSuccess || !fn)) encode_err = cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (encode_err != cudaSuccess) return encode_err;
    constexpr int kMaxDevices = 64;
    static std::once_flag dev_once[kMaxDevices];
    static cudaError_t dev_err[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(dev_once[dev], [dev] {
        cudaError_t r = set_smem<32>();
        if (r == cudaSuccess) r = set_smem<64>();
        if (r == cudaSuccess) r = set_smem<128>();
        if (r == cudaSuccess) r = set_smem<256>();
        dev_err[dev] = r;
    });
    return dev_err[dev];
}

cudaError_t launch_gemm(const GemmArgs &g, int split_k, cudaStream_t st) {
    if (g.K % kBK != 0 || g.M <= 0 || g.N <= 0 || split_k < 1 || !g_encode) return cudaErrorInvalidValue;
    if (g.a_conv == CONV_PAIRS || g.b_conv == CONV_PAIRS) {
        // the first conv: K = 16 taps x 4 channels = 64 (A), or N = 64 (B, MN-major);
        // boxes of 128 (A) or 64 (B) pixels within one output row
        const int ho = g.conv_side;
        if (ho < 128 || (ho & (ho - 1)) || g.conv_batch < 1 || (g.a_conv && g.b_conv) ||
            (g.a_conv && (g.K != 64 || g.a_mn)) || (g.b_conv && (g.N != 64 || !g.b_mn)))
            return cudaErrorInvalidValue;
    } else if (g.a_conv || g.b_conv) {
        // whole output rows per box (Ho <= 64), 64-channel K steps, a conv B operand
        // given MN-major, and room for a box that spans two images
        const int ho = g.conv_side;
        if (ho < 8 || ho > 64 || (ho & (ho - 1)) || g.conv_chan < 64 || (g.conv_chan & (g.conv_chan - 1)) ||
            g.conv_batch < 2 || (g.a_conv && g.a_mn) ||
            (g.b_conv && !g.b_mn) || (g.a_conv && g.b_conv))
            return cudaErrorInvalidValue;
    }
    if (g.groups != 1 && (g.groups != 4 || g.b_mn || g.b_conv || (g.N & 31))) return cudaErrorInvalidValue;
    if (g.out_kind != OUT_PLAIN && (g.out_side < 2 || (g.out_side & 1) || (g.N & 15) || g.mode == GEMM_ATOMIC_F32))
        return cudaErrorInvalidValue;
    if (g.mask && g.out_kind != OUT_DGRAD) return cudaErrorInvalidValue;
    if (g.col_remap && (g.col_remap & 31 || g.N != 16 * g.col_remap)) return cudaErrorInvalidValue;
    // tile width: the narrowest of {32 (K-major B only: MN-major boxes are 64 wide), 64,
    // 128, 256} covering N, halved (down to 64) while twice the CTAs still fit one wave
    const int sms = sm_count();
    int bn = g.N <= 32 && !g.b_mn ? 32 : g.N <= 64 ? 64 : g.N <= 128 ? 128 : 256;
    const int64_t rows = (g.M + kBM - 1) / kBM;
    while (bn > 64 && 2 * rows * ((g.N + bn - 1) / bn) * split_k * g.groups <= sms) bn /= 2;
    if (bn == 32) return launch_gemm_t<32>(g, split_k, sms, st);
    if (bn == 64) return launch_gemm_t<64>(g, split_k, sms, st);
    if (bn == 128) return launch_gemm_t<128>(g, split_k, sms, st);
    return launch_gemm_t<256>(g, split_k, sms, st);
}

}  // namespace dbmp
