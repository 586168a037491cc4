// BF16 GEMM on the sm_103a tensor cores (tcgen05 + TMEM), FP32 accumulation.
//
//   C[m][n] (op)= sum_k A[m][k] * B[n][k]      A: M x K, B: N x K, both K-contiguous BF16
//
// One CTA computes a 128 x BN tile.  128 threads stream K in stages of 64 with
// cp.async (16-byte chunks, zero-filled outside M / N) into shared memory laid out
// as the canonical no-swizzle K-major core-matrix layout: a core matrix is 8 rows
// x 16 bytes, core matrices adjacent in K are 128 bytes apart (leading byte offset)
// and those adjacent in M/N 1024 bytes apart (stride byte offset).  One elected
// thread issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into a TMEM
// accumulator of BN fp32 columns and commits each stage to an mbarrier, so loads of
// later stages overlap the tensor-core work.  The epilogue reads TMEM with
// tcgen05.ld (32 lanes x 32 bit per warp), applies the requested operation and
// writes C.  Split-K over gridDim.z adds partial tiles with fp32 atomics.
//
// Every mbarrier wait is bounded; a wait that gives up sets the status flag, the
// CTA drains its own copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbmp_internal.cuh"

namespace dbmp {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kStages = 3;
constexpr uint32_t kWaitLimit = 1u << 26;  // polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

// Waits for the phase of parity `parity` to complete; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major, version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    // base offset 0, lbo mode 0, layout type 0 (no swizzle)
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = 128, N = BN.
template <int BN>
__device__ __forceinline__ uint32_t instr_desc() {
    return (1u << 4)                 // D format: f32
           | (1u << 7)               // A format: bf16
           | (1u << 10)              // B format: bf16
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

// Byte offset of row r, 16-byte K-chunk kc inside one operand stage.
__device__ __forceinline__ uint32_t core_off(int r, int kc) {
    return (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
}

template <int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[kStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    constexpr int A_BYTES = kBM * kBK * 2;   // 16 KB
    constexpr int B_BYTES = BN * kBK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // align the dynamic buffer to 1024 bytes
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const uint32_t sbase = smem_u32(smem);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    (void)STAGE_BYTES;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kt_total = g.K / kBK;
    const int kt_per = (kt_total + gridDim.z - 1) / gridDim.z;
    const int kt0 = blockIdx.z * kt_per;
    const int T = min(kt_per, kt_total - kt0);

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&mbar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    auto load_stage = [&](int slot, int kt) {
        const uint32_t sa = sbase + slot * STAGE_BYTES, sb = sa + A_BYTES;
        const int kbase = (kt0 + kt) * kBK;
        // A: 128 rows x 8 chunks
        for (int c = tid; c < kBM * 8; c += 128) {
            const int r = c >> 3, kc = c & 7;
            const int m = m0 + r;
            const bool ok = m < g.M;
            const __nv_bfloat16 *src =
                reinterpret_cast<const __nv_bfloat16 *>(g.A) + (size_t)(ok ? m : 0) * g.lda + kbase + kc * 8;
            cp_async16_zfill(sa + core_off(r, kc), src, ok);
        }
        for (int c = tid; c < BN * 8; c += 128) {
            const int r = c >> 3, kc = c & 7;
            const int n = n0 + r;
            const bool ok = n < g.N;
            const __nv_bfloat16 *src =
                reinterpret_cast<const __nv_bfloat16 *>(g.B) + (size_t)(ok ? n : 0) * g.ldb + kbase + kc * 8;
            cp_async16_zfill(sb + core_off(r, kc), src, ok);
        }
    };

    bool ok = T > 0;
    if (ok) {
        for (int t = 0; t < kStages - 1; ++t) {
            if (t < T) load_stage(t, t);
            cp_async_commit();
        }
        const uint32_t idesc = instr_desc<BN>();
        for (int t = 0; t < T; ++t) {
            const int s = t % kStages;
            const int tp = t + kStages - 1;
            if (tp < T) {
                if (t >= 1) {
                    // the slot being refilled was read by MMA t-1
                    if (!mbar_wait(smem_u32(&mbar[(t - 1) % kStages]), ((t - 1) / kStages) & 1)) abort_flag = 1;
                }
                load_stage(tp % kStages, tp);
            }
            cp_async_commit();
            cp_async_wait<kStages - 1>();
            fence_async_smem();
            __syncthreads();
            if (abort_flag) {
                ok = false;
                break;
            }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t sa = sbase + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
                for (int ks = 0; ks < kBK / 16; ++ks) {
                    const uint64_t ad = smem_desc(sa + ks * 256, 128, 1024);
                    const uint64_t bd = smem_desc(sb + ks * 256, 128, 1024);
                    mma_bf16(tmem, ad, bd, idesc, (t > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(smem_u32(&mbar[s]));
            }
        }
        if (ok && !mbar_wait(smem_u32(&mbar[(T - 1) % kStages]), ((T - 1) / kStages) & 1)) abort_flag = 1;
    }
    cp_async_wait_all();
    __syncthreads();
    ok = ok && !abort_flag;  // uniform over the CTA: the epilogue's TMEM loads are warp-collective
    if (!ok && T > 0 && tid == 0 && g.status) atomicExch(g.status, (int)DBMP_ERR_TIMEOUT);
    tc_fence_after();

    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
            if (row >= g.M) continue;
            const int nb = n0 + c0;
            if (g.mode == GEMM_STORE_F32 || g.mode == GEMM_BIAS_F32) {
                float *out = g.Cf + (size_t)row * g.ldc + nb;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (nb + i < g.N) out[i] = v[i] + (g.mode == GEMM_BIAS_F32 ? g.bias[nb + i] : 0.0f);
            } else if (g.mode == GEMM_ATOMIC_F32) {
                float *out = g.Cf + (size_t)row * g.ldc + nb;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (nb + i < g.N) atomicAdd(out + i, v[i]);
            } else {  // GEMM_BIAS_RELU_BF16
                __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(g.Cb) + (size_t)row * g.ldc + nb;
                __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float b = nb + i < g.N ? g.bias[nb + i] : 0.0f;
                    h[i] = __float2bfloat16_rn(fmaxf(v[i] + b, 0.0f));
                }
                if (nb + 16 <= g.N && ((g.ldc & 7) == 0) && ((nb & 7) == 0)) {
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
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
}

template <int BN>
cudaError_t launch_gemm_t(const GemmArgs &g, int split_k, cudaStream_t st) {
    constexpr int smem = kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
    dim3 grid((g.M + kBM - 1) / kBM, (g.N + BN - 1) / BN, split_k);
    k_gemm_tc<BN><<<grid, 128, smem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t init_gemm_kernels() {
    constexpr int s32 = kStages * (kBM * kBK * 2 + 32 * kBK * 2) + 1024;
    constexpr int s64 = kStages * (kBM * kBK * 2 + 64 * kBK * 2) + 1024;
    constexpr int s128 = kStages * (kBM * kBK * 2 + 128 * kBK * 2) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, s128);
    return e;
}

cudaError_t launch_gemm(const GemmArgs &g, int split_k, cudaStream_t st) {
    if (g.K % kBK != 0 || g.M <= 0 || g.N <= 0 || split_k < 1) return cudaErrorInvalidValue;
    if (g.N <= 32) return launch_gemm_t<32>(g, split_k, st);
    if (g.N <= 64) return launch_gemm_t<64>(g, split_k, st);
    return launch_gemm_t<128>(g, split_k, st);
}

}  // namespace dbmp
