// gemm_tc.cuh -- BF16 GEMM on the fifth-generation tensor cores (tcgen05,
// sm_103a): C[z] (+)= alpha A[z] B[z], A (M x K) and B (K x N) BF16 with
// arbitrary element strides, C FP32 with arbitrary strides.
//
// One CTA of 128 threads computes a 128 x BN tile of C:
//   * warp 0 allocates BN columns of tensor memory (TMEM) for the FP32
//     accumulator (128 lanes = the tile's rows);
//   * per K slice of 32, all threads gather the A tile (128 x 32) and the B
//     tile (BN x 32, i.e. B^T) into shared memory in the canonical K-major
//     layout without swizzle: 8-row x 16-byte core matrices, the two K halves
//     of a 16-wide MMA step at LBO, successive 8-row groups at SBO;
//   * thread 0 issues two tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulation, M = 128, N = BN, K = 16) and commits them to an
//     mbarrier that every thread waits on before the next gather;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32 w .. 32 w + 31, one row per thread) and applies alpha / beta /
//     the atomic add.
// Every mbarrier wait is bounded: on expiry the kernel sets *err, waits once
// more (bounded) for the MMAs in flight, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mmk {

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    float* C;
    int M, N, K;
    long long sam, sak, sbk, sbn, scm, scn;     // element strides
    long long zA, zB, zC;                        // batch strides
    float alpha, beta;
    int atomic;                                  // accumulate into C with atomicAdd
    int* err;                                    // set to 1 when a tensor-core wait expires
};

constexpr int kTcM = 128, kTcK = 32, kTcThreads = 128;
constexpr long long kTcWaitLimit = 1LL << 22;   // non-blocking mbarrier polls (well under a second)

// Shared-memory matrix descriptor of a K-major operand without swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);           // start address (16-byte units)
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;         // leading-dimension (K) core-matrix offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;         // stride-dimension (M / N) core-matrix offset
    d |= (uint64_t)1 << 46;                              // descriptor version for tcgen05
    return d;                                            // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int m, int n) {
    return (1u << 4)                                     // D format: F32
           | (1u << 7)                                   // A format: BF16
           | (1u << 10)                                  // B format: BF16
           | ((uint32_t)(n >> 3) << 17)                  // N / 8
           | ((uint32_t)(m >> 4) << 24);                 // M / 16
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kTcWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Offset in bytes of element (row r, k) of a K-major tile of 32 columns:
// core matrix (r / 8, k / 8) at (r / 8) * 512 + (k / 8) * 128, its row r % 8
// at 16 (r % 8), its element k % 8 at 2 (k % 8).  LBO = 128, SBO = 512.
__device__ __forceinline__ uint32_t tc_tile_off(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Epilogue of a 128 x BN tile: row m0 + 32 warp + lane, 16 columns per
// tcgen05.ld (issued false: nothing was accumulated, K = 0, the product is
// zero); alpha / beta / the atomic add; 16-byte stores where C is row-major
// with 16-byte aligned rows.
template <int BN>
__device__ __forceinline__ void tc_epilogue(const GemmArgs& a, float* C, uint32_t tmem, int m0, int n0, int warp,
                                            int lane, bool issued) {
    const int r = m0 + warp * 32 + lane;
    const bool c_vec = !a.atomic && a.scn == 1 && a.scm % 4 == 0 && a.zC % 4 == 0 &&
                       (reinterpret_cast<uintptr_t>(a.C) & 15) == 0;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16] = {};
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        if (issued) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
        if (r < a.M) {
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
                const int c = n0 + c0 + 4 * j4;
                if (c_vec && c + 3 < a.N) {
                    float4* p = reinterpret_cast<float4*>(C + r * a.scm + c);
                    float4 o = make_float4(a.alpha * __uint_as_float(v[4 * j4]),
                                           a.alpha * __uint_as_float(v[4 * j4 + 1]),
                                           a.alpha * __uint_as_float(v[4 * j4 + 2]),
                                           a.alpha * __uint_as_float(v[4 * j4 + 3]));
                    if (a.beta != 0.f) {
                        const float4 q = *p;
                        o.x += a.beta * q.x;
                        o.y += a.beta * q.y;
                        o.z += a.beta * q.z;
                        o.w += a.beta * q.w;
                    }
                    *p = o;
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (c + j < a.N) {
                        float* p = C + r * a.scm + (c + j) * a.scn;
                        const float val = a.alpha * __uint_as_float(v[4 * j4 + j]);
                        if (a.atomic) atomicAdd(p, val);
                        else *p = (a.beta != 0.f) ? a.beta * *p + val : val;
                    }
                }
            }
        }
    }
}

// Epilogue for a row-major C with 16-byte aligned rows: per 16-column
// chunk the warp's 32 rows go through the warp's 32 x 17 float buffer `buf`
// in shared memory; lane l then stores 4 columns of rows 8 i + l / 4.
template <int BN>
__device__ __forceinline__ void tc_epilogue_rows(const GemmArgs& a, float* C, uint32_t tmem, int m0, int n0,
                                                 int warp, int lane, float* buf) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) buf[lane * 17 + j] = __uint_as_float(v[j]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int rr = 8 * i + (lane >> 2), cq = lane & 3;
            const int row = m0 + warp * 32 + rr, col = n0 + c0 + 4 * cq;
            const float* b = buf + rr * 17 + 4 * cq;
            if (row < a.M) {
                float* p = C + (long long)row * a.scm + col;
                if (col + 3 < a.N) {
                    float4 o = make_float4(a.alpha * b[0], a.alpha * b[1], a.alpha * b[2], a.alpha * b[3]);
                    if (a.beta != 0.f) {
                        const float4 q = *reinterpret_cast<const float4*>(p);
                        o.x += a.beta * q.x;
                        o.y += a.beta * q.y;
                        o.z += a.beta * q.z;
                        o.w += a.beta * q.w;
                    }
                    *reinterpret_cast<float4*>(p) = o;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (col + j < a.N) p[j] = (a.beta != 0.f) ? a.beta * p[j] + a.alpha * b[j] : a.alpha * b[j];
                }
            }
        }
        __syncwarp();
    }
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(GemmArgs a) {
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "MMA N and TMEM columns");
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* As = tc_smem;                          // 128 x 32 BF16 = 8 KB
    unsigned char* Bs = tc_smem + kTcM * kTcK * 2;        // BN x 32 BF16
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    const int z = blockIdx.z;
    const __nv_bfloat16* A = a.A + z * a.zA;
    const __nv_bfloat16* B = a.B + z * a.zB;
    float* C = a.C + z * a.zC;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(&mbar);
    const uint32_t As_s = (uint32_t)__cvta_generic_to_shared(As);
    const uint32_t Bs_s = (uint32_t)__cvta_generic_to_shared(Bs);

    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;                      // lane 0, first allocated column

    constexpr uint32_t idesc = tc_idesc_bf16(kTcM, BN);
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    uint32_t parity = 0;
    bool ok = true;
    bool issued = false;
    // A with unit K stride, 8 | K and 16-byte aligned rows: each core-matrix
    // row (8 consecutive k of one row) is one 16-byte load and store, and the
    // next K slice is loaded into registers while the MMAs of this one run.
    // Otherwise element gathers whose consecutive threads follow the operand's
    // unit-stride axis.
    const bool a_vec = a.sak == 1 && a.K % 8 == 0 && a.sam % 8 == 0 && a.zA % 8 == 0 &&
                       (reinterpret_cast<uintptr_t>(a.A) & 15) == 0;
    const bool a_mfast = !a_vec && a.sam == 1;
    const bool b_kfast = a.sbk == 1 && a.sbn != 1;
    constexpr int AV = kTcM * (kTcK / 8) / kTcThreads;    // 16-byte chunks of A per thread
    uint4 pre[AV];
    auto load_a = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AV; ++q) {
            const int e = threadIdx.x + q * kTcThreads;
            const int r = e / (kTcK / 8), c = e % (kTcK / 8);
            const int gi = m0 + r, gk = k0 + 8 * c;
            pre[q] = make_uint4(0u, 0u, 0u, 0u);
            if (gi < a.M && gk < a.K) pre[q] = *reinterpret_cast<const uint4*>(A + gi * a.sam + gk);
        }
    };
    if (a_vec && a.K > 0) load_a(0);
    for (int k0 = 0; k0 < a.K && ok; k0 += kTcK) {
        // gather: element (row, k) of each tile, zero outside the matrices
        if (a_vec) {
#pragma unroll
            for (int q = 0; q < AV; ++q) {
                const int e = threadIdx.x + q * kTcThreads;
                const int r = e / (kTcK / 8), c = e % (kTcK / 8);
                *reinterpret_cast<uint4*>(As + tc_tile_off(r, 8 * c)) = pre[q];
            }
        } else {
            for (int e = threadIdx.x; e < kTcM * kTcK; e += kTcThreads) {
                const int r = a_mfast ? e % kTcM : e / kTcK, k = a_mfast ? e / kTcM : e % kTcK;
                const int gi = m0 + r, gk = k0 + k;
                const __nv_bfloat16 v = (gi < a.M && gk < a.K) ? A[gi * a.sam + gk * a.sak] : zero;
                *reinterpret_cast<__nv_bfloat16*>(As + tc_tile_off(r, k)) = v;
            }
        }
        for (int e = threadIdx.x; e < BN * kTcK; e += kTcThreads) {
            const int k = b_kfast ? e % kTcK : e / BN, n = b_kfast ? e / kTcK : e % BN;
            const int gk = k0 + k, gj = n0 + n;
            const __nv_bfloat16 v = (gk < a.K && gj < a.N) ? B[gk * a.sbk + gj * a.sbn] : zero;
            *reinterpret_cast<__nv_bfloat16*>(Bs + tc_tile_off(n, k)) = v;
        }
        // generic-proxy stores -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks) {
                // K step ks covers core-matrix columns 2 ks and 2 ks + 1
                const uint64_t ad = tc_smem_desc(As_s + ks * 256, 128, 512);
                const uint64_t bd = tc_smem_desc(Bs_s + ks * 256, 128, 512);
                const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_s)
                         : "memory");
        }
        issued = true;
        if (a_vec && k0 + kTcK < a.K) load_a(k0 + kTcK);  // in flight during the MMAs
        // one decision for the whole CTA, so that every thread leaves the
        // loop at the same barrier
        ok = __syncthreads_and(tc_wait(mbar_s, parity) ? 1 : 0) != 0;
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(a.err, 1);
        tc_wait(mbar_s, parity ^ 1u);                     // the abandoned phase, bounded again
    }
    if (ok) tc_epilogue<BN>(a, C, tmem, m0, n0, warp, lane, issued);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// All of K resident (K a multiple of 16 up to kTcKFull, both operands
// K-contiguous with 16-byte aligned rows): every 16-byte chunk of the A
// (128 x K) and B (BN x K) tiles is requested at once with cp.async (zero
// fill outside M and N), then thread 0 issues the K / 16 MMAs back to back
// and commits them once.  A tile costs one memory latency and one MMA wait
// instead of one of each per 32-wide K slice.  Tile layout: K-major core
// matrices without swizzle, row r and chunk c (k = 8 c .. 8 c + 7) at
// (r / 8) * (K / 8) * 128 + c * 128 + (r % 8) * 16: LBO 128, SBO 16 K.
constexpr int kTcKFull = 256;

__device__ __forceinline__ void tc_cp16(uint32_t dst, const void* src, bool in) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc_kfull(GemmArgs a) {
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "MMA N and TMEM columns");
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int K = a.K, KC = K / 8;                        // 16-byte chunks per row
    const uint32_t As_s = (uint32_t)__cvta_generic_to_shared(tc_smem);
    const uint32_t Bs_s = As_s + (uint32_t)(kTcM * K * 2);
    const uint32_t sbo = (uint32_t)KC * 128;

    const int z = blockIdx.z;
    const __nv_bfloat16* A = a.A + z * a.zA;
    const __nv_bfloat16* B = a.B + z * a.zB;
    float* C = a.C + z * a.zC;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(&mbar);
    // launched with programmatic serialisation: the predecessor's writes
    // first (no-op otherwise); then the successor may start launching
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // the whole tile pair in flight before anything else
    for (int e = threadIdx.x; e < kTcM * KC; e += kTcThreads) {
        const int r = e / KC, c = e - r * KC;
        const bool in = m0 + r < a.M;
        tc_cp16(As_s + (uint32_t)((r >> 3) * sbo + c * 128 + (r & 7) * 16),
                in ? (const void*)(A + (long long)(m0 + r) * a.sam + 8 * c) : (const void*)A, in);
    }
    for (int e = threadIdx.x; e < BN * KC; e += kTcThreads) {
        const int n = e / KC, c = e - n * KC;
        const bool in = n0 + n < a.N;
        tc_cp16(Bs_s + (uint32_t)((n >> 3) * sbo + c * 128 + (n & 7) * 16),
                in ? (const void*)(B + (long long)(n0 + n) * a.sbn + 8 * c) : (const void*)B, in);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // this thread's copies -> visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    constexpr uint32_t idesc = tc_idesc_bf16(kTcM, BN);
    if (threadIdx.x == 0) {
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc_smem_desc(As_s + ks * 256, 128, sbo);
            const uint64_t bd = tc_smem_desc(Bs_s + ks * 256, 128, sbo);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_s)
                     : "memory");
    }
    const bool ok = __syncthreads_and(tc_wait(mbar_s, 0) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(a.err, 1);
        tc_wait(mbar_s, 0);                               // the MMAs in flight, bounded again
    } else if (!a.atomic && a.scn == 1 && a.scm % 4 == 0 && a.zC % 4 == 0 &&
               (reinterpret_cast<uintptr_t>(a.C) & 15) == 0) {
        // row-major C: the operand tiles are free now; each warp passes its
        // rows through 32 x 17 floats of them so that a store instruction
        // writes 64 contiguous bytes of each of 8 rows
        tc_epilogue_rows<BN>(a, C, tmem, m0, n0, warp, lane,
                             reinterpret_cast<float*>(tc_smem) + warp * 32 * 17);
    } else {
        tc_epilogue<BN>(a, C, tmem, m0, n0, warp, lane, true);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// Dynamic shared memory of k_gemm_tc_kfull<BN> for a given K: the tiles,
// padded like gemm_tc_smem so that at most 512 / BN CTAs share an SM.
template <int BN> inline size_t gemm_tc_kfull_smem(int K) {
    const size_t tiles = (size_t)(kTcM + BN) * K * 2;
    const size_t floor_ = 227 * 1024 / (512 / BN) + 1024;
    return tiles > floor_ ? tiles : floor_;
}
template <int BN> constexpr size_t gemm_tc_kfull_smem_max() {
    return (size_t)(kTcM + BN) * kTcKFull * 2 > 227 * 1024 / (512 / BN) + 1024
               ? (size_t)(kTcM + BN) * kTcKFull * 2
               : 227 * 1024 / (512 / BN) + 1024;
}

// Dynamic shared memory of k_gemm_tc<BN>: the two tiles, padded so that at
// most 512 / BN CTAs share an SM's 512 TMEM columns.
template <int BN> constexpr size_t gemm_tc_smem() {
    constexpr size_t tiles = (size_t)(kTcM + BN) * kTcK * 2;
    constexpr size_t per_sm = 227 * 1024;
    constexpr size_t floor_ = per_sm / (512 / BN) + 1024;
    return tiles > floor_ ? tiles : floor_;
}

}  // namespace mmk
