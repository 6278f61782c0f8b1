// fno.cu -- Fourier-neural-operator surrogate of the demag field: BF16
// storage, FP32 accumulation, forward, backward and Adam on the GPU.
//
// Not in the paper.  The network maps a magnetisation increment dM/Ms on an
// H x W film to its demag field H_demag(dM)/Ms (H_demag is linear in M, so
// between exact refreshes H_demag(M) = H_demag(M_ref) + Ms FNO((M-M_ref)/Ms)).
//   v0 = P [x; y/H; x/W] + p (two coordinate channels let the operator see
//   the film's edges);  for l < L: u = W_l v + b_l + S_l(v), v = gelu(u) (not on
//   the last layer);  y = Q v + q;  S_l keeps kx < m and ky in
//   {0..m-1} U {H-m..H-1}, with complex weights R_l[c][o] per mode.
// Dense contractions (the x-direction mode transforms, the channel mixes)
// run on the fifth-generation tensor cores (tcgen05 MMAs with the FP32
// accumulator in tensor memory, gemm_tc.cuh); the small complex transforms along y and the per-mode
// channel mix run as FP32 kernels.  Parameters live as an FP32 master copy
// (Adam moments beside it) and a BF16 copy for the GEMMs.
#include <cuda_bf16.h>
#include <cuda_pipeline.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mm.h"
#include "mm_internal.h"
#include "gemm_tc.cuh"

using namespace mmk;

namespace mmk {

// ------------------------------------------------------------ BF16 GEMM --
// The tcgen05 kernel of gemm_tc.cuh; the tile width follows N.  A product
// with fewer rows than a 128-row tile and more columns (the per-sample
// channel mix, C x C times C x HW) runs as its transpose C^T = B^T A^T.
// Launch with programmatic stream serialisation when `pdl` (the forward
// pass: every kernel of it waits on griddepcontrol before touching data
// and lets its successor launch right after that wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t s, bool pdl,
                            Args... args) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(grid, threads, smem, s, attr, pdl);
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

template <int BN> static cudaError_t gemm_launch(const GemmArgs& g, int batch, cudaStream_t s) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + kTcM - 1) / kTcM, batch);
    k_gemm_tc<BN><<<grid, kTcThreads, gemm_tc_smem<BN>(), s>>>(g);
    return cudaGetLastError();
}

template <int BN> static cudaError_t gemm_launch_kfull(const GemmArgs& g, int batch, cudaStream_t s, bool pdl) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + kTcM - 1) / kTcM, batch);
    return launch_k(k_gemm_tc_kfull<BN>, grid, kTcThreads, gemm_tc_kfull_smem<BN>(g.K), s, pdl, g);
}

// Both operands K-contiguous with 16-byte aligned rows and K a multiple of
// 16 up to kTcKFull: the all-of-K-resident kernel.
static bool gemm_kfull_ok(const GemmArgs& g) {
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return g.K > 0 && g.K % 16 == 0 && g.K <= kTcKFull && g.sak == 1 && g.sbk == 1 && g.sam % 8 == 0 &&
           g.sbn % 8 == 0 && g.zA % 8 == 0 && g.zB % 8 == 0 && al(g.A) && al(g.B);
}

static cudaError_t gemm(GemmArgs g, int batch, int* err, cudaStream_t s, bool pdl = false) {
    g.err = err;
    if (g.M < kTcM && g.N > g.M) {
        GemmArgs t = g;
        t.A = g.B; t.B = g.A; t.M = g.N; t.N = g.M;
        t.sam = g.sbn; t.sak = g.sbk; t.sbk = g.sak; t.sbn = g.sam;
        t.scm = g.scn; t.scn = g.scm; t.zA = g.zB; t.zB = g.zA;
        g = t;
    }
    // (the per-slice kernel has no programmatic wait: launched plainly, it
    // starts after its predecessor has finished)
    if (gemm_kfull_ok(g)) {
        if (g.N <= 32) return gemm_launch_kfull<32>(g, batch, s, pdl);
        if (g.N <= 64) return gemm_launch_kfull<64>(g, batch, s, pdl);
        return gemm_launch_kfull<128>(g, batch, s, pdl);
    }
    if (g.N <= 32) return gemm_launch<32>(g, batch, s);
    if (g.N <= 64) return gemm_launch<64>(g, batch, s);
    return gemm_launch<128>(g, batch, s);
}

__global__ void k_ydft_blk(const float* __restrict__ A, int ldA, int H, int m, const float* __restrict__ Fre,
                           const float* __restrict__ Fim, int ny_out, float* __restrict__ ore,
                           float* __restrict__ oim, float scale, int double_kx, int S);
constexpr int kYdftThreads = 256;
constexpr size_t kYdftSmemMax = 200 * 1024;

static cudaError_t gemm_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_tc_smem<32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem<64>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_tc_smem<128>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc_kfull<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_tc_kfull_smem_max<32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc_kfull<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_tc_kfull_smem_max<64>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc_kfull<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_tc_kfull_smem_max<128>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ydft_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYdftSmemMax);
    return e;
}

// ------------------------------------------------------ small FP32 kernels --
__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n, float scale) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(scale * in[i]);
}

// 1x1 channel map per pixel: out[b][o][p] = sum_c Wt[o][c] in[b][c][p] + bias[o]
// (trans: Wt stored [c][o], i.e. the transposed map)
__global__ void k_pointwise(const float* __restrict__ in, int cin, const float* __restrict__ Wt,
                            const float* __restrict__ bias, int cout, long long npix, int B, int trans,
                            float* __restrict__ outf) {
    const long long total = (long long)B * npix;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        const long long p = t - (long long)b * npix;
        float x[64];
        for (int c = 0; c < cin; ++c) x[c] = in[((long long)b * cin + c) * npix + p];
        for (int o = 0; o < cout; ++o) {
            float s = bias ? bias[o] : 0.f;
            for (int c = 0; c < cin; ++c) s += (trans ? Wt[c * cout + o] : Wt[o * cin + c]) * x[c];
            outf[((long long)b * cout + o) * npix + p] = s;
        }
    }
}

// y-direction transform of the x-mode coefficients (complex, FP32):
// out[b][c][iy][kx] = sum_y F[iy][y] * A[b][c][y][kx] (+/- conj by sign)
// A: re at [.. y][kx], im at [.. y][m + kx] with row stride ldA (= 2m).
// F: Fre/Fim (ny_out x H).  out: re/im planes [bc][iy][kx].
__global__ void k_ydft(const float* __restrict__ A, int ldA, int H, int m, const float* __restrict__ Fre,
                       const float* __restrict__ Fim, int ny_out, int BC, float* __restrict__ ore,
                       float* __restrict__ oim, float scale, int double_kx) {
    const long long total = (long long)BC * ny_out * m;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(t % m);
        const int iy = (int)((t / m) % ny_out);
        const long long bc = t / ((long long)m * ny_out);
        const float* a = A + bc * H * ldA;
        float sr = 0.f, si = 0.f;
        for (int y = 0; y < H; ++y) {
            const float fr = Fre[iy * H + y], fi = Fim[iy * H + y];
            const float ar = a[y * ldA + kx], ai = a[y * ldA + m + kx];
            sr += fr * ar - fi * ai;
            si += fr * ai + fi * ar;
        }
        const float sc = (double_kx && kx > 0) ? 2.f * scale : scale;
        ore[t] = sc * sr;
        oim[t] = sc * si;
    }
}

// The same transform, one block per (b, c, group of ny_out / G iy).  The
// block stages the (b, c) slab of A (H x 2m, contiguous) in shared memory
// with 16-byte asynchronous copies (all in flight at once); work item w <
// NT S takes the quad q = w % NT (iy = iy0 + q / mq, kx = 4 (q % mq) .. + 3)
// over the y share w / NT, and the S shares of each output are summed in
// order through shared memory.
__global__ void __launch_bounds__(kYdftThreads)
    k_ydft_blk(const float* __restrict__ A, int ldA, int H, int m, const float* __restrict__ Fre,
               const float* __restrict__ Fim, int ny_out, float* __restrict__ ore, float* __restrict__ oim,
               float scale, int double_kx, int S) {
    extern __shared__ __align__(16) float ys[];
    const int bc = blockIdx.x, m2 = 2 * m, mq = (m + 3) / 4;
    const int nyb = ny_out / gridDim.y, iy0 = blockIdx.y * nyb, NT = nyb * mq;
    float* sa = ys;                                        // [y][2m]
    float* part = ys + (((size_t)H * m2 + 3) & ~(size_t)3);   // [share][quad][4 re, 4 im]
    const float* a = A + (size_t)bc * H * ldA;
    pdl_wait();
    pdl_trigger();
    if (ldA == m2 && ((H * m2) & 3) == 0 && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
        for (int i = threadIdx.x; i < H * m2 / 4; i += blockDim.x)
            __pipeline_memcpy_async(sa + 4 * i, a + 4 * i, 16);
        __pipeline_commit();
        __pipeline_wait_prior(0);
    } else {
        for (int i = threadIdx.x; i < H * m2; i += blockDim.x) {
            const int y = i / m2, k = i - y * m2;
            sa[i] = a[(size_t)y * ldA + k];
        }
    }
    __syncthreads();
    const int yl = (H + S - 1) / S;
    for (int w = threadIdx.x; w < NT * S; w += blockDim.x) {
        const int q = w % NT, sh = w / NT;
        const int iy = iy0 + q / mq, k0 = 4 * (q % mq);
        const int y0 = sh * yl, y1 = min(H, y0 + yl);
        const float* fr = Fre + (size_t)iy * H;
        const float* fi = Fim + (size_t)iy * H;
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
        int y = y0;
        if (((H | yl) & 3) == 0) {                          // four y per F load
            for (; y + 3 < y1; y += 4) {
                const float4 c4 = __ldg(reinterpret_cast<const float4*>(fr + y));
                const float4 d4 = __ldg(reinterpret_cast<const float4*>(fi + y));
                const float crv[4] = {c4.x, c4.y, c4.z, c4.w}, civ[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float* row = sa + (y + u) * m2;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int kx = min(k0 + j, m - 1);  // lanes past m are dropped below
                        const float ar = row[kx], ai = row[m + kx];
                        sr[j] += crv[u] * ar - civ[u] * ai;
                        si[j] += crv[u] * ai + civ[u] * ar;
                    }
                }
            }
        }
        for (; y < y1; ++y) {
            const float cr = __ldg(fr + y), ci = __ldg(fi + y);
            const float* row = sa + y * m2;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kx = min(k0 + j, m - 1);
                const float ar = row[kx], ai = row[m + kx];
                sr[j] += cr * ar - ci * ai;
                si[j] += cr * ai + ci * ar;
            }
        }
        float* p = part + ((size_t)sh * NT + q) * 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p[j] = sr[j];
            p[4 + j] = si[j];
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nyb * m; o += blockDim.x) {
        const int il = o / m, kx = o - il * m;
        const int q = il * mq + kx / 4, j = kx % 4;
        float r = 0.f, im = 0.f;
        for (int sh = 0; sh < S; ++sh) {
            r += part[((size_t)sh * NT + q) * 8 + j];
            im += part[((size_t)sh * NT + q) * 8 + 4 + j];
        }
        const float sc = (double_kx && kx > 0) ? 2.f * scale : scale;
        const size_t oi = ((size_t)bc * ny_out + iy0 + il) * m + kx;
        ore[oi] = sc * r;
        oim[oi] = sc * im;
    }
}

// The per-mode channel mix and the inverse y transform of one output
// channel, one cluster of gridDim.y blocks per (b, o), block r of it taking
// the rows y of range r:
//   wh[iy][kx] = sum_c R[c][o][iy m + kx] vh[b][c][iy m + kx]
//   (conjT: sum_c conj(R[o][c][iy m + kx]) vh[b][c][iy m + kx]),
//   Zb[b][o][y][kx] = sum_iy G[y][iy] wh[iy][kx] in BF16 for the inverse x
//   GEMM (real parts at kx, imaginary parts at m + kx).
// Block r forms the modes of share r (nmode / gridDim.y of them; with
// `vec`, four modes per work item, eight lanes splitting c, float4 loads
// all issued together, the lanes combined by shuffles), the cluster
// exchanges the shares through distributed shared memory, and then each
// work item (y, kx quad) sums the 2m terms from shared memory.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float ld_cluster_f32(const float* local, int rank) {
    uint32_t ra;
    float v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}

__global__ void __launch_bounds__(256)
    k_mode_inv(const float* __restrict__ vhr, const float* __restrict__ vhi, const float* __restrict__ Rre,
               const float* __restrict__ Rim, int C, int m, int conjT, const float* __restrict__ Gre,
               const float* __restrict__ Gim, int H, __nv_bfloat16* __restrict__ Zb, int vec) {
    extern __shared__ __align__(16) float wsm[];
    const int nmode = 2 * m * m, nky = 2 * m, mq = (m + 3) / 4;
    const int bo = blockIdx.x, b = bo / C, o = bo - b * C;
    const int YS = gridDim.y, rank = blockIdx.y;           // the cluster spans gridDim.y
    const int share = nmode / YS, md0 = rank * share;
    float* wr = wsm;
    float* wi = wsm + nmode;
    pdl_wait();
    pdl_trigger();
    const float sgn = conjT ? -1.f : 1.f;
    if (vec) {
        constexpr int CG = 8;                              // lanes per four modes (adjacent lanes)
        for (int it = threadIdx.x; it < (share / 4) * CG; it += blockDim.x) {   // warp-uniform: share % 16 == 0
            const int md = md0 + 4 * (it / CG), cg = it % CG;
            float4 sr = make_float4(0.f, 0.f, 0.f, 0.f), si = sr;
#pragma unroll 4
            for (int c = cg; c < C; c += CG) {
                const long long ri = conjT ? ((long long)o * C + c) * nmode + md : ((long long)c * C + o) * nmode + md;
                const float4 rr = __ldg(reinterpret_cast<const float4*>(Rre + ri));
                float4 rm = __ldg(reinterpret_cast<const float4*>(Rim + ri));
                rm.x *= sgn;
                rm.y *= sgn;
                rm.z *= sgn;
                rm.w *= sgn;
                const long long vi = ((long long)b * C + c) * nmode + md;
                const float4 xr = __ldg(reinterpret_cast<const float4*>(vhr + vi));
                const float4 xi = __ldg(reinterpret_cast<const float4*>(vhi + vi));
                sr.x += rr.x * xr.x - rm.x * xi.x;
                sr.y += rr.y * xr.y - rm.y * xi.y;
                sr.z += rr.z * xr.z - rm.z * xi.z;
                sr.w += rr.w * xr.w - rm.w * xi.w;
                si.x += rr.x * xi.x + rm.x * xr.x;
                si.y += rr.y * xi.y + rm.y * xr.y;
                si.z += rr.z * xi.z + rm.z * xr.z;
                si.w += rr.w * xi.w + rm.w * xr.w;
            }
#pragma unroll
            for (int off = 1; off < CG; off <<= 1) {
                sr.x += __shfl_xor_sync(0xffffffffu, sr.x, off);
                sr.y += __shfl_xor_sync(0xffffffffu, sr.y, off);
                sr.z += __shfl_xor_sync(0xffffffffu, sr.z, off);
                sr.w += __shfl_xor_sync(0xffffffffu, sr.w, off);
                si.x += __shfl_xor_sync(0xffffffffu, si.x, off);
                si.y += __shfl_xor_sync(0xffffffffu, si.y, off);
                si.z += __shfl_xor_sync(0xffffffffu, si.z, off);
                si.w += __shfl_xor_sync(0xffffffffu, si.w, off);
            }
            if (cg == 0) {
                *reinterpret_cast<float4*>(wr + md) = sr;
                *reinterpret_cast<float4*>(wi + md) = si;
            }
        }
    } else {
        for (int md = md0 + threadIdx.x; md < md0 + share; md += blockDim.x) {
            float sr = 0.f, si = 0.f;
#pragma unroll 8
            for (int c = 0; c < C; ++c) {
                const long long ri = conjT ? ((long long)o * C + c) * nmode + md : ((long long)c * C + o) * nmode + md;
                const float rr = Rre[ri], rim = sgn * Rim[ri];
                const float xr = vhr[((long long)b * C + c) * nmode + md];
                const float xi = vhi[((long long)b * C + c) * nmode + md];
                sr += rr * xr - rim * xi;
                si += rr * xi + rim * xr;
            }
            wr[md] = sr;
            wi[md] = si;
        }
    }
    cluster_sync_all();                                    // every share formed
    for (int md = threadIdx.x; md < nmode; md += blockDim.x) {
        const int owner = md / share;
        if (owner == rank) continue;
        wr[md] = ld_cluster_f32(wr + md, owner);
        wi[md] = ld_cluster_f32(wi + md, owner);
    }
    cluster_sync_all();                                    // no share is read after its block moves on
    const int yr = (H + YS - 1) / YS, y0 = rank * yr;
    const int y1 = min(H, y0 + yr);
    for (int it = threadIdx.x; it < (y1 - y0) * mq; it += blockDim.x) {
        const int y = y0 + it / mq, k0 = 4 * (it % mq);
        const float* gr = Gre + (size_t)y * nky;
        const float* gi = Gim + (size_t)y * nky;
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
        // four iy per G load (a warp's lanes span several rows y); rows of
        // 2m floats start on 16 bytes for even m
        for (int i4 = 0; (nky & 3) == 0 && i4 < nky; i4 += 4) {
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(gr + i4));
            const float4 c4 = __ldg(reinterpret_cast<const float4*>(gi + i4));
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int iy = i4 + u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int kx = min(k0 + j, m - 1);     // lanes past m are not stored
                    const float xr = wr[iy * m + kx], xi = wi[iy * m + kx];
                    sr[j] += av[u] * xr - cv[u] * xi;
                    si[j] += av[u] * xi + cv[u] * xr;
                }
            }
        }
        for (int iy = 0; (nky & 3) != 0 && iy < nky; ++iy) {
            const float a = __ldg(gr + iy), c = __ldg(gi + iy);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kx = min(k0 + j, m - 1);
                const float xr = wr[iy * m + kx], xi = wi[iy * m + kx];
                sr[j] += a * xr - c * xi;
                si[j] += a * xi + c * xr;
            }
        }
        __nv_bfloat16* z = Zb + ((size_t)bo * H + y) * nky;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (k0 + j < m) {
                z[k0 + j] = __float2bfloat16(sr[j]);
                z[m + k0 + j] = __float2bfloat16(si[j]);
            }
    }
}

// dR[c][o][mode] += sum_b dw[b][o][mode] * conj(vh[b][c][mode])
__global__ void k_dR(const float* __restrict__ dwr, const float* __restrict__ dwi, const float* __restrict__ vr,
                     const float* __restrict__ vi, int C, int nmode, int B, float* __restrict__ gre,
                     float* __restrict__ gim) {
    const long long total = (long long)C * C * nmode;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int md = (int)(t % nmode);
        const int o = (int)((t / nmode) % C);
        const int c = (int)(t / ((long long)nmode * C));
        float sr = 0.f, si = 0.f;
        for (int b = 0; b < B; ++b) {
            const float gr = dwr[((long long)b * C + o) * nmode + md], gi = dwi[((long long)b * C + o) * nmode + md];
            const float ar = vr[((long long)b * C + c) * nmode + md], ai = -vi[((long long)b * C + c) * nmode + md];
            sr += gr * ar - gi * ai;
            si += gr * ai + gi * ar;
        }
        gre[t] += sr;
        gim[t] += si;
    }
}

// lift: out[b][o][p] = sum_{c<3} P[o][c] x[b][c][p] + P[o][3] y/H + P[o][4] x/W + bias[o]
__global__ void k_lift(const float* __restrict__ in, const float* __restrict__ P, const float* __restrict__ bias,
                       int C, int H, int W, int B, float* __restrict__ out, __nv_bfloat16* __restrict__ outb) {
    const long long np = (long long)H * W, total = (long long)B * np;
    pdl_wait();
    pdl_trigger();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / np);
        const long long p = t - (long long)b * np;
        const float x0 = in[((long long)b * 3 + 0) * np + p], x1 = in[((long long)b * 3 + 1) * np + p];
        const float x2 = in[((long long)b * 3 + 2) * np + p];
        const float cy = (float)(p / W) / (float)H, cx = (float)(p % W) / (float)W;
        for (int o = 0; o < C; ++o) {
            const float val =
                bias[o] + P[o * 5] * x0 + P[o * 5 + 1] * x1 + P[o * 5 + 2] * x2 + P[o * 5 + 3] * cy + P[o * 5 + 4] * cx;
            if (out) out[((long long)b * C + o) * np + p] = val;
            outb[((long long)b * C + o) * np + p] = __float2bfloat16(val);
        }
    }
}

// g[o][c] += sum_p dv[b][o][p] * feature_c(p), features 3 and 4 the coordinates
__global__ void k_outer_lift(const float* __restrict__ a, int C, const float* __restrict__ x, int H, int W, int B,
                             float* __restrict__ g) {
    const int o = blockIdx.y / 5, c = blockIdx.y % 5;
    const long long np = (long long)H * W;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * np;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / np);
        const long long p = t - (long long)b * np;
        const float f = c < 3 ? x[((long long)b * 3 + c) * np + p]
                              : (c == 3 ? (float)(p / W) / (float)H : (float)(p % W) / (float)W);
        acc += a[((long long)b * C + o) * np + p] * f;
    }
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + o * 5 + c, acc);
}

// u[b][o][p] += bias[o] (kept in u when keep_u, for the backward pass);
// v = gelu(u) when act, else u, in BF16 and, when vf is given, in FP32.
// Four pixels per thread where np is a multiple of 4.
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__global__ void k_bias_act(float* __restrict__ u, const float* __restrict__ bias, int C, long long np, int B,
                           __nv_bfloat16* __restrict__ v, float* __restrict__ vf, int keep_u, int act) {
    const long long n = (long long)B * C * np;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if ((np & 3) == 0) {
        for (long long i4 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i4 < n / 4; i4 += stride) {
            const float b = bias[(int)(((4 * i4) / np) % C)];
            float4 x = reinterpret_cast<const float4*>(u)[i4];
            x.x += b;
            x.y += b;
            x.z += b;
            x.w += b;
            if (keep_u) reinterpret_cast<float4*>(u)[i4] = x;
            const float4 y = act ? make_float4(gelu_f(x.x), gelu_f(x.y), gelu_f(x.z), gelu_f(x.w)) : x;
            reinterpret_cast<__nv_bfloat162*>(v)[2 * i4] = __floats2bfloat162_rn(y.x, y.y);
            reinterpret_cast<__nv_bfloat162*>(v)[2 * i4 + 1] = __floats2bfloat162_rn(y.z, y.w);
            if (vf) reinterpret_cast<float4*>(vf)[i4] = y;
        }
    } else {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const float x = u[i] + bias[(int)((i / np) % C)];
            if (keep_u) u[i] = x;
            const float y = act ? gelu_f(x) : x;
            v[i] = __float2bfloat16(y);
            if (vf) vf[i] = y;
        }
    }
}

// GELU with erf from Abramowitz & Stegun 7.1.26 (Hastings' rational
// approximation, |error of erf| <= 1.5e-7, far below the BF16 the
// activations are stored in): erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 +
// t a5)))) exp(-z^2), t = 1 / (1 + p z), z >= 0, odd in z.
__device__ __forceinline__ float gelu_as(float x) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.f, fmaf(0.3275911f, z, 1.f));
    float q = fmaf(1.061405429f, t, -1.453152027f);
    q = fmaf(q, t, 1.421413741f);
    q = fmaf(q, t, -0.284496736f);
    q = fmaf(q, t, 0.254829592f);
    const float e = 1.f - q * t * __expf(-z * z);        // erf(|x| / sqrt 2)
    return 0.5f * x * (1.f + copysignf(e, x));
}

// The tail of a layer for width CW:
// u[b][o][p] = S(v)[b][o][p] (in u) + sum_c W[o][c] v[b][c][p] + bias[o],
// kept in u when TRAIN; v' = gelu(u) except on the last layer (PROJ), in
// BF16 and, when TRAIN, in FP32.  The channel map is a CW x CW contraction
// per pixel, too small for the tensor cores to pay for the transposed copy
// of v their operand layout would need.  A block takes tiles of TP pixels
// x CW channels: the tile's v (BF16) and u rows are staged in shared memory
// with 16-byte loads issued together, W (FP32) once per block; thread
// (p, og) then forms the CW / OG outputs of group og at pixel p and stores
// them (consecutive threads, consecutive pixels).  PROJ (the last layer):
// no activation, and the projection y[b][j][p] = sum_o Q[j][o] v'[b][o][p]
// + q[j] (3 outputs) summed over the groups through shared memory, so that
// v' is not stored unless TRAIN.
template <int CW, bool PROJ, bool TRAIN>
__global__ void __launch_bounds__(256) k_mix_bias_act(float* __restrict__ u, const __nv_bfloat16* __restrict__ v,
                                                      const float* __restrict__ Wl, const float* __restrict__ bias,
                                                      long long np, int B, __nv_bfloat16* __restrict__ vout,
                                                      float* __restrict__ vf, const float* __restrict__ Q,
                                                      const float* __restrict__ qb, float* __restrict__ yout) {
    constexpr int T = 256, TP = CW <= 32 ? 64 : 32, OG = T / TP, OPG = CW / OG;
    static_assert(CW % OG == 0 && CW % 4 == 0, "output groups");
    __shared__ __align__(16) float Ws[CW * CW];
    __shared__ float bs[CW];
    __shared__ float Qs[PROJ ? 3 * CW + 3 : 1];
    __shared__ __align__(16) __nv_bfloat16 vs[CW * TP];
    __shared__ __align__(16) float us[CW * TP];
    __shared__ float ps[PROJ ? 3 * T : 1];
    pdl_wait();
    pdl_trigger();
    for (int i = threadIdx.x; i < CW * CW; i += T) Ws[i] = Wl[i];
    for (int i = threadIdx.x; i < CW; i += T) bs[i] = bias[i];
    if constexpr (PROJ) {
        for (int i = threadIdx.x; i < 3 * CW; i += T) Qs[i] = Q[i];
        if (threadIdx.x < 3) Qs[3 * CW + threadIdx.x] = qb[threadIdx.x];
    }
    const long long tpb = (np + TP - 1) / TP, ntiles = (long long)B * tpb;
    const bool vec = (np & 7) == 0;                        // 16-byte aligned tile rows
    const int p = threadIdx.x % TP, og = threadIdx.x / TP;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / tpb);
        const long long p0 = (tile - (long long)b * tpb) * TP;
        const int tw = (int)(np - p0 < TP ? np - p0 : TP);
        const long long base = (long long)b * CW * np + p0;
        __syncthreads();                                   // the previous tile's reads are done
        if (vec && tw == TP) {
            for (int e = threadIdx.x; e < CW * TP / 8; e += T) {
                const int c = e / (TP / 8), q = e - c * (TP / 8);
                reinterpret_cast<uint4*>(vs)[e] = *reinterpret_cast<const uint4*>(v + base + c * np + 8 * q);
            }
            for (int e = threadIdx.x; e < CW * TP / 4; e += T) {
                const int c = e / (TP / 4), q = e - c * (TP / 4);
                reinterpret_cast<float4*>(us)[e] = *reinterpret_cast<const float4*>(u + base + c * np + 4 * q);
            }
        } else {
            for (int e = threadIdx.x; e < CW * TP; e += T) {
                const int c = e / TP, q = e - c * TP;
                vs[e] = q < tw ? v[base + c * np + q] : __float2bfloat16(0.f);
                us[e] = q < tw ? u[base + c * np + q] : 0.f;
            }
        }
        __syncthreads();
        float xv[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) xv[c] = __bfloat162float(vs[c * TP + p]);
        float y0 = 0.f, y1 = 0.f, y2 = 0.f;
        const bool live = p < tw;
        const long long g0 = base + (long long)(og * OPG) * np + p;   // output og * OPG at this pixel
#pragma unroll 2
        for (int j = 0; j < OPG; ++j) {
            const int o = og * OPG + j;
            float acc = us[o * TP + p] + bs[o];
            const float4* w4 = reinterpret_cast<const float4*>(Ws + o * CW);
#pragma unroll
            for (int c4 = 0; c4 < CW / 4; ++c4) {
                const float4 w = w4[c4];
                acc = fmaf(w.x, xv[4 * c4], acc);
                acc = fmaf(w.y, xv[4 * c4 + 1], acc);
                acc = fmaf(w.z, xv[4 * c4 + 2], acc);
                acc = fmaf(w.w, xv[4 * c4 + 3], acc);
            }
            const float yv = PROJ ? acc : gelu_as(acc);
            if (live) {
                const long long gi = g0 + (long long)j * np;
                if constexpr (TRAIN) {
                    u[gi] = acc;
                    vf[gi] = yv;
                }
                if (!PROJ || TRAIN) vout[gi] = __float2bfloat16(yv);
            }
            if constexpr (PROJ) {
                y0 = fmaf(Qs[o], yv, y0);
                y1 = fmaf(Qs[CW + o], yv, y1);
                y2 = fmaf(Qs[2 * CW + o], yv, y2);
            }
        }
        if constexpr (PROJ) {
            ps[threadIdx.x] = y0;
            ps[T + threadIdx.x] = y1;
            ps[2 * T + threadIdx.x] = y2;
            __syncthreads();
            if (og == 0 && live) {
                float s0 = Qs[3 * CW], s1 = Qs[3 * CW + 1], s2 = Qs[3 * CW + 2];
                for (int g = 0; g < OG; ++g) {
                    s0 += ps[g * TP + p];
                    s1 += ps[T + g * TP + p];
                    s2 += ps[2 * T + g * TP + p];
                }
                const long long yb = (long long)b * 3 * np + p0 + p;
                yout[yb] = s0;
                yout[yb + np] = s1;
                yout[yb + 2 * np] = s2;
            }
        }
    }
}

// du = dv * gelu'(u)
__global__ void k_act_back(const float* __restrict__ u, float* __restrict__ dv, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = u[i];
        const float g = 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.3989422804014327f;
        dv[i] *= g;
    }
}

// loss = mean (y - t)^2 (partial sums, FP64 atomics) and dy = 2 (y - t) / n
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, long long n, float* __restrict__ dy,
                       double* __restrict__ loss) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        dy[i] = 2.f * d / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// sum over pixels of x[b][c][p] into g[c]
__global__ void k_colsum(const float* __restrict__ x, int C, long long npix, int B, float* __restrict__ g) {
    const int c = blockIdx.y;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * npix;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        acc += x[((long long)b * C + c) * npix + (t - (long long)b * npix)];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + c, acc);
}

// g[o][c] += sum_p a[b][o][p] x[b][c][p] (small channel counts, FP32)
__global__ void k_outer(const float* __restrict__ a, int Ca, const float* __restrict__ x, int Cx, long long npix, int B,
                        float* __restrict__ g) {
    const int o = blockIdx.y / Cx, c = blockIdx.y % Cx;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * npix;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        const long long p = t - (long long)b * npix;
        acc += a[((long long)b * Ca + o) * npix + p] * x[((long long)b * Cx + c) * npix + p];
    }
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + o * Cx + c, acc);
}

// Weight gradients of a per-pixel channel map: g[o][c] += sum_{b,p}
// a[b][o][p] f_c(b, p) for o < CA, c < CB, and, when gb, gb[o] += sum_{b,p}
// a[b][o][p].  f_c is xm[b][c][p], or with LIFT the lift's features (x[b][c][p]
// for c < 3, then y / H and x / W of pixel p).  A block reduces PCH pixels of
// one sample: 64-pixel tiles of a and f staged in shared memory with
// 16-byte loads, thread (pixel group, RO x RC output tile) accumulating in
// registers, the pixel groups summed through shared memory at the end, one
// atomic add per output and block.
template <int CA, int CB, bool LIFT>
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ a, const float* __restrict__ xm, int H, int W,
                                               long long np, int B, float* __restrict__ g, float* __restrict__ gb) {
    constexpr int T = 256, PCH = 2048;
    constexpr int RO = CA < 4 ? CA : 4, RC = CB == 5 ? 5 : 4;
    static_assert(CA % RO == 0 && CB % RC == 0, "output tiles");
    constexpr int NGO = CA / RO, NGC = CB / RC, GS = NGO * NGC, PG = T / GS;
    constexpr int TP = PG > 64 ? PG : 64;                  // pixels per staged tile
    static_assert(T % GS == 0 && TP % PG == 0 && PCH % TP == 0, "pixel groups");
    constexpr int NV = RO * RC + RO;                       // per-thread sums (outputs, then biases)
    constexpr int TS = TP + 1;                             // padded tile row: rows 4 apart in banks differ
    constexpr int SU = (CA + CB) * TS > T * NV ? (CA + CB) * TS : T * NV;
    __shared__ __align__(16) float su[SU];                 // tiles, then the group reduction
    float* as = su;
    float* fs = su + CA * TS;
    float* red = su;
    const long long cpb = (np + PCH - 1) / PCH;
    const int b = (int)(blockIdx.x / cpb);
    const long long c0 = (blockIdx.x - (long long)b * cpb) * PCH;
    const long long c1 = np - c0 < PCH ? np : c0 + PCH;
    const int gi = threadIdx.x % GS, pg = threadIdx.x / GS;
    const int o0 = (gi / NGC) * RO, k0 = (gi % NGC) * RC;
    float acc[RO][RC], bacc[RO];
#pragma unroll
    for (int i = 0; i < RO; ++i) {
        bacc[i] = 0.f;
#pragma unroll
        for (int j = 0; j < RC; ++j) acc[i][j] = 0.f;
    }
    const float* ab = a + (long long)b * CA * np;
    const bool vec = (np & 3) == 0;
    for (long long p0 = c0; p0 < c1; p0 += TP) {
        const int tw = (int)(c1 - p0 < TP ? c1 - p0 : TP);
        __syncthreads();
        if (vec && tw == TP) {
            for (int e = threadIdx.x; e < CA * TP / 4; e += T) {
                const int r = e / (TP / 4), q = e - r * (TP / 4);
                const float4 v4 = *reinterpret_cast<const float4*>(ab + r * np + p0 + 4 * q);
                float* d = as + r * TS + 4 * q;
                d[0] = v4.x;
                d[1] = v4.y;
                d[2] = v4.z;
                d[3] = v4.w;
            }
        } else {
            for (int e = threadIdx.x; e < CA * TP; e += T) {
                const int r = e / TP, q = e - r * TP;
                as[r * TS + q] = q < tw ? ab[r * np + p0 + q] : 0.f;
            }
        }
        for (int e = threadIdx.x; e < CB * TP; e += T) {
            const int r = e / TP, q = e - r * TP;
            const long long pp = p0 + q;
            float v = 0.f;
            if (q < tw) {
                if (LIFT && r >= 3)
                    v = r == 3 ? (float)(pp / W) / (float)H : (float)(pp % W) / (float)W;
                else
                    v = xm[((long long)b * (LIFT ? 3 : CB) + r) * np + pp];
            }
            fs[r * TS + q] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int q = pg; q < TP; q += PG) {
            float av[RO], fv[RC];
#pragma unroll
            for (int i = 0; i < RO; ++i) av[i] = as[(o0 + i) * TS + q];
#pragma unroll
            for (int j = 0; j < RC; ++j) fv[j] = fs[(k0 + j) * TS + q];
#pragma unroll
            for (int i = 0; i < RO; ++i) {
                bacc[i] += av[i];
#pragma unroll
                for (int j = 0; j < RC; ++j) acc[i][j] = fmaf(av[i], fv[j], acc[i][j]);
            }
        }
    }
    // sum the pixel groups: red[pg][gi][..] over the tiles' space
    __syncthreads();
    float* mine = red + (size_t)threadIdx.x * NV;
#pragma unroll
    for (int i = 0; i < RO; ++i) {
        mine[RO * RC + i] = bacc[i];
#pragma unroll
        for (int j = 0; j < RC; ++j) mine[i * RC + j] = acc[i][j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < GS * NV; e += T) {
        const int gg = e / NV, k = e - gg * NV;
        float sum = 0.f;
        for (int q = 0; q < PG; ++q) sum += red[((size_t)q * GS + gg) * NV + k];
        const int oo = (gg / NGC) * RO, kk = (gg % NGC) * RC;
        if (k < RO * RC)
            atomicAdd(g + (oo + k / RC) * CB + kk + k % RC, sum);
        else if (gb && gg % NGC == 0)
            atomicAdd(gb + oo + (k - RO * RC), sum);
    }
}

// Per-pixel channel map through a transposed matrix:
// out[b][j][p] = sum_i M[i][j] in[b][i][p] (M stored CI x CO), FP32.  Tiles
// of 64 pixels x CI channels staged in shared memory with 16-byte loads;
// thread (p, og) forms CO / OG outputs and stores them (consecutive
// threads, consecutive pixels).
template <int CI, int CO>
__global__ void __launch_bounds__(256) k_chanmap_t(const float* __restrict__ in, const float* __restrict__ M,
                                                   long long np, int B, float* __restrict__ out) {
    constexpr int T = 256, TP = 64, OG = T / TP, OPG = CO / OG;
    static_assert(CO % OG == 0, "output groups");
    constexpr int CP = (CI + 3) & ~3;                      // row of the transposed matrix, padded to 4
    __shared__ __align__(16) float Ms[CO * CP];            // Ms[j][i] = M[i][j]
    __shared__ __align__(16) float is[CI * TP];
    for (int e = threadIdx.x; e < CO * CP; e += T) {
        const int j = e / CP, i = e - j * CP;
        Ms[e] = i < CI ? M[i * CO + j] : 0.f;
    }
    const long long tpb = (np + TP - 1) / TP, ntiles = (long long)B * tpb;
    const bool vec = (np & 3) == 0;
    const int p = threadIdx.x % TP, og = threadIdx.x / TP;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / tpb);
        const long long p0 = (tile - (long long)b * tpb) * TP;
        const int tw = (int)(np - p0 < TP ? np - p0 : TP);
        const float* ib = in + (long long)b * CI * np + p0;
        __syncthreads();
        if (vec && tw == TP) {
            for (int e = threadIdx.x; e < CI * TP / 4; e += T) {
                const int r = e / (TP / 4), q = e - r * (TP / 4);
                reinterpret_cast<float4*>(is)[e] = *reinterpret_cast<const float4*>(ib + r * np + 4 * q);
            }
        } else {
            for (int e = threadIdx.x; e < CI * TP; e += T) {
                const int r = e / TP, q = e - r * TP;
                is[e] = q < tw ? ib[r * np + q] : 0.f;
            }
        }
        __syncthreads();
        if (p >= tw) continue;
        float xv[CP];
#pragma unroll
        for (int i = 0; i < CP; ++i) xv[i] = i < CI ? is[i * TP + p] : 0.f;
        float* ob = out + (long long)b * CO * np + p0 + p;
#pragma unroll 4
        for (int jj = 0; jj < OPG; ++jj) {
            const int j = og * OPG + jj;
            const float4* m4 = reinterpret_cast<const float4*>(Ms + j * CP);
            float acc = 0.f;
#pragma unroll
            for (int i4 = 0; i4 < CP / 4; ++i4) {
                const float4 w = m4[i4];
                acc = fmaf(w.x, xv[4 * i4], acc);
                acc = fmaf(w.y, xv[4 * i4 + 1], acc);
                acc = fmaf(w.z, xv[4 * i4 + 2], acc);
                acc = fmaf(w.w, xv[4 * i4 + 3], acc);
            }
            ob[(long long)j * np] = acc;
        }
    }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float s = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = s;
        w[i] -= lr * (a / c1) / (sqrtf(s / c2) + eps);
    }
}

}  // namespace mmk

// -------------------------------------------------------------- the model --
struct mm_fno {
    int H, W, C, m, L, Bmax;
    long long np;                 // pixels per channel
    cudaStream_t s;
    // parameters: FP32 master, gradient, Adam moments; layout
    // [P (C*5), p (C), R_re (L*C*C*2m*m), R_im, W (L*C*C), b (L*C), Q (3*C), q (3)]
    long long n_params;
    long long oP, op, oRr, oRi, oW, ob, oQ, oq;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16* wb = nullptr;  // BF16 copy of W (per layer C*C)
    bool wb_valid = false;        // wb matches w (cleared when w changes)
    // the inference forward as a graph, for one (batch, input, output)
    cudaStream_t cap = nullptr;   // private capture stream
    cudaGraphExec_t fwd_exec = nullptr;
    int fwd_B = 0;
    const float* fwd_x = nullptr;
    float* fwd_y = nullptr;
    int step = 0;
    // mode matrices, stored with the GEMMs' contraction index contiguous
    __nv_bfloat16* Fx = nullptr;    // [mode][x] (2m x W): cos | -sin (forward x, K = x)
    __nv_bfloat16* Gx = nullptr;    // [x][mode] (W x 2m): a cos/(HW) | -a sin/(HW) (inverse x, K = mode)
    __nv_bfloat16* Gxa = nullptr;   // [x][mode] (W x 2m): cos | -sin (adjoint of the forward x)
    float *Fyre = nullptr, *Fyim = nullptr;   // 2m x H: exp(-2 pi i ky y / H)
    float *Gyre = nullptr, *Gyim = nullptr;   // H x 2m: exp(+2 pi i ky y / H)
    // activations (per layer): v (bf16 + f32), u (f32), x-modes A1 (f32), vh re/im
    std::vector<float*> vf, u, A1, vhr, vhi;
    std::vector<__nv_bfloat16*> vb;
    float *Z = nullptr, *acc = nullptr, *y = nullptr, *dy = nullptr, *dv = nullptr,
          *du = nullptr, *tmp = nullptr, *dwr = nullptr, *dwi = nullptr;
    __nv_bfloat16 *zb = nullptr, *db16 = nullptr;
    double* dloss = nullptr;
    int* err = nullptr;           // set by a tensor-core GEMM whose wait expired
};

static int fno_fail(int code, const char* msg) { return set_error(code, msg); }

#define FCU(expr)                                                                                    \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) {                                                                     \
            char _m[256];                                                                            \
            snprintf(_m, sizeof(_m), "%s: %s", #expr, cudaGetErrorString(_e));                       \
            return fno_fail(_e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA, _m);             \
        }                                                                                            \
    } while (0)

static int grid1(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// deterministic N(0,1) samples: splitmix64 + Box-Muller
static uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double gauss(uint64_t& st) {
    const double u1 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
}

static void fno_free(mm_fno* f) {
    if (f->fwd_exec) cudaGraphExecDestroy(f->fwd_exec);
    if (f->cap) cudaStreamDestroy(f->cap);
    cudaFree(f->w); cudaFree(f->g); cudaFree(f->m1); cudaFree(f->m2); cudaFree(f->wb);
    cudaFree(f->Fx); cudaFree(f->Gx); cudaFree(f->Gxa);
    cudaFree(f->Fyre); cudaFree(f->Fyim); cudaFree(f->Gyre); cudaFree(f->Gyim);
    for (auto p : f->vf) cudaFree(p);
    for (auto p : f->u) cudaFree(p);
    for (auto p : f->A1) cudaFree(p);
    for (auto p : f->vhr) cudaFree(p);
    for (auto p : f->vhi) cudaFree(p);
    for (auto p : f->vb) cudaFree(p);
    cudaFree(f->Z); cudaFree(f->acc); cudaFree(f->y); cudaFree(f->dy);
    cudaFree(f->dv); cudaFree(f->du); cudaFree(f->tmp); cudaFree(f->dwr); cudaFree(f->dwi);
    cudaFree(f->zb); cudaFree(f->db16); cudaFree(f->dloss); cudaFree(f->err);
}

extern "C" int mm_fno_create(mm_fno** out, int H, int W, int width, int modes, int layers, int max_batch,
                             unsigned long long seed, void* stream) {
    if (!out) return fno_fail(MM_EINVAL, "out is NULL");
    *out = nullptr;
    if (H < 8 || W < 8 || width < 1 || width > 64 || modes < 1 || 2 * modes > H || 2 * modes >= W || layers < 1 ||
        max_batch < 1)
        return fno_fail(MM_EINVAL, "need H, W >= 8, 1 <= width <= 64, 2 modes <= H, 2 modes < W, layers, batch >= 1");
    mm_fno* f = new (std::nothrow) mm_fno();
    if (!f) return fno_fail(MM_ENOMEM, "host allocation failed");
    f->H = H; f->W = W; f->C = width; f->m = modes; f->L = layers; f->Bmax = max_batch;
    f->np = (long long)H * W;
    f->s = (cudaStream_t)stream;
    const int C = width, m = modes, L = layers;
    const long long nR = (long long)L * C * C * 2 * m * m;
    f->oP = 0; f->op = 5LL * C; f->oRr = f->op + C; f->oRi = f->oRr + nR; f->oW = f->oRi + nR;
    f->ob = f->oW + (long long)L * C * C; f->oQ = f->ob + (long long)L * C; f->oq = f->oQ + 3LL * C;
    f->n_params = f->oq + 3;
    int rc = [&]() -> int {
        const long long n = f->n_params;
        FCU(cudaMalloc(&f->w, 4 * n)); FCU(cudaMalloc(&f->g, 4 * n));
        FCU(cudaMalloc(&f->m1, 4 * n)); FCU(cudaMalloc(&f->m2, 4 * n));
        FCU(cudaMemset(f->m1, 0, 4 * n)); FCU(cudaMemset(f->m2, 0, 4 * n));
        FCU(cudaMalloc(&f->wb, 2LL * L * C * C));
        // seeded initial weights (scale as in the FP64 reference): P ~ N/sqrt5,
        // R ~ N/C, W ~ N/sqrt C, Q ~ N/sqrt C, biases 0
        std::vector<float> h(n, 0.f);
        uint64_t st = seed;
        for (long long i = 0; i < 5LL * C; ++i) h[f->oP + i] = (float)(gauss(st) / std::sqrt(5.0));
        for (long long i = 0; i < 2 * nR; ++i) h[f->oRr + i] = (float)(gauss(st) / C);
        for (long long i = 0; i < (long long)L * C * C; ++i) h[f->oW + i] = (float)(gauss(st) / std::sqrt((double)C));
        for (long long i = 0; i < 3LL * C; ++i) h[f->oQ + i] = (float)(gauss(st) / std::sqrt((double)C));
        FCU(cudaMemcpy(f->w, h.data(), 4 * n, cudaMemcpyHostToDevice));
        // mode matrices (FP64 -> BF16 / FP32)
        const double pi = 3.14159265358979323846;
        std::vector<__nv_bfloat16> fx((size_t)W * 2 * m), gx((size_t)2 * m * W), gxa((size_t)2 * m * W);
        for (int x = 0; x < W; ++x)
            for (int k = 0; k < m; ++k) {
                const double th = 2.0 * pi * k * x / W, a = (k == 0 ? 1.0 : 2.0) / ((double)H * W);
                fx[(size_t)k * W + x] = __float2bfloat16((float)std::cos(th));
                fx[(size_t)(m + k) * W + x] = __float2bfloat16((float)-std::sin(th));
                gx[(size_t)x * 2 * m + k] = __float2bfloat16((float)(a * std::cos(th)));
                gx[(size_t)x * 2 * m + m + k] = __float2bfloat16((float)(-a * std::sin(th)));
                gxa[(size_t)x * 2 * m + k] = __float2bfloat16((float)std::cos(th));
                gxa[(size_t)x * 2 * m + m + k] = __float2bfloat16((float)-std::sin(th));
            }
        std::vector<float> fyr((size_t)2 * m * H), fyi((size_t)2 * m * H), gyr((size_t)H * 2 * m), gyi((size_t)H * 2 * m);
        for (int iy = 0; iy < 2 * m; ++iy) {
            const int ky = iy < m ? iy : H - 2 * m + iy;
            for (int y = 0; y < H; ++y) {
                const double th = 2.0 * pi * ky * y / H;
                fyr[(size_t)iy * H + y] = (float)std::cos(th);
                fyi[(size_t)iy * H + y] = (float)-std::sin(th);
                gyr[(size_t)y * 2 * m + iy] = (float)std::cos(th);
                gyi[(size_t)y * 2 * m + iy] = (float)std::sin(th);
            }
        }
        FCU(cudaMalloc(&f->Fx, 2 * fx.size())); FCU(cudaMemcpy(f->Fx, fx.data(), 2 * fx.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gx, 2 * gx.size())); FCU(cudaMemcpy(f->Gx, gx.data(), 2 * gx.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gxa, 2 * gxa.size())); FCU(cudaMemcpy(f->Gxa, gxa.data(), 2 * gxa.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Fyre, 4 * fyr.size())); FCU(cudaMemcpy(f->Fyre, fyr.data(), 4 * fyr.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Fyim, 4 * fyi.size())); FCU(cudaMemcpy(f->Fyim, fyi.data(), 4 * fyi.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gyre, 4 * gyr.size())); FCU(cudaMemcpy(f->Gyre, gyr.data(), 4 * gyr.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gyim, 4 * gyi.size())); FCU(cudaMemcpy(f->Gyim, gyi.data(), 4 * gyi.size(), cudaMemcpyHostToDevice));
        const long long act = (long long)max_batch * C * f->np;
        const long long modes_n = (long long)max_batch * C * 2 * m * m;
        f->vf.resize(L + 1); f->vb.resize(L + 1); f->u.resize(L); f->A1.resize(L); f->vhr.resize(L); f->vhi.resize(L);
        for (int l = 0; l <= L; ++l) {
            FCU(cudaMalloc(&f->vf[l], 4 * act));
            FCU(cudaMalloc(&f->vb[l], 2 * act));
        }
        for (int l = 0; l < L; ++l) {
            FCU(cudaMalloc(&f->u[l], 4 * act));
            FCU(cudaMalloc(&f->A1[l], 4LL * max_batch * C * H * 2 * m));
            FCU(cudaMalloc(&f->vhr[l], 4 * modes_n));
            FCU(cudaMalloc(&f->vhi[l], 4 * modes_n));
        }
        FCU(cudaMalloc(&f->dwr, 4 * modes_n)); FCU(cudaMalloc(&f->dwi, 4 * modes_n));
        FCU(cudaMalloc(&f->Z, 4LL * max_batch * C * H * 2 * m));
        FCU(cudaMalloc(&f->zb, 2LL * max_batch * C * H * 2 * m));
        FCU(cudaMalloc(&f->acc, 4 * act)); FCU(cudaMalloc(&f->dv, 4 * act)); FCU(cudaMalloc(&f->du, 4 * act));
        FCU(cudaMalloc(&f->tmp, 4 * act)); FCU(cudaMalloc(&f->db16, 2 * act));
        FCU(cudaMalloc(&f->y, 4LL * max_batch * 3 * f->np)); FCU(cudaMalloc(&f->dy, 4LL * max_batch * 3 * f->np));
        FCU(cudaMalloc(&f->dloss, 8));
        FCU(cudaMalloc(&f->err, sizeof(int)));
        FCU(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking));
        FCU(cudaMemset(f->err, 0, sizeof(int)));
        FCU(gemm_configure());
        return MM_OK;
    }();
    if (rc != MM_OK) {
        fno_free(f);
        delete f;
        return rc;
    }
    *out = f;
    return MM_OK;
}

extern "C" int mm_fno_destroy(mm_fno* f) {
    if (!f) return MM_OK;
    cudaStreamSynchronize(f->s);
    fno_free(f);
    delete f;
    return MM_OK;
}

extern "C" long long mm_fno_param_count(const mm_fno* f) { return f ? f->n_params : -1; }

extern "C" int mm_fno_set_params(mm_fno* f, const float* p) {
    if (!f || !p) return fno_fail(MM_EINVAL, "null argument");
    FCU(cudaMemcpyAsync(f->w, p, 4 * f->n_params, cudaMemcpyDefault, f->s));
    f->wb_valid = false;
    FCU(cudaMemsetAsync(f->m1, 0, 4 * f->n_params, f->s));
    FCU(cudaMemsetAsync(f->m2, 0, 4 * f->n_params, f->s));
    FCU(cudaStreamSynchronize(f->s));
    f->step = 0;
    return MM_OK;
}

extern "C" int mm_fno_get_params(mm_fno* f, float* p) {
    if (!f || !p) return fno_fail(MM_EINVAL, "null argument");
    FCU(cudaMemcpyAsync(p, f->w, 4 * f->n_params, cudaMemcpyDefault, f->s));
    FCU(cudaStreamSynchronize(f->s));
    return MM_OK;
}

// The layer tail fused on the CUDA cores (k_mix_bias_act) for the widths it
// is instantiated for, with the projection to y on the last layer; false:
// the caller runs the tensor-core channel map, k_bias_act and k_pointwise.
template <int CW, bool PROJ, bool TRAIN>
static cudaError_t mix_launch_t(mm_fno* f, int l, int B, float* y, cudaStream_t s) {
    const int C = f->C;
    const long long np = f->np;
    constexpr int TP = CW <= 32 ? 64 : 32;                 // the kernel's pixels per tile
    const long long tiles = (long long)B * ((np + TP - 1) / TP);
    const dim3 grid((unsigned)(tiles < 152 * 8 ? tiles : 152 * 8));
    return launch_k(k_mix_bias_act<CW, PROJ, TRAIN>, grid, 256, 0, s, true, f->u[l], (const __nv_bfloat16*)f->vb[l],
                    (const float*)(f->w + f->oW + (long long)l * C * C), (const float*)(f->w + f->ob + (long long)l * C),
                    np, B, f->vb[l + 1], TRAIN ? f->vf[l + 1] : (float*)nullptr, (const float*)(f->w + f->oQ),
                    (const float*)(f->w + f->oq), y);
}

template <int CW>
static cudaError_t mix_launch(mm_fno* f, int l, int B, bool train, float* y, cudaStream_t s) {
    const bool last = l == f->L - 1;
    if (last) return train ? mix_launch_t<CW, true, true>(f, l, B, y, s) : mix_launch_t<CW, true, false>(f, l, B, y, s);
    return train ? mix_launch_t<CW, false, true>(f, l, B, y, s) : mix_launch_t<CW, false, false>(f, l, B, y, s);
}

static bool mix_tail(mm_fno* f, int l, int B, bool train, float* y, cudaStream_t s) {
    switch (f->C) {
        case 8: mix_launch<8>(f, l, B, train, y, s); return true;
        case 16: mix_launch<16>(f, l, B, train, y, s); return true;
        case 32: mix_launch<32>(f, l, B, train, y, s); return true;
        case 64: mix_launch<64>(f, l, B, train, y, s); return true;
        default: return false;
    }
}

// Mode mix + inverse y (k_mode_inv) of B samples from (vr, vi) into f->zb
// with the R of layer l (conjT: its adjoint): clusters of YS blocks per
// (b, o), YS chosen to spread over the SMs.
static cudaError_t mode_inv(const mm_fno* f, int l, int B, const float* vr, const float* vi, int conjT,
                            cudaStream_t s, bool pdl = false) {
    const int C = f->C, m = f->m, H = f->H, nmode = 2 * m * m;
    const long long ro = (long long)l * C * C * nmode;
    const float* Rr = f->w + f->oRr + ro;
    const float* Ri = f->w + f->oRi + ro;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec4 = nmode % 16 == 0 && al(Rr) && al(Ri) && al(vr) && al(vi);
    int YS = 1;
    while (B * C * YS < 128 && YS < 8 && H / (2 * YS) >= 8 && nmode % (2 * YS) == 0 &&
           (!vec4 || (nmode / (2 * YS)) % 16 == 0))
        YS *= 2;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = YS;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B * C, YS);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sizeof(float) * 2 * nmode;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_mode_inv, vr, vi, Rr, Ri, C, m, conjT, (const float*)f->Gyre,
                              (const float*)f->Gyim, H, f->zb, vec4 ? 1 : 0);
}

// y transform of the x-mode coefficients A ([bc][y][2m], BC slabs) into
// (ore, oim) [bc][2m][m]: one block per slab where the slab fits in shared
// memory, else one thread per output.
static cudaError_t ydft(const mm_fno* f, const float* A, int BC, float* ore, float* oim, float scale, int double_kx,
                        cudaStream_t s, bool pdl = false) {
    const int m = f->m, H = f->H, ny = 2 * m;
    // iy groups per slab: enough blocks to spread over the SMs
    int G = 1;
    while (BC * G < 128 && ny % (2 * G) == 0 && ny / (2 * G) >= 4) G *= 2;
    const int NT = (ny / G) * ((m + 3) / 4);
    int S = kYdftThreads / NT;
    S = S < 1 ? 1 : (S > 8 ? 8 : S);
    const size_t smem = sizeof(float) * ((((size_t)H * 2 * m + 3) & ~(size_t)3) + (size_t)S * NT * 8);
    if (smem <= kYdftSmemMax)
        return launch_k(k_ydft_blk, dim3(BC, G), kYdftThreads, smem, s, pdl, A, 2 * m, H, m, (const float*)f->Fyre,
                        (const float*)f->Fyim, ny, ore, oim, scale, double_kx, S);
    else
        k_ydft<<<grid1((long long)BC * ny * m), 256, 0, s>>>(A, 2 * m, H, m, f->Fyre, f->Fyim, ny, BC, ore, oim, scale,
                                                            double_kx);
    return cudaGetLastError();
}

// forward pass of B samples; x (B, 3, H, W) FP32 device; result in y
// (f->y when null).  train: keep what the backward pass reads (u with its
// bias, the FP32 activations); otherwise only the BF16 activations the next
// layer reads and the last layer's FP32 output.
static int fno_forward(mm_fno* f, int B, const float* x, bool train, float* y = nullptr) {
    const int C = f->C, m = f->m, L = f->L, H = f->H, W = f->W;
    const long long np = f->np, act = (long long)B * C * np;
    cudaStream_t s = f->s;
    // every kernel below waits for its predecessor programmatically (PDL)
    FCU(launch_k(k_lift, dim3(grid1(B * np)), 256, 0, s, true, x, (const float*)(f->w + f->oP),
                 (const float*)(f->w + f->op), C, H, W, B, train ? f->vf[0] : (float*)nullptr, f->vb[0]));
    float* yo = y ? y : f->y;
    bool projected = false;
    for (int l = 0; l < L; ++l) {
        // x modes: A1[(b,c,y)][2m] = v[(b,c,y)][x] . Fx[x][2m]
        GemmArgs g{};
        g.A = f->vb[l]; g.B = f->Fx; g.C = f->A1[l];
        g.M = B * C * H; g.N = 2 * m; g.K = W;
        g.sam = W; g.sak = 1; g.sbk = 1; g.sbn = W; g.scm = 2 * m; g.scn = 1;
        g.alpha = 1.f; g.beta = 0.f;
        FCU(gemm(g, 1, f->err, s, true));
        // y modes
        FCU(ydft(f, f->A1[l], B * C, f->vhr[l], f->vhi[l], 1.f, 0, s, true));
        // mode mix, back along y: Zb[(b,o,y)][2m]
        FCU(mode_inv(f, l, B, f->vhr[l], f->vhi[l], 0, s, true));
        // u = S(v): acc[(b,o,y)][x] = Z . Gx
        GemmArgs g2{};
        g2.A = f->zb; g2.B = f->Gx; g2.C = f->u[l];
        g2.M = B * C * H; g2.N = W; g2.K = 2 * m;
        g2.sam = 2 * m; g2.sak = 1; g2.sbk = 1; g2.sbn = 2 * m; g2.scm = W; g2.scn = 1;
        g2.alpha = 1.f; g2.beta = 0.f;
        FCU(gemm(g2, 1, f->err, s, true));
        // u += W_l v (per sample: (C x C) . (C x np)) + b_l, activation
        if (mix_tail(f, l, B, train, yo, s)) {
            projected = l == L - 1;
            continue;
        }
        if (!f->wb_valid) {                                // BF16 copy of the channel maps
            k_to_bf16<<<grid1((long long)L * C * C), 256, 0, s>>>(f->w + f->oW, f->wb, (long long)L * C * C, 1.f);
            f->wb_valid = true;
        }
        GemmArgs g3{};
        g3.A = f->wb + (long long)l * C * C; g3.B = f->vb[l]; g3.C = f->u[l];
        g3.M = C; g3.N = (int)np; g3.K = C;
        g3.sam = C; g3.sak = 1; g3.sbk = np; g3.sbn = 1; g3.scm = np; g3.scn = 1;
        g3.zA = 0; g3.zB = (long long)C * np; g3.zC = (long long)C * np;
        g3.alpha = 1.f; g3.beta = 1.f;
        FCU(gemm(g3, B, f->err, s));
        // + b_l, activation
        k_bias_act<<<grid1(act / 4 + 1), 256, 0, s>>>(f->u[l], f->w + f->ob + (long long)l * C, C, np, B, f->vb[l + 1],
                                                       (train || l == L - 1) ? f->vf[l + 1] : nullptr, train ? 1 : 0,
                                                       l < L - 1 ? 1 : 0);
    }
    if (!projected) k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->vf[L], C, f->w + f->oQ, f->w + f->oq, 3, np, B, 0, yo);
    FCU(cudaGetLastError());
    return MM_OK;
}

// backward pass for the batch whose forward pass is in f; t (B, 3, H, W)
// FP32 device; gradients into f->g, loss (FP64) into f->dloss.
// Tiled backward helpers for the widths they are instantiated for.
template <int CW>
static void bw_launch(mm_fno* f, int B, int which, int l, const float* a, const float* xm, const float* xin) {
    const long long np = f->np;
    const int C = f->C;
    const unsigned blocks = (unsigned)(B * ((np + 2047) / 2048));
    const long long tiles = (long long)B * ((np + 63) / 64);
    const unsigned cgrid = (unsigned)(tiles < 152 * 8 ? tiles : 152 * 8);
    cudaStream_t s = f->s;
    switch (which) {
        case 0:   // Q, q from dy and the last activations; dv = Q^T dy
            k_wgrad<3, CW, false><<<blocks, 256, 0, s>>>(a, xm, f->H, f->W, np, B, f->g + f->oQ, f->g + f->oq);
            k_chanmap_t<3, CW><<<cgrid, 256, 0, s>>>(a, f->w + f->oQ, np, B, f->dv);
            break;
        case 1:   // W_l, b_l from du and v_l; tmp = W_l^T du
            k_wgrad<CW, CW, false><<<blocks, 256, 0, s>>>(a, xm, f->H, f->W, np, B, f->g + f->oW + (long long)l * C * C,
                                                          f->g + f->ob + (long long)l * C);
            k_chanmap_t<CW, CW><<<cgrid, 256, 0, s>>>(a, f->w + f->oW + (long long)l * C * C, np, B, f->tmp);
            break;
        default:  // P, p from dv_0 and the lift's features
            k_wgrad<CW, 5, true><<<blocks, 256, 0, s>>>(a, xin, f->H, f->W, np, B, f->g + f->oP, f->g + f->op);
            break;
    }
}

static bool bw_tiled(mm_fno* f, int B, int which, int l, const float* a, const float* xm, const float* xin) {
    switch (f->C) {
        case 8: bw_launch<8>(f, B, which, l, a, xm, xin); return true;
        case 16: bw_launch<16>(f, B, which, l, a, xm, xin); return true;
        case 32: bw_launch<32>(f, B, which, l, a, xm, xin); return true;
        case 64: bw_launch<64>(f, B, which, l, a, xm, xin); return true;
        default: return false;
    }
}

static int fno_backward(mm_fno* f, int B, const float* x, const float* t) {
    const int C = f->C, m = f->m, L = f->L, H = f->H, W = f->W;
    const long long np = f->np, act = (long long)B * C * np, ny = (long long)B * 3 * np;
    const int nmode = 2 * m * m;
    cudaStream_t s = f->s;
    FCU(cudaMemsetAsync(f->g, 0, 4 * f->n_params, s));
    FCU(cudaMemsetAsync(f->dloss, 0, 8, s));
    k_loss<<<grid1(ny), 256, 0, s>>>(f->y, t, ny, f->dy, f->dloss);
    const int gx = 64;
    if (!bw_tiled(f, B, 0, 0, f->dy, f->vf[L], x)) {
        k_outer<<<dim3(gx, 3 * C), 256, 0, s>>>(f->dy, 3, f->vf[L], C, np, B, f->g + f->oQ);
        k_colsum<<<dim3(gx, 3), 256, 0, s>>>(f->dy, 3, np, B, f->g + f->oq);
        k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->dy, 3, f->w + f->oQ, nullptr, C, np, B, 1, f->dv);
    }
    for (int l = L - 1; l >= 0; --l) {
        if (l < L - 1) k_act_back<<<grid1(act), 256, 0, s>>>(f->u[l], f->dv, act);
        // dv now holds du for layer l
        if (!bw_tiled(f, B, 1, l, f->dv, f->vf[l], x)) {
            k_colsum<<<dim3(gx, C), 256, 0, s>>>(f->dv, C, np, B, f->g + f->ob + (long long)l * C);
            k_outer<<<dim3(gx, C * C), 256, 0, s>>>(f->dv, C, f->vf[l], C, np, B,
                                                     f->g + f->oW + (long long)l * C * C);
            k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->dv, C, f->w + f->oW + (long long)l * C * C, nullptr, C, np, B,
                                                       1, f->tmp);
        }
        // spectral path: dw = (a/(HW)) modes(du); dR += dw conj(vh); dvh = R^H dw
        k_to_bf16<<<grid1(act), 256, 0, s>>>(f->dv, f->db16, act, 1.f);
        GemmArgs g{};
        g.A = f->db16; g.B = f->Fx; g.C = f->Z;
        g.M = B * C * H; g.N = 2 * m; g.K = W;
        g.sam = W; g.sak = 1; g.sbk = 1; g.sbn = W; g.scm = 2 * m; g.scn = 1;
        g.alpha = 1.f; g.beta = 0.f;
        FCU(gemm(g, 1, f->err, s));
        FCU(ydft(f, f->Z, B * C, f->dwr, f->dwi, 1.f / ((float)H * W), 1, s));
        const long long ro = (long long)l * C * C * nmode;
        k_dR<<<grid1((long long)C * C * nmode), 256, 0, s>>>(f->dwr, f->dwi, f->vhr[l], f->vhi[l], C, nmode, B,
                                                             f->g + f->oRr + ro, f->g + f->oRi + ro);
        FCU(mode_inv(f, l, B, f->dwr, f->dwi, 1, s));
        GemmArgs g2{};
        g2.A = f->zb; g2.B = f->Gxa; g2.C = f->tmp;
        g2.M = B * C * H; g2.N = W; g2.K = 2 * m;
        g2.sam = 2 * m; g2.sak = 1; g2.sbk = 1; g2.sbn = 2 * m; g2.scm = W; g2.scn = 1;
        g2.alpha = 1.f; g2.beta = 1.f;
        FCU(gemm(g2, 1, f->err, s));
        float* t2 = f->dv;
        f->dv = f->tmp;
        f->tmp = t2;
    }
    if (!bw_tiled(f, B, 2, 0, f->dv, nullptr, x)) {
        k_outer_lift<<<dim3(gx, C * 5), 256, 0, s>>>(f->dv, C, x, H, W, B, f->g + f->oP);
        k_colsum<<<dim3(gx, C), 256, 0, s>>>(f->dv, C, np, B, f->g + f->op);
    }
    FCU(cudaGetLastError());
    return MM_OK;
}

// A tensor-core GEMM whose wait expired left its output incomplete; read
// after the stream has been synchronised.
static int fno_check_tc(const mm_fno* f) {
    int e = 0;
    FCU(cudaMemcpyAsync(&e, f->err, sizeof(int), cudaMemcpyDeviceToHost, f->s));
    FCU(cudaStreamSynchronize(f->s));
    if (e) return fno_fail(MM_ETIMEOUT, "a tensor-core GEMM wait timed out; the result is incomplete");
    return MM_OK;
}

static int fno_check_batch(const mm_fno* f, int B, const void* x, const void* y) {
    if (!f || !x || !y) return fno_fail(MM_EINVAL, "null argument");
    if (B < 1 || B > f->Bmax) return fno_fail(MM_EINVAL, "batch out of range");
    return MM_OK;
}

// The inference forward replayed from a graph captured on the private
// stream (kernel parameters are pointers: the network's weights are read at
// replay, so the graph stays valid until B, x or y change).  Widths without
// the fused layer tail run eagerly (their BF16 weight copy is refreshed
// lazily).
static int fno_forward_graph(mm_fno* f, int B, const float* x, float* y, cudaStream_t s) {
    const int C = f->C;
    if (!(C == 8 || C == 16 || C == 32 || C == 64)) {
        cudaStream_t keep = f->s;
        f->s = s;
        const int rc = fno_forward(f, B, x, false, y);
        f->s = keep;
        return rc;
    }
    if (!f->fwd_exec || f->fwd_B != B || f->fwd_x != x || f->fwd_y != y) {
        if (f->fwd_exec) {
            cudaGraphExecDestroy(f->fwd_exec);
            f->fwd_exec = nullptr;
        }
        cudaStream_t keep = f->s;
        f->s = f->cap;
        FCU(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = fno_forward(f, B, x, false, y);
        f->s = keep;
        cudaGraph_t gph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(f->cap, &gph);
        if (rc != MM_OK || e != cudaSuccess) {
            if (gph) cudaGraphDestroy(gph);
            return rc != MM_OK ? rc : fno_fail(MM_ECUDA, "capture of the forward pass failed");
        }
        const cudaError_t ei = cudaGraphInstantiate(&f->fwd_exec, gph, 0);
        cudaGraphDestroy(gph);
        FCU(ei);
        f->fwd_B = B;
        f->fwd_x = x;
        f->fwd_y = y;
    }
    FCU(cudaGraphLaunch(f->fwd_exec, s));
    return MM_OK;
}

extern "C" int mm_fno_forward(mm_fno* f, int B, const float* x, float* y) {
    int rc = fno_check_batch(f, B, x, y);
    if (rc != MM_OK) return rc;
    return fno_forward_graph(f, B, x, y, f->s);
}

extern "C" int mm_fno_grad(mm_fno* f, int B, const float* x, const float* t, double* loss, float* grad) {
    int rc = fno_check_batch(f, B, x, t);
    if (rc != MM_OK) return rc;
    rc = fno_forward(f, B, x, true);
    if (rc == MM_OK) rc = fno_backward(f, B, x, t);
    if (rc != MM_OK) return rc;
    if (grad) FCU(cudaMemcpyAsync(grad, f->g, 4 * f->n_params, cudaMemcpyDefault, f->s));
    double l = 0.0;
    FCU(cudaMemcpyAsync(&l, f->dloss, 8, cudaMemcpyDeviceToHost, f->s));
    FCU(cudaStreamSynchronize(f->s));
    rc = fno_check_tc(f);
    if (rc != MM_OK) return rc;
    if (loss) *loss = l / (3.0 * B * f->np);
    return MM_OK;
}

extern "C" int mm_fno_train_step(mm_fno* f, int B, const float* x, const float* t, float lr, double* loss) {
    int rc = fno_check_batch(f, B, x, t);
    if (rc != MM_OK) return rc;
    rc = fno_forward(f, B, x, true);
    if (rc == MM_OK) rc = fno_backward(f, B, x, t);
    if (rc != MM_OK) return rc;
    f->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, f->step), c2 = 1.f - (float)std::pow((double)b2, f->step);
    k_adam<<<grid1(f->n_params), 256, 0, f->s>>>(f->w, f->g, f->m1, f->m2, f->n_params, lr, b1, b2, c1, c2, 1e-8f);
    f->wb_valid = false;
    FCU(cudaGetLastError());
    if (loss) {
        double l = 0.0;
        FCU(cudaMemcpyAsync(&l, f->dloss, 8, cudaMemcpyDeviceToHost, f->s));
        FCU(cudaStreamSynchronize(f->s));
        rc = fno_check_tc(f);
        if (rc != MM_OK) return rc;
        *loss = l / (3.0 * B * f->np);
    }
    return MM_OK;
}

// error word of mm_gemm_bf16 (one per device image of the library)
static __device__ int g_gemm_err;

extern "C" int mm_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, long long sam,
                            long long sak, long long sbk, long long sbn, long long scm, long long scn, int batch,
                            long long zA, long long zB, long long zC, float alpha, float beta, int atomic,
                            void* cuda_stream) {
    if (!C || (K > 0 && (!A || !B))) return fno_fail(MM_EINVAL, "null argument");
    if (M < 1 || N < 1 || K < 0 || batch < 1 || batch > 65535 || M > 65535LL * kTcM || N > 65535LL * kTcM)
        return fno_fail(MM_EINVAL, "need M, N in 1..65535*128, K >= 0, batch in 1..65535");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* errp = nullptr;
    FCU(cudaGetSymbolAddress(&errp, g_gemm_err));
    FCU(gemm_configure());
    FCU(cudaMemsetAsync(errp, 0, sizeof(int), s));
    GemmArgs g{};
    g.A = (const __nv_bfloat16*)A; g.B = (const __nv_bfloat16*)B; g.C = C;
    g.M = M; g.N = N; g.K = K;
    g.sam = sam; g.sak = sak; g.sbk = sbk; g.sbn = sbn; g.scm = scm; g.scn = scn;
    g.zA = zA; g.zB = zB; g.zC = zC;
    g.alpha = alpha; g.beta = beta; g.atomic = atomic ? 1 : 0;
    FCU(gemm(g, batch, (int*)errp, s));
    int e = 0;
    FCU(cudaMemcpyAsync(&e, errp, sizeof(int), cudaMemcpyDeviceToHost, s));
    FCU(cudaStreamSynchronize(s));
    if (e) return fno_fail(MM_ETIMEOUT, "a tensor-core GEMM wait timed out; C is incomplete");
    return MM_OK;
}

namespace mmk {
// Forward of one sample for the surrogate stepper (x, y: 3 * H * W FP32 on
// the device), on stream s.
int fno_apply(mm_fno* f, const float* x, float* y, cudaStream_t s) { return fno_forward_graph(f, 1, x, y, s); }
bool fno_matches(const mm_fno* f, int nx, int ny, int nz) { return f && nz == 1 && f->W == nx && f->H == ny; }
}  // namespace mmk
