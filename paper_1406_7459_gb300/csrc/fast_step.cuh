// fast_step.cuh -- the two-kernel Euler step for power-of-two grids.
//
// Step n (spectrum S of M^n already formed):
//   K_A  k_plane_pdl   per kx plane: y FFT, the z part of the convolution
//                      as a direct sum over the nz layers with the (x, y)
//                      tensor spectrum of each z offset (exact, and cheaper
//                      than a length-2nz transform pair for nz <= 8), the
//                      tensor product (Eq. (15)), inverse y; S -> Sh.  The
//                      zero-padded exchange stencil of Eq. (4) rides in the
//                      same spectrum.
//   K_B  k_xstep_pdl   per (layer, row pair): inverse x C2R (Eq. (16)), the
//                      field and LLG update of Eqs. (2)-(6) with the Euler
//                      step and renormalisation, and then the forward x R2C
//                      (Eq. (14)) of the new rows into S, which is the
//                      first pass of step n+1.
// So a step is two kernels and M^{n+1} is never re-read for its transform.
//
// Both kernels are launched with programmatic dependent launch.  Before
// `griddepcontrol.wait` each one only touches data that no kernel of the
// previous step writes: K_A prefetches the twiddles (its tensor-spectrum
// slice follows its S lines, after the wait, so that a cold start streams
// the transforms' inputs first); K_B prefetches twiddles and its M^n tile
// (M^n was written two launches earlier, and K_A triggers its dependents
// only once it has passed its own wait, which orders it after that writer).  Each kernel triggers
// after its last global store (or K_A right after its wait, see
// early_trigger), so the next kernel's launch and prologue overlap its tail.
#pragma once
#include <cuda_pipeline.h>

#include "bulk_copy.cuh"
#include "fast_passes.cuh"

namespace mmk {


// 16-byte asynchronous copies global -> shared (both 16-byte aligned).
__device__ __forceinline__ void copy16(void* dst, const void* src) { __pipeline_memcpy_async(dst, src, 16); }

template <int a, int b> struct cmax { static constexpr int v = a > b ? a : b; };

// Rows of one x-step tile (row pairs pack two real rows into one complex
// transform).  Both kernels keep the spectrum as [kx][c][k][j]: a plane
// reads and writes whole lines, an x-step tile gathers and scatters R-row
// runs (32 bytes for four rows: one sector per (c, kx)).
constexpr int kStepRows = 4;

// The plane kernel lets the x-step launch right after its own wait
// (early_trigger != 0) or only at its end.  Early: x-step blocks start on the
// SMs that hold one plane block (their registers allow one x-step block
// beside a plane block, two once it has left, so no SM ends up with three)
// and fetch their twiddles and M tile while the planes run.  The plan picks
// it where it measured faster (fast_step_early_trigger).

// ------------------------------------------------------------- K_A plane --
template <int NY, int NZ> struct PlaneLayout {
    using F = Fft2<NY>;
    static constexpr int LY = 2 * NY, NL = 3 * NZ;
    // a line is two halves [h] of F::EX slots: the first NY of a half hold
    // its data in natural order, all F::EX serve as the padded exchange of
    // that half's transform (Fft2::store_ex / stepB)
    static constexpr int HALF = F::EX;
    static constexpr int ZS = 2 * HALF;                   // line stride
    static constexpr int HY = NY + 1;
    static constexpr int HYP = kd_row(HY);                // row of the 2-D spectrum, 16-byte multiple
    static constexpr int KY_EVEN = (HY + 1) / 2;          // even ky' stored first in a row, then odd
    static constexpr int KT_FLOATS = HYP * NZ * 6;        // one kx slice of the 2-D spectrum,
    // [dz*6 + c][ky] as stored, so that consecutive threads (consecutive ky)
    // read consecutive words
    static constexpr int KT_C = KT_FLOATS / 2;            // in float2 units
    static constexpr int WORK = NL * ZS;
    static constexpr int TW_OFF = 0, TA_OFF = LY, KT_OFF = LY + NY, WORK_OFF = KT_OFF + ((KT_C + 1) / 2) * 2;
    static constexpr size_t BYTES = sizeof(float2) * (WORK_OFF + WORK);
    static constexpr int THREADS = 2 * NL * F::G;
};

// Lanes of the calling thread's warp that exist in a block of T threads
// (the last warp of a block whose size is not a multiple of 32 is partial).
template <int T> __device__ __forceinline__ unsigned warp_lanes() {
    if constexpr (T % 32 == 0) return 0xffffffffu;
    const int base = threadIdx.x & ~31;
    const int n = T - base < 32 ? T - base : 32;
    return n == 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// ta[a Q + t] = W_N^{t a} = tw[2 t a] from the W_2N table tw (both in
// shared memory; visible to the block after its next barrier).
template <int N, int Q, int T>
__device__ __forceinline__ void fill_ta(float2* ta, const float2* tw) {
#pragma unroll
    for (int i = threadIdx.x; i < N; i += T) {
        const int a = i / Q, tt = i - a * Q;
        ta[i] = tw[2 * tt * a];
    }
}

// Direct z sum of one (kx, ky) column for output component a, with
// M_z' = i M_z and H_z' = i H_z (real couplings, see k_pack2d):
//   H'_a(k) = sum_k' sum_b D_ab(k - k') M'_b(k'),
// D(dz) from the stored d(|dz|) = (xx, xy, xz, yy, yz, zz): row x uses
// (xx, xy, xz), row y (xy, yy, yz), row z' (-xz, -yz, zz); xz and yz change
// sign for dz < 0 (odd in z) and xy, yz for a mirrored ky (odd in y).
// coef(dz, c) gives d_c(dz) with the ky mirror sign already applied.
template <int NZ, class Coef>
__device__ __forceinline__ void zdirect_task(const float2 (&m)[3][NZ], Coef coef, int a, float2 (&h)[NZ]) {
#pragma unroll
    for (int k = 0; k < NZ; ++k) h[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz) {
        const float xx = coef(dz, 0), xy = coef(dz, 1), xz = coef(dz, 2);
        const float yy = coef(dz, 3), yz = coef(dz, 4), zz = coef(dz, 5);
        float cb0, cb1, cb2;                              // D_a,b for b = x, y, z' at +dz
        float ob0, ob1, ob2;                              // sign-adjusted for -dz
        if (a == 0) { cb0 = xx; cb1 = xy; cb2 = xz; ob0 = xx; ob1 = xy; ob2 = -xz; }
        else if (a == 1) { cb0 = xy; cb1 = yy; cb2 = yz; ob0 = xy; ob1 = yy; ob2 = -yz; }
        else { cb0 = -xz; cb1 = -yz; cb2 = zz; ob0 = xz; ob1 = yz; ob2 = zz; }
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            // k - k' = +dz  -> k' = k - dz
            if (k - dz >= 0) {
                const int kp = k - dz;
                h[k] = cfma_real(cb0, m[0][kp], h[k]);
                h[k] = cfma_real(cb1, m[1][kp], h[k]);
                h[k] = cfma_real(cb2, m[2][kp], h[k]);
            }
            // k - k' = -dz (dz > 0) -> k' = k + dz
            if (dz > 0 && k + dz < NZ) {
                const int kp = k + dz;
                h[k] = cfma_real(ob0, m[0][kp], h[k]);
                h[k] = cfma_real(ob1, m[1][kp], h[k]);
                h[k] = cfma_real(ob2, m[2][kp], h[k]);
            }
        }
    }
}

// The plane work of K_A for plane kx.  The plane's S lines are on their way
// into the first halves of the shared lines zb (bulk copies counted on
// barrier b_s, phase parity par); tw, ta are in shared memory (and visible
// after the first block barrier here), the 2-D spectrum slice Ks after
// barrier b_k (phase 0).  2 NL groups of G threads, one per (line, half);
// threads beyond them (T larger than the plane's own block) only help in
// the z sum.  Each group transforms its half of a line in place in its own
// half of zb (warp barriers only); block barriers separate the forward
// transforms, the z sum (which reads all lines of a column) and the inverse
// transforms.  Returns false, uniformly over the block, when a copy wait gave
// up (or ok_in is false); nothing is written to Sh then.
template <int NY, int NZ, int T>
__device__ __forceinline__ bool plane_body(const Geom& g, int kx, bool ok_in, const float2* tw, const float2* ta,
                                           const float* Ks, float2* zb, uint32_t b_s, uint32_t par, uint32_t b_k,
                                           float2* __restrict__ Sh) {
    using Lay = PlaneLayout<NY, NZ>;
    using F = Fft2<NY>;
    constexpr int P = F::P, Q = F::Q, G = F::G, LY = Lay::LY, ZS = Lay::ZS, NL = Lay::NL, HALF = Lay::HALF;
    static_assert(T >= Lay::THREADS, "block smaller than the plane's groups");
    const unsigned lanes = warp_lanes<T>();
    const bool act = T == Lay::THREADS || threadIdx.x < Lay::THREADS;
    bool ok = ok_in;
    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int line = grp >> 1, h = grp & 1;               // inverse y: a line's halves in one warp
    // forward y: where the groups of a warp can share the half, they do, so
    // that the odd half's twiddle multiply does not diverge within a warp
    constexpr int GW = G <= 32 ? 32 / G : 1;              // groups per warp
    constexpr bool UNI = GW >= 2 && NL % GW == 0;
    int lf = line, hf = h;
    if constexpr (UNI) {
        const int wq = grp / GW, s = grp % GW;
        hf = wq & 1;
        lf = (wq >> 1) * GW + s;
    }
    ok = ok && mbar_wait(b_s, par);
    float2 v[P];
    if (ok && act && t < Q) {
        const float2* src = zb + lf * ZS;                 // both halves' groups read the line
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = src[t + Q * q];
    }
    if (__syncthreads_or(!ok)) return false;
    // forward y (pruned input): odd half pre-multiplied by W_LY^j; the
    // group's own half-line is its exchange buffer
    float2* rf = zb + lf * ZS + hf * HALF;
    if (act && t < Q) {
        if (hf) F::odd_input_tab(v, t, tw);
        F::stepA_tab(v, t, ta, rf, false);
    }
    __syncwarp(lanes);
    float2 w[Q];
    if (act && t < P) F::stepB(w, t, rf, false);
    __syncwarp(lanes);
    if (act && t < P) {
#pragma unroll
        for (int q = 0; q < Q; ++q) rf[t + P * q] = w[q];
    }
    if (__syncthreads_or(!mbar_wait(b_k, 0))) return false;   // 2-D spectrum slice
    // z part of the convolution: direct sum over the layers, one (ky)
    // column per task, read and written back by the same thread
#pragma unroll
    for (int col = threadIdx.x; col < LY; col += T) {
        const int hh = col / NY, mm = col - hh * NY;      // ky = 2 mm + hh
        const int ky = 2 * mm + hh;
        const int e = hh * HALF + mm;
        float2 m[3][NZ];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < NZ; ++k) m[c][k] = zb[(c * NZ + k) * ZS + e];
#pragma unroll
        for (int k = 0; k < NZ; ++k) m[2][k] = make_float2(-m[2][k].y, m[2][k].x);   // i M_z
        int kyp = ky;
        float sy = 1.f;
        if (2 * ky > LY) { kyp = LY - ky; sy = -1.f; }
        // the stored row: even ky' first, then odd (same parity as ky)
        kyp = (kyp & 1) ? Lay::KY_EVEN + (kyp >> 1) : (kyp >> 1);
        // the column's couplings: read once for the three output components
        // when registers allow (nz <= 4), else per component
        constexpr bool HOIST = NZ <= 4;
        float d[HOIST ? NZ : 1][6];
        if constexpr (HOIST) {
#pragma unroll
            for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    d[dz][c] = (c == 1 || c == 4 ? sy : 1.f) * Ks[(dz * 6 + c) * Lay::HYP + kyp];
        }
        auto coef = [&](int dz, int c) -> float {
            if constexpr (HOIST) return d[dz][c];
            return (c == 1 || c == 4 ? sy : 1.f) * Ks[(dz * 6 + c) * Lay::HYP + kyp];
        };
        float2 hres[NZ];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            zdirect_task<NZ>(m, coef, a, hres);
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                const float2 o = (a == 2) ? make_float2(hres[k].y, -hres[k].x) : hres[k];   // -i H_z'
                zb[(a * NZ + k) * ZS + e] = o;
            }
        }
    }
    __syncthreads();
    // inverse y (pruned output), in place in the group's own half-line
    float2* ri = zb + line * ZS + h * HALF;
    if (act && t < Q) {
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = ri[t + Q * q];
    }
    __syncwarp(lanes);
    if (act && t < Q) F::stepA_tab(v, t, ta, ri, true);
    __syncwarp(lanes);
    if (act && t < P) {
        F::stepB(w, t, ri, true);
        if (h) F::odd_output_tab(w, t, tw);
    }
    float2* outp = Sh + (size_t)kx * NL * g.Jst;
    if constexpr (G == 16) {
        // the two halves of a line are lanes t and t + 16 of one warp
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float ox = __shfl_down_sync(0xffffffffu, w[q].x, 16);
            const float oy = __shfl_down_sync(0xffffffffu, w[q].y, 16);
            if (act && h == 0) outp[(size_t)line * g.Jst + t + P * q] = make_float2(w[q].x + ox, w[q].y + oy);
        }
    } else {
        // halves in different warps: through the shared lines
        __syncwarp(lanes);
        if (act && t < P) {
#pragma unroll
            for (int q = 0; q < Q; ++q) ri[t + P * q] = w[q];
        }
        __syncthreads();
#pragma unroll
        for (int idx = threadIdx.x; idx < NL * NY; idx += T) {
            const int l = idx / NY, n = idx % NY;
            outp[(size_t)l * g.Jst + n] = cadd(zb[l * ZS + n], zb[l * ZS + HALF + n]);
        }
    }
    return true;
}

// K_A as a kernel: one kx plane per CTA.
template <int NY, int NZ>
__global__ void __launch_bounds__(PlaneLayout<NY, NZ>::THREADS, (PlaneLayout<NY, NZ>::THREADS <= 512) ? 2 : 1)
    k_plane_pdl(const __grid_constant__ Geom g, const float* __restrict__ Kd, const float2* __restrict__ S,
                float2* __restrict__ Sh, int* __restrict__ flag, int early_trigger) {
    using Lay = PlaneLayout<NY, NZ>;
    using F = Fft2<NY>;
    constexpr int Q = F::Q, LY = Lay::LY, ZS = Lay::ZS, NL = Lay::NL;
    constexpr int T = Lay::THREADS;                       // the launch's block size
    extern __shared__ __align__(16) float2 sm[];
    __shared__ __align__(8) uint64_t bars[3];             // twiddles, S lines, spectrum slice
    float2* tw = sm + Lay::TW_OFF;
    float2* ta = sm + Lay::TA_OFF;
    float* Ks = reinterpret_cast<float*>(sm + Lay::KT_OFF);
    float2* zb = sm + Lay::WORK_OFF;
    const int kx = blockIdx.x;
    const uint32_t b_tw = smem_addr(&bars[0]), b_s = smem_addr(&bars[1]), b_k = smem_addr(&bars[2]);

    // prologue: bulk copies by one thread.  The twiddles (constant data)
    // before the wait; after it the plane's S lines (each into the first half
    // of its shared line), then this kx's slice of the 2-D spectrum, which
    // only the z sum needs: a cold start streams the transforms' inputs first
    if (threadIdx.x == 0) {
        mbar_init(b_tw, 1);
        mbar_init(b_s, 1);
        mbar_init(b_k, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(b_tw, LY * sizeof(float2));
        bulk_g2s(smem_addr(tw), g.twy, LY * sizeof(float2), b_tw);
    }
    pdl_wait();
    // S of the previous x-step is complete: the next kernel may launch and
    // run its prologue (it reads nothing this kernel writes before its own wait)
    if (early_trigger) pdl_trigger();
    if (threadIdx.x == 0) {
        proxy_fence_global();                             // S came from ordinary stores
        const float2* plane = S + (size_t)kx * NL * g.Jst;
        mbar_expect_tx(b_s, NL * NY * sizeof(float2));
#pragma unroll 1
        for (int l = 0; l < NL; ++l) bulk_g2s(smem_addr(zb + l * ZS), plane + (size_t)l * g.Jst, NY * sizeof(float2), b_s);
        mbar_expect_tx(b_k, Lay::KT_FLOATS * sizeof(float));
        bulk_g2s(smem_addr(Ks), Kd + (size_t)kx * Lay::KT_FLOATS, Lay::KT_FLOATS * sizeof(float), b_k);
    }
    const bool ok = mbar_wait(b_tw, 0);
    if (ok) fill_ta<NY, Q, T>(ta, tw);
    if (!plane_body<NY, NZ, T>(g, kx, ok, tw, ta, Ks, zb, b_s, 0, b_k, Sh)) {
        // a wait gave up: every thread leaves together, once the copies in
        // flight have landed (bounded again)
        if (threadIdx.x == 0) {
            atomicOr(flag, kFlagTimeout);
            mbar_wait(b_tw, 0);
            mbar_wait(b_s, 0);
            mbar_wait(b_k, 0);
        }
        __syncthreads();
        return;
    }
    if (!early_trigger) pdl_trigger();
}

// ------------------------------------------------------------- K_B xstep --
template <int N, int R> struct XstepLayout {
    static_assert(R == 2 || R == 4, "row pairs per tile: a pair shares one complex transform");
    using F = Fft2<N>;
    static constexpr int L = 2 * N, H = N + 1, NL = 3 * R / 2;
    static constexpr int HM = N / 2 + 1;                  // staged kx per parity: kx = 2 m + parity
    static constexpr int HP = 2 * HM;                     // staged positions per component
    static constexpr int HOFF = N + 8;                    // odd-kx half of a forward line, shifted by
                                                          // 64 bytes against the even half
    static constexpr int ZS = N + HOFF + 4;               // forward line stride: the split's two row
                                                          // pairs of a half-warp 32 bytes apart in banks
    static constexpr int MROWS = R;                        // rows of the M tile per component
    static constexpr int TW_OFF = 0, TA_OFF = L;
    static constexpr int MT_OFF = L + N;                          // float2 units; floats: 3*MROWS*N
    static constexpr int MT_C = 3 * MROWS * N / 2;
    static constexpr int SB_OFF = MT_OFF + MT_C;                  // staged spectrum / new M rows
    static constexpr int SB_C = cmax<3 * HP * R, 3 * R * N / 2>::v;
    static constexpr int W_OFF = SB_OFF + ((SB_C + 1) / 2) * 2;
    static constexpr int W_C = cmax<cmax<2 * NL * F::EX, NL * L>::v, NL * ZS>::v;
    static constexpr int BAR_OFF = W_OFF + W_C;                   // mbarrier of the tiled gather
    static constexpr size_t BYTES = sizeof(float2) * (BAR_OFF + 2);
    // one tile's box of the tiled gather / scatter: 2R floats of each of
    // the 3 HP (c, parity, kx / 2) positions
    static constexpr uint32_t BOX_BYTES = 3 * HP * R * sizeof(float2);
    static_assert((SB_OFF * sizeof(float2)) % 128 == 0, "staged spectrum on 128 bytes (tiled copies)");
    static constexpr int THREADS = cmax<2 * NL * F::G, 128>::v;
};

// Tiled tensor copies of the x-step's spectrum traffic: `in` gathers the
// tile's rows of Sh into sb (one box per tile, counted on the shared
// mbarrier `bar`), `out` scatters the next spectrum from sb to Snext.  The
// box of both maps is the layout sb has anyway, [c][kx parity][kx / 2][2R
// floats of rows j0 ..], so the arithmetic between them is unchanged.  Null
// maps: 16-byte asynchronous copies per thread and plain stores.
struct XTma {
    const CUtensorMap* in = nullptr;
    const CUtensorMap* out = nullptr;
    uint32_t bar = 0;
};

// MODE kModeStep: the Euler step (M^{n+1} replaces M^n in Mt and goes to
// Mout when Mout is given; Snext = its x spectrum); kModeHeff: Mout = H_eff
// of M (Sh from the spectrum with the exchange stencil folded in);
// kModeDemag: Mout = H_demag (Sh from the plain tensor spectrum, Mt unused).
// Snext, flag and Mcopy (a second destination of M^{n+1}, may be null) are
// used by the step only.
//
// The x-step work for tile `tile` (layer k, rows j0 .. j0 + R - 1): tw, ta
// (x twiddles) and, except for kModeDemag, the tile's M^n rows Mt
// (floats [c][row][i]) are in shared memory or on their way there as
// 16-byte asynchronous copies of this thread (the gather below waits for
// all of them).  sb stages the tile's rows of Sh, wk the transforms.
template <int N, int R, int MODE, int T>
__device__ __forceinline__ void xstep_body(const Geom& g, const LlgCoef& cf, int tile, const float2* tw,
                                           const float2* ta, float* Mt, float2* sb, float2* wk,
                                           const float2* __restrict__ Sh, float2* __restrict__ Snext,
                                           float* __restrict__ Mout, int* __restrict__ flag,
                                           float* __restrict__ Mcopy = nullptr, const XTma& xt = XTma{}) {
    using Lay = XstepLayout<N, R>;
    using F = Fft2<N>;
    constexpr int P = F::P, Q = F::Q, G = F::G, L = Lay::L, H = Lay::H, NL = Lay::NL, ZS = Lay::ZS;
    constexpr int HM = Lay::HM, HP = Lay::HP, HOFF = Lay::HOFF;
    constexpr int RP = R / 2;                             // row pairs of the tile
    static_assert(T >= 2 * NL * G, "block smaller than the tile's transform groups");
    const int ntj = g.ny / R;
    const int jt = tile % ntj;
    const int k = tile / ntj;
    const int j0 = jt * R;
    // 32-bit offsets: the plan admits this kernel only when 3 (nx + 1) nz ny
    // complex values and 3 nx ny nz floats index below 2^31
    const int Nc = g.N;
    const int plane_xy = N * g.ny;
    const int s_c = g.nz * g.Jst, s_kx = 3 * s_c;            // spectrum strides of c and kx
    const int s_base = k * g.Jst + j0;

    // staged half-spectrum of the tile, split by the parity of kx:
    // s4[(c * HP + pos(kx)) * RP + pr] = rows (j0 + 2 pr, j0 + 2 pr + 1) of
    // (c, kx), pos(kx) = (kx & 1) HM + kx / 2, so that the inverse transform
    // below reads consecutive 16-byte words (every RP-th one); the RP chunks
    // of one (c, kx) are adjacent in global memory and go to adjacent lanes.
    // With a tiled map the same layout is one box: the odd-parity position
    // kx / 2 = HM - 1 (kx = N + 1) reads the buffer's pad plane and is never
    // used.
    if (xt.in) {
        if (threadIdx.x == 0) {
            proxy_fence_global();                          // Sh: ordinary stores of the previous kernel
            mbar_expect_tx(xt.bar, Lay::BOX_BYTES);
            tensor_g2s_4d(smem_addr(sb), xt.in, 2 * s_base, 0, 0, 0, xt.bar);
        }
        __pipeline_commit();
        __pipeline_wait_prior(0);
        const bool ok = mbar_wait(xt.bar, 0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                if (flag) atomicOr(flag, kFlagTimeout);
                mbar_wait(xt.bar, 0);                      // the copy in flight lands first (bounded)
            }
            return;
        }
    } else {
#pragma unroll
        for (int idx = threadIdx.x; idx < 3 * H * RP; idx += T) {
            const int pr = idx % RP, ck = idx / RP;
            const int c = ck / H, kx = ck - c * H;
            copy16(sb + ((c * HP + (kx & 1) * HM + (kx >> 1)) * RP + pr) * 2,
                   Sh + kx * s_kx + c * s_c + s_base + 2 * pr);
        }
        __pipeline_commit();
        __pipeline_wait_prior(0);
        __syncthreads();
    }

    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int line = grp >> 1, h = grp & 1;                 // line = c * RP + pr
    const int lc = line / RP, pr = line % RP;
    const bool fft_thread = grp < 2 * NL;
    float2 v[P];
    float2 w[Q];
    // ---- inverse x: rebuild Z = A + iB (A, B the rows' half-spectra) at
    // kk = 2 m + h, m = t + Q q: kk <= N reads kx = kk, above it the mirror
    // kx = L - kk conjugated.  Only q = P/2 straddles kk = N.
    if (fft_thread && t < Q) {
        const float4* s4 = reinterpret_cast<const float4*>(sb) + (size_t)lc * HP * RP + pr;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int m = t + Q * q;
            const bool low = q < P / 2 ? true : (q > P / 2 ? false : (h == 0 && t == 0));
            const int pos = low ? h * HM + m : (h ? HM + N - 1 - m : N - m);
            float4 ab = s4[pos * RP];
            if ((q == 0 || q == P / 2) && h == 0 && t == 0) {   // kx = 0 and N: real
                ab.y = 0.f;
                ab.w = 0.f;
            }
            v[q] = low ? make_float2(ab.x - ab.w, ab.y + ab.z) : make_float2(ab.x + ab.w, ab.z - ab.y);
        }
        F::stepA_tab(v, t, ta, wk + grp * F::EX, true);
    }
    __syncthreads();
    if (fft_thread && t < P) {
        F::stepB(w, t, wk + grp * F::EX, true);
        if (h) F::odd_output_tab(w, t, tw);
    }
    __syncthreads();
    if constexpr (G == 16) {
        // halves of a line sit in lanes t and t + 16 of one warp: combine
        // by shuffle and keep only the sum, ob[line][n]
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float ox = __shfl_down_sync(0xffffffffu, w[q].x, 16);
            const float oy = __shfl_down_sync(0xffffffffu, w[q].y, 16);
            if (fft_thread && h == 0) wk[line * L + t + P * q] = make_float2(w[q].x + ox, w[q].y + oy);
        }
    } else {
        if (fft_thread && t < P) {
#pragma unroll
            for (int q = 0; q < Q; ++q) wk[line * L + h * N + t + P * q] = w[q];   // ob[line][h][n]
        }
        __syncthreads();
#pragma unroll
        for (int idx = threadIdx.x; idx < NL * N; idx += T) {
            const int ln = idx / N, n = idx % N;
            wk[ln * L + n] = cadd(wk[ln * L + n], wk[ln * L + N + n]);
        }
    }
    __syncthreads();
    // ---- field, LLG, Euler, renormalisation per cell; new rows to Mt.
    // The spectrum carries the zero-padded exchange stencil; a cell on a
    // free face lacks that neighbour, whose term in Eq. (4) is M(i) itself
    // (zero change), so each missing neighbour adds pexch M(i) / delta^2.
    const float bz = cf.pexch * (float)((g.nz > 1) * ((k == 0) + (k == g.nz - 1))) * cf.idz2;
#pragma unroll
    for (int idx = threadIdx.x; idx < R * N; idx += T) {
        const int r = idx / N;
        const int i = idx % N;
        const int j = j0 + r;
        float hd[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const float2 z = wk[(cc * RP + (r >> 1)) * L + i];   // pair line of rows (r & ~1, r | 1)
            hd[cc] = (r & 1) ? z.y : z.x;
        }
        const int cell = i + N * (j0 + r) + plane_xy * k;
        if constexpr (MODE == kModeDemag) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) Mout[cc * Nc + cell] = hd[cc];
            continue;
        }
        const float bnd = bz + cf.pexch * ((float)((i == 0) + (i == N - 1)) * cf.idx2 +
                                           (float)((g.ny > 1) * ((j == 0) + (j == g.ny - 1))) * cf.idy2);
        float m[3], hh[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const float m0 = Mt[(cc * R + r) * N + i];
            m[cc] = m0;
            hh[cc] = hd[cc] + bnd * m0;
        }
        hh[0] += cf.hx;
        hh[1] += cf.panis * m[1] + cf.hy;
        hh[2] += cf.panis * m[2] + cf.hz;
        if constexpr (MODE == kModeHeff) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) Mout[cc * Nc + cell] = hh[cc];
            continue;
        }
        const float p0 = m[1] * hh[2] - m[2] * hh[1];
        const float p1 = m[2] * hh[0] - m[0] * hh[2];
        const float p2 = m[0] * hh[1] - m[1] * hh[0];
        const float q0 = m[1] * p2 - m[2] * p1;
        const float q1 = m[2] * p0 - m[0] * p2;
        const float q2 = m[0] * p1 - m[1] * p0;
        const float n0 = m[0] + cf.dt * (cf.c1 * p0 + cf.c2 * q0);
        const float n1 = m[1] + cf.dt * (cf.c1 * p1 + cf.c2 * q1);
        const float n2 = m[2] + cf.dt * (cf.c1 * p2 + cf.c2 * q2);
        const float s = cf.Ms * rsqrtf(n0 * n0 + n1 * n1 + n2 * n2);
        const float o0 = n0 * s, o1 = n1 * s, o2 = n2 * s;
        if (!isfinite(o0 + o1 + o2)) atomicOr(flag, kFlagNonFinite);   // |o| <= Ms when finite
        if (Mout) {
            Mout[cell] = o0;
            Mout[Nc + cell] = o1;
            Mout[2 * Nc + cell] = o2;
        }
        if (Mcopy) {                                       // e.g. a host buffer, written over the link
            Mcopy[cell] = o0;
            Mcopy[Nc + cell] = o1;
            Mcopy[2 * Nc + cell] = o2;
        }
        // M^{n+1} replaces M^n in the tile (this thread read its own cell above)
        Mt[(0 * R + r) * N + i] = o0;
        Mt[(1 * R + r) * N + i] = o1;
        Mt[(2 * R + r) * N + i] = o2;
    }
    __syncthreads();
    if constexpr (MODE == kModeStep) {
        // ---- forward x of the new rows (first pass of the next step)
        if (fft_thread && t < Q) {
            const float* ra = Mt + (size_t)(lc * R + 2 * pr) * N;
            const float* rb = ra + N;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int jx = t + Q * q;
                v[q] = make_float2(ra[jx], rb[jx]);
            }
            if (h) F::odd_input_tab(v, t, tw);
            F::stepA_tab(v, t, ta, wk + grp * F::EX, false);
        }
        __syncthreads();
        if (fft_thread && t < P) F::stepB(w, t, wk + grp * F::EX, false);
        __syncthreads();
        if (fft_thread && t < P) {
#pragma unroll
            for (int q = 0; q < Q; ++q) wk[line * ZS + h * HOFF + t + P * q] = w[q];   // Z[2 n + h]
        }
        __syncthreads();
        // split each pair into the two rows' half-spectra and store to Snext
        // (the RP pairs of one (c, kx) are adjacent in global memory and go
        // to adjacent lanes), or stage them in sb, free since the inverse
        // transform, for one tiled store
#pragma unroll
        for (int idx = threadIdx.x; idx < 3 * H * RP; idx += T) {
            const int p2 = idx % RP, ck = idx / RP;
            const int c = ck / H, kx = ck - c * H;
            const float2* ln = wk + (c * RP + p2) * ZS;
            const int km = (L - kx) & (L - 1);
            const float2 zk = ln[(kx & 1) * HOFF + (kx >> 1)];
            const float2 zm = ln[(km & 1) * HOFF + (km >> 1)];
            const float4 o = make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y),
                                         0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            if (xt.out)
                reinterpret_cast<float4*>(sb)[(c * HP + (kx & 1) * HM + (kx >> 1)) * RP + p2] = o;
            else
                *reinterpret_cast<float4*>(Snext + kx * s_kx + c * s_c + s_base + 2 * p2) = o;
        }
        if (xt.out) {
            proxy_fence_shared();                          // this thread's staging stores, then the copy
            __syncthreads();
            if (threadIdx.x == 0) {
                tensor_s2g_4d(xt.out, 2 * s_base, 0, 0, 0, smem_addr(sb));
                bulk_commit();
                bulk_wait_all();                           // written before the block leaves
            }
        }
    }
}

// Fill the tile's M^n rows (floats [c][row][i]) with 16-byte asynchronous
// copies (committed with the caller's next group).
template <int N, int R, int T>
__device__ __forceinline__ void load_mtile(const Geom& g, int tile, const float* __restrict__ M, float* Mt) {
    constexpr int CH = N / 4;                               // 16-byte chunks per row
    const int ntj = g.ny / R;
    const int k = tile / ntj, j0 = (tile % ntj) * R;
#pragma unroll
    for (int idx = threadIdx.x; idx < 3 * R * CH; idx += T) {
        const int ch = idx % CH;
        const int row = (idx / CH) % R;
        const int c = idx / (CH * R);
        copy16(Mt + (c * R + row) * N + 4 * ch, M + (size_t)c * g.N + (size_t)k * N * g.ny + (j0 + row) * N + 4 * ch);
    }
}

// K_B as a kernel: one (layer, R rows) tile per CTA.
template <int N, int R, int MODE>
__global__ void __launch_bounds__(XstepLayout<N, R>::THREADS)
    k_xstep_pdl(const __grid_constant__ Geom g, const __grid_constant__ LlgCoef cf, const float2* __restrict__ Sh,
                float2* __restrict__ Snext, const float* __restrict__ M, float* __restrict__ Mout,
                int* __restrict__ flag, float* __restrict__ Mcopy) {
    using Lay = XstepLayout<N, R>;
    using F = Fft2<N>;
    constexpr int L = Lay::L;
    constexpr int T = Lay::THREADS;                       // the launch's block size
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm + Lay::TW_OFF;
    float2* ta = sm + Lay::TA_OFF;
    float* Mt = reinterpret_cast<float*>(sm + Lay::MT_OFF);
    float2* sb = sm + Lay::SB_OFF;
    float2* wk = sm + Lay::W_OFF;
    // prologue: twiddles and the tile's own M^n rows, which no kernel of
    // this step writes.  The exchange stencil of Eq. (4) is folded into the
    // 2-D spectrum as the zero-padded stencil, so no neighbour rows are
    // needed; what remains of the free-boundary rule is local (see the field
    // loop of xstep_body).
#pragma unroll
    for (int i = threadIdx.x; i < L / 2; i += T) copy16(tw + 2 * i, g.twx + 2 * i);
    F::template load_ta<T>(ta, g.twx);
    if constexpr (MODE != kModeDemag) load_mtile<N, R, T>(g, blockIdx.x, M, Mt);
    __pipeline_commit();
    pdl_wait();
    xstep_body<N, R, MODE, T>(g, cf, blockIdx.x, tw, ta, Mt, sb, wk, Sh, Snext, Mout, flag, Mcopy);
    __syncthreads();
    pdl_trigger();
}

// K_B with its spectrum gather (from Sh; bit 0 of `use`) and, for the step,
// its scatter (to Snext; bit 1) as tiled tensor copies through `tin` and
// `tout`, maps encoded for exactly those buffers (encode_xstep_maps).
template <int N, int R, int MODE>
__global__ void __launch_bounds__(XstepLayout<N, R>::THREADS)
    k_xstep_tma(const __grid_constant__ Geom g, const __grid_constant__ LlgCoef cf, const float2* __restrict__ Sh,
                float2* __restrict__ Snext, const float* __restrict__ M, float* __restrict__ Mout,
                int* __restrict__ flag, float* __restrict__ Mcopy, const __grid_constant__ CUtensorMap tin,
                const __grid_constant__ CUtensorMap tout, int use) {
    using Lay = XstepLayout<N, R>;
    using F = Fft2<N>;
    constexpr int L = Lay::L;
    constexpr int T = Lay::THREADS;
    extern __shared__ __align__(128) float2 sm[];
    float2* tw = sm + Lay::TW_OFF;
    float2* ta = sm + Lay::TA_OFF;
    float* Mt = reinterpret_cast<float*>(sm + Lay::MT_OFF);
    float2* sb = sm + Lay::SB_OFF;
    float2* wk = sm + Lay::W_OFF;
    const uint32_t bar = smem_addr(sm + Lay::BAR_OFF);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
        tensor_prefetch(&tin);
        if (MODE == kModeStep && (use & 2)) tensor_prefetch(&tout);
    }
    __syncthreads();
#pragma unroll
    for (int i = threadIdx.x; i < L / 2; i += T) copy16(tw + 2 * i, g.twx + 2 * i);
    F::template load_ta<T>(ta, g.twx);
    if constexpr (MODE != kModeDemag) load_mtile<N, R, T>(g, blockIdx.x, M, Mt);
    __pipeline_commit();
    pdl_wait();
    // the tiled copies want the box on 128 bytes (the layout puts it there;
    // the per-thread copies serve otherwise)
    XTma xt;
    if ((smem_addr(sb) & 127u) == 0) {
        xt.in = (use & 1) ? &tin : nullptr;
        xt.out = MODE == kModeStep && (use & 2) ? &tout : nullptr;
        xt.bar = bar;
    }
    xstep_body<N, R, MODE, T>(g, cf, blockIdx.x, tw, ta, Mt, sb, wk, Sh, Snext, Mout, flag, Mcopy, xt);
    __syncthreads();
    pdl_trigger();
}

}  // namespace mmk
