// step_persist.cuh -- the power-of-two Euler step as one persistent
// cooperative kernel: K_A phase -> grid barrier -> K_B phase, for n steps
// in one launch.
//
// Each block owns at most one kx plane (K_A work) and one (layer, R rows)
// tile (K_B work) for the whole launch, so what those need and what does
// not change between steps stays in shared memory: the y and x twiddles,
// the plane's slice of the 2-D tensor spectrum and the tile's M rows (M^n
// in, M^{n+1} written over it by the update, copied to global memory only
// after the last step).  Per step the only global traffic is the spectrum
// S (read by the planes with bulk copies) and Sh (written by the planes,
// gathered by the tiles), which is what the convolution's transposes must
// move.  The arithmetic is the two-kernel step's, in the same order
// (plane_body and xstep_body of fast_step.cuh), so both give the same bits.
//
// The grid barrier (grid_sync) is an arrival counter in global memory that
// grows through the launch.  Its waits are bounded by a poll limit given
// per launch: a wait that runs out records kFlagTimeout, waits (bounded) for
// the block's bulk copies in flight and leaves; the other blocks then run
// out at their next barrier and leave too.  The last block to leave resets
// the counters, so the next launch starts clean even after a timeout.  The
// launch must make every block co-resident (cooperative launch attribute).
#pragma once
#include "fast_step.cuh"
#include "grid_sync.cuh"

namespace mmk {

// Shared memory of the persistent step (float2 units; every region starts
// on 16 bytes).  Resident: y twiddles and their table, the plane's 2-D
// spectrum slice, x twiddles and their table, the tile's M rows.  Then one
// region used in turn by the plane (lines zb) and the tile (staged Sh rows
// sb, transforms wk).
template <int NY, int NZ, int NX, int R> struct PersistLayout {
    using A = PlaneLayout<NY, NZ>;
    using B = XstepLayout<NX, R>;
    static constexpr int T = cmax<A::THREADS, B::THREADS>::v;
    static constexpr int TWY = 0;
    static constexpr int TAY = TWY + A::LY;
    static constexpr int KS = TAY + NY;
    static constexpr int TWX = KS + ((A::KT_C + 1) / 2) * 2;
    static constexpr int TAX = TWX + 2 * NX;
    static constexpr int MT = TAX + NX;
    static constexpr int U = MT + B::MT_C;
    static constexpr int SB_C = ((3 * B::HP * R + 1) / 2) * 2;
    static constexpr int WK = U + SB_C;
    static constexpr int U_C = cmax<A::WORK, SB_C + B::W_C>::v;
    static constexpr size_t BYTES = sizeof(float2) * (U + U_C);
};

template <int NY, int NZ, int NX, int R>
__global__ void __launch_bounds__(PersistLayout<NY, NZ, NX, R>::T, 2)
    k_step_persist(const __grid_constant__ Geom g, const __grid_constant__ LlgCoef cf, const float* __restrict__ Kd, float2* S, float2* Sh,
                   const float* __restrict__ Min, float* __restrict__ Mout, int nsteps, int* __restrict__ flag,
                   GridBar* __restrict__ gb, long long wait_limit) {
    using Lay = PersistLayout<NY, NZ, NX, R>;
    using LA = PlaneLayout<NY, NZ>;
    constexpr int T = Lay::T, NL = LA::NL, ZS = LA::ZS;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ __align__(8) uint64_t bars[4];             // twiddles, spectrum slice, M tile, S lines
    float2* twy = sm + Lay::TWY;
    float2* tay = sm + Lay::TAY;
    float* Ks = reinterpret_cast<float*>(sm + Lay::KS);
    float2* twx = sm + Lay::TWX;
    float2* tax = sm + Lay::TAX;
    float* Mt = reinterpret_cast<float*>(sm + Lay::MT);
    float2* zb = sm + Lay::U;
    float2* sb = sm + Lay::U;
    float2* wk = sm + Lay::WK;
    const int blk = blockIdx.x;
    const int ntj = g.ny / R;
    const bool has_plane = blk < g.Hx, has_tile = blk < g.nz * ntj;
    const uint32_t b_tw = smem_addr(&bars[0]), b_k = smem_addr(&bars[1]), b_m = smem_addr(&bars[2]),
                   b_s = smem_addr(&bars[3]);
    const float2* plane = S + (size_t)blk * NL * g.Jst;

    if (threadIdx.x == 0) {
        mbar_init(b_tw, 1);
        mbar_init(b_k, 1);
        mbar_init(b_m, 1);
        mbar_init(b_s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // set-up copies, all at once: twiddles, the plane's first S lines, its
    // spectrum slice, the tile's M^n rows (each component's R rows are one
    // contiguous run)
    if (threadIdx.x == 0) {
        proxy_fence_global();
        mbar_expect_tx(b_tw, (LA::LY + 2 * NX) * sizeof(float2));
        bulk_g2s(smem_addr(twy), g.twy, LA::LY * sizeof(float2), b_tw);
        bulk_g2s(smem_addr(twx), g.twx, 2 * NX * sizeof(float2), b_tw);
        if (has_plane) {
            mbar_expect_tx(b_s, NL * NY * sizeof(float2));
#pragma unroll 1
            for (int l = 0; l < NL; ++l)
                bulk_g2s(smem_addr(zb + l * ZS), plane + (size_t)l * g.Jst, NY * sizeof(float2), b_s);
            mbar_expect_tx(b_k, LA::KT_FLOATS * sizeof(float));
            bulk_g2s(smem_addr(Ks), Kd + (size_t)blk * LA::KT_FLOATS, LA::KT_FLOATS * sizeof(float), b_k);
        }
        if (has_tile) {
            const int k = blk / ntj, j0 = (blk % ntj) * R;
            mbar_expect_tx(b_m, 3 * R * NX * sizeof(float));
#pragma unroll 1
            for (int c = 0; c < 3; ++c)
                bulk_g2s(smem_addr(Mt + c * R * NX), Min + (size_t)c * g.N + ((size_t)k * g.ny + j0) * NX,
                         R * NX * sizeof(float), b_m);
        }
    }
    bool ok = mbar_wait(b_tw, 0);
    if (ok) {
        fill_ta<NY, Fft2<NY>::Q, T>(tay, twy);
        fill_ta<NX, Fft2<NX>::Q, T>(tax, twx);
    }
    ok = !__syncthreads_or(!ok);
    int s = 0;
    for (; ok && s < nsteps; ++s) {
        if (has_plane) {
            if (s > 0 && threadIdx.x == 0) {
                // the region held the previous step's tile work; S is the
                // previous step's x-step output (ordinary stores)
                proxy_fence_shared();
                proxy_fence_global();
                mbar_expect_tx(b_s, NL * NY * sizeof(float2));
#pragma unroll 1
                for (int l = 0; l < NL; ++l)
                    bulk_g2s(smem_addr(zb + l * ZS), plane + (size_t)l * g.Jst, NY * sizeof(float2), b_s);
            }
            ok = plane_body<NY, NZ, T>(g, blk, true, twy, tay, Ks, zb, b_s, s & 1, b_k, Sh);
            if (!ok) break;
        }
        ok = grid_sync(gb, 2 * s, wait_limit);            // every plane's Sh written
        if (!ok) break;
        if (has_tile) {
            if (s == 0) {
                ok = !__syncthreads_or(!mbar_wait(b_m, 0));
                if (!ok) break;
            }
            xstep_body<NX, R, kModeStep, T>(g, cf, blk, twx, tax, Mt, sb, wk, Sh, S, s == nsteps - 1 ? Mout : nullptr,
                                            flag);
        }
        if (s + 1 < nsteps) {
            ok = grid_sync(gb, 2 * s + 1, wait_limit);    // every tile's S written
            if (!ok) break;
        }
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(flag, kFlagTimeout);
        // let the copies in flight land before the block leaves (bounded)
        mbar_wait(b_tw, 0);
        if (has_plane) {
            mbar_wait(b_k, 0);
            mbar_wait(b_s, s & 1);                        // the S lines of the last step begun
        }
        if (has_tile) mbar_wait(b_m, 0);
    }
    grid_exit(gb);
}

}  // namespace mmk
