// plane_kernel.cuh -- pass 2 of the demag convolution, one CTA per kx plane.
//
// For one kx of the x half-spectrum: forward y FFT of the 3*nz lines (only
// the first ny inputs nonzero; Sec. 2 step (1) on the y axis), then for
// every ky the forward z DFT (nz nonzero inputs), the member-wise product
// with the real symmetric tensor spectrum (Eq. (13)/(15)), the inverse z DFT
// keeping k < nz, and finally the inverse y FFT keeping j < ny (Eq. (16);
// the padded half is discarded).  The plane stays in shared memory between
// the steps; the tensor octant is read with the sign flips of its mirrored
// quadrants (odd components change sign when ky or kz is mirrored).
// Instantiated for each padded z length LZ in plane_*.cu so the translation
// units compile in parallel.
#pragma once
#include "mm_internal.h"

namespace mmk {

// ------------------------------------------------------- pass 2 (plane) --
// Length-LZ DFT of a register array with only the first `nin` inputs
// nonzero; forward (W = exp(-2 pi i/LZ)) or inverse (conjugate twiddles).
// Only the first `nout` outputs are formed.  tw[m] = W_LZ^m.
template <int LZ>
__device__ __forceinline__ void small_dft(float2 (&a)[LZ], int nin, int nout, const float2* __restrict__ tw,
                                          bool inverse) {
    if (LZ == 1) return;
    float2 o[LZ];
#pragma unroll
    for (int q = 0; q < LZ; ++q) {
        float2 acc = make_float2(0.f, 0.f);
        if (q < nout) {
#pragma unroll
            for (int k = 0; k < LZ; ++k) {
                if (k < nin) {
                    float2 w = __ldg(tw + (k * q) % LZ);
                    if (inverse) w.y = -w.y;
                    acc = cadd(acc, cmul(a[k], w));
                }
            }
        }
        o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < LZ; ++q) a[q] = o[q];
}

// np consecutive kx planes from kx0 (their lines are contiguous in S):
// every line of the np planes transformed together (one pass of barriers
// for all of them), then the z DFTs and the product for each (kx, ky).
// Each line's transform and each (kx, ky)'s product are the arithmetic of
// one plane alone, so any np gives the same bits.  Shared memory: two
// buffers of np 3 nz lines of padded_len(Ly).
template <int LZ>
__device__ __forceinline__ void plane_body_multi(const Geom& g, int group, float2* __restrict__ S, int kx0, int np) {
    extern __shared__ float2 sm[];
    const int lstride = padded_len(g.Ly);
    const int nz = g.nz;
    const int nl = 3 * nz;
    const int nlt = np * nl;
    float2* plane = S + (size_t)kx0 * nl * g.Jst;

    StrideDiv wi(g.ny);
    for (int idx = threadIdx.x; idx < nlt * g.ny; idx += blockDim.x, wi.next())
        sm[wi.q * lstride + padi(wi.r)] = plane[(size_t)wi.q * g.Jst + wi.r];
    fft_lines(sm, sm + nlt * lstride, lstride, nlt, group, g.py, g.twy, g.ny, false);

    StrideDiv wp(g.Ly);
    for (int t = threadIdx.x; t < np * g.Ly; t += blockDim.x, wp.next()) {
        const int pp = wp.q, ky = wp.r;
        const float* Kp = g.Kt + (size_t)(kx0 + pp) * g.Hz * g.Hy * 6;
        float2* sp = sm + (size_t)pp * nl * lstride;
        float2 m[3][LZ];
        const int e = padi(ky);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int k = 0; k < LZ; ++k)
                m[c][k] = (k < nz) ? sp[(c * nz + k) * lstride + e] : make_float2(0.f, 0.f);
            small_dft<LZ>(m[c], nz, LZ, g.twz, false);
        }
        int kyp = ky;
        float sy = 1.f;
        if (2 * ky > g.Ly) { kyp = g.Ly - ky; sy = -1.f; }
#pragma unroll
        for (int kz = 0; kz < LZ; ++kz) {
            int kzp = kz;
            float sz = 1.f;
            if (2 * kz > LZ) { kzp = LZ - kz; sz = -1.f; }
            const float* kk = Kp + ((size_t)kzp * g.Hy + kyp) * 6;
            const float kxx = __ldg(kk + 0), kxy = sy * __ldg(kk + 1), kxz = sz * __ldg(kk + 2);
            const float kyy = __ldg(kk + 3), kyz = sy * sz * __ldg(kk + 4), kzz = __ldg(kk + 5);
            const float2 mx = m[0][kz], my = m[1][kz], mz = m[2][kz];
            m[0][kz] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
            m[1][kz] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
            m[2][kz] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            small_dft<LZ>(m[c], LZ, nz, g.twz, true);
#pragma unroll
            for (int k = 0; k < LZ; ++k)
                if (k < nz) sp[(c * nz + k) * lstride + e] = m[c][k];
        }
    }
    fft_lines(sm, sm + nlt * lstride, lstride, nlt, group, g.py, g.twy, g.Ly, true);

    StrideDiv wo(g.ny);
    for (int idx = threadIdx.x; idx < nlt * g.ny; idx += blockDim.x, wo.next())
        plane[(size_t)wo.q * g.Jst + wo.r] = sm[wo.q * lstride + padi(wo.r)];
}

template <int LZ>
__device__ __forceinline__ void plane_body(const Geom& g, int group, float2* __restrict__ S, int kx) {
    plane_body_multi<LZ>(g, group, S, kx, 1);
}

template <int LZ>
__global__ void __launch_bounds__(512) k_plane(Geom g, int group, float2* __restrict__ S) {
    pdl_wait();
    plane_body<LZ>(g, group, S, blockIdx.x);
}

}  // namespace mmk
