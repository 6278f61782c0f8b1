// pass_bodies.cuh -- device bodies of the generic pass-1 and pass-3 kernels
// (x R2C; x C2R + field + LLG), parameterised by the tile index so that the
// single-grid kernels (demag_passes.cu) and the batched kernels (batch.cu)
// share them.  See demag_passes.cu for what each pass computes.
#pragma once
#include "mm_internal.h"

namespace mmk {

// ---------------------------------------------------------------- pass 1 --
__device__ __forceinline__ void pass1_body(const Geom& g, int R, int group, const float* __restrict__ M,
                                           float2* __restrict__ S, int tile) {
    extern __shared__ float2 sm[];
    const int lstride = padded_len(g.Lx);
    const int ntj = (g.ny + R - 1) / R;
    int b = tile;
    const int jt = b % ntj;
    b /= ntj;
    const int k = b % g.nz;
    const int c = b / g.nz;
    const int j0 = jt * R;

    const float* Mc = M + (size_t)c * g.N + (size_t)k * g.nx * g.ny;
    StrideDiv wl(g.nx);
    for (int idx = threadIdx.x; idx < R * g.nx; idx += blockDim.x, wl.next()) {
        const int r = wl.q;
        const int i = wl.r;
        const int j = j0 + r;
        const float v = (j < g.ny) ? __ldg(Mc + (size_t)j * g.nx + i) : 0.f;
        reinterpret_cast<float*>(sm + (r >> 1) * lstride + padi(i))[r & 1] = v;
    }
    fft_lines(sm, sm + (R / 2) * lstride, lstride, R / 2, group, g.px, g.twx, g.nx, false);

    // Split Z = A + iB into the spectra of the two real rows:
    // A[k] = (Z[k] + conj Z[L-k]) / 2, B[k] = -i (Z[k] - conj Z[L-k]) / 2.
    StrideDiv ws(R);
    for (int idx = threadIdx.x; idx < g.Hx * R; idx += blockDim.x, ws.next()) {
        const int r = ws.r;
        const int kx = ws.q;
        const int j = j0 + r;
        if (j >= g.ny) continue;
        const float2* line = sm + (r >> 1) * lstride;
        const float2 zk = line[padi(kx)];
        const float2 zm = line[padi(kx == 0 ? 0 : g.Lx - kx)];
        float2 o;
        if ((r & 1) == 0) o = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        else o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        S[(((size_t)kx * 3 + c) * g.nz + k) * g.Jst + j] = o;
    }
}

// ---------------------------------------------------------------- pass 3 --
template <int MODE>
__device__ __forceinline__ void pass3_body(const Geom& g, int R, int group, const LlgCoef& cf,
                                           const float2* S, const float* __restrict__ M,
                                           float* __restrict__ out, int* __restrict__ flag, int tile,
                                           float2* Snext = nullptr) {
    extern __shared__ float2 sm[];
    const int lstride = padded_len(g.Lx);
    const int ntj = (g.ny + R - 1) / R;
    const int jt = tile % ntj;
    const int k = tile / ntj;
    const int j0 = jt * R;
    const int half = R / 2;

    // Rebuild Z = A + iB for each pair of rows (A: row 2p, B: row 2p+1) on
    // the full length Lx from the stored half-spectrum (Hermitian symmetry).
    const FastDiv byHx(g.Hx);                             // t < 3 Hx < 2^16
    StrideDiv wr(half);
    for (int idx = threadIdx.x; idx < 3 * g.Hx * half; idx += blockDim.x, wr.next()) {
        const int rp = wr.r;
        const int t = wr.q;
        const int c = byHx.div(t);
        const int kx = t - c * g.Hx;
        const int ja = j0 + 2 * rp;
        const float2* src = S + (((size_t)kx * 3 + c) * g.nz + k) * g.Jst;
        float2 A = (ja < g.ny) ? src[ja] : make_float2(0.f, 0.f);
        float2 B = (ja + 1 < g.ny) ? src[ja + 1] : make_float2(0.f, 0.f);
        const bool selfconj = (kx == 0) || (2 * kx == g.Lx);
        if (selfconj) { A.y = 0.f; B.y = 0.f; }
        float2* line = sm + (c * half + rp) * lstride;
        line[padi(kx)] = make_float2(A.x - B.y, A.y + B.x);
        if (!selfconj) line[padi(g.Lx - kx)] = make_float2(A.x + B.y, B.x - A.y);
    }
    fft_lines(sm, sm + 3 * half * lstride, lstride, 3 * half, group, g.px, g.twx, g.Lx, true);

    const size_t N = (size_t)g.N;
    StrideDiv wf(g.nx);
    for (int idx = threadIdx.x; idx < R * g.nx; idx += blockDim.x, wf.next()) {
        const int r = wf.q;
        const int i = wf.r;
        const int j = j0 + r;
        if (j >= g.ny) {
            if (MODE == kModeStepX) {
                // a row past the sample: zero, as the x pass would read it
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    reinterpret_cast<float*>(sm + (c * half + (r >> 1)) * lstride + padi(i))[r & 1] = 0.f;
            }
            continue;
        }
        float hd[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 z = sm[(c * half + (r >> 1)) * lstride + padi(i)];
            hd[c] = (r & 1) ? z.y : z.x;
        }
        const size_t cell = (size_t)i + (size_t)g.nx * ((size_t)j + (size_t)g.ny * k);
        if (MODE == kModeDemag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) out[c * N + cell] = hd[c];
            continue;
        }
        const size_t xm = (i > 0) ? cell - 1 : cell;
        const size_t xp = (i + 1 < g.nx) ? cell + 1 : cell;
        const size_t ym = (j > 0) ? cell - g.nx : cell;
        const size_t yp = (j + 1 < g.ny) ? cell + g.nx : cell;
        const size_t sxy = (size_t)g.nx * g.ny;
        const size_t zm = (k > 0) ? cell - sxy : cell;
        const size_t zp = (k + 1 < g.nz) ? cell + sxy : cell;
        float m[3], h[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* Mc = M + c * N;
            const float m0 = __ldg(Mc + cell);
            const float lap = (__ldg(Mc + xp) - 2.f * m0 + __ldg(Mc + xm)) * cf.idx2 +
                              (__ldg(Mc + yp) - 2.f * m0 + __ldg(Mc + ym)) * cf.idy2 +
                              (__ldg(Mc + zp) - 2.f * m0 + __ldg(Mc + zm)) * cf.idz2;
            m[c] = m0;
            h[c] = hd[c] + cf.pexch * lap;
        }
        h[0] += cf.hx;
        h[1] += cf.panis * m[1] + cf.hy;
        h[2] += cf.panis * m[2] + cf.hz;
        if (MODE == kModeHeff) {
#pragma unroll
            for (int c = 0; c < 3; ++c) out[c * N + cell] = h[c];
            continue;
        }
        // Eq. (6): dM/dt = c1 M x H + c2 M x (M x H)
        const float p0 = m[1] * h[2] - m[2] * h[1];
        const float p1 = m[2] * h[0] - m[0] * h[2];
        const float p2 = m[0] * h[1] - m[1] * h[0];
        const float q0 = m[1] * p2 - m[2] * p1;
        const float q1 = m[2] * p0 - m[0] * p2;
        const float q2 = m[0] * p1 - m[1] * p0;
        const float n0 = m[0] + cf.dt * (cf.c1 * p0 + cf.c2 * q0);
        const float n1 = m[1] + cf.dt * (cf.c1 * p1 + cf.c2 * q1);
        const float n2 = m[2] + cf.dt * (cf.c1 * p2 + cf.c2 * q2);
        const float s = cf.Ms / sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
        const float o0 = n0 * s, o1 = n1 * s, o2 = n2 * s;
        if (!(isfinite(o0) && isfinite(o1) && isfinite(o2))) atomicOr(flag, 1);
        out[cell] = o0;
        out[N + cell] = o1;
        out[2 * N + cell] = o2;
        if (MODE == kModeStepX) {
            // the new row values replace this row's half of the pair line
            // (each float is read above and written here by this thread only)
            reinterpret_cast<float*>(sm + (0 * half + (r >> 1)) * lstride + padi(i))[r & 1] = o0;
            reinterpret_cast<float*>(sm + (1 * half + (r >> 1)) * lstride + padi(i))[r & 1] = o1;
            reinterpret_cast<float*>(sm + (2 * half + (r >> 1)) * lstride + padi(i))[r & 1] = o2;
        }
    }
    if (MODE == kModeStepX) {
        // forward x R2C of the new rows (inputs beyond nx are taken as zero),
        // then the split into the rows' half-spectra, into Snext (which may
        // be S itself: this tile read exactly these (kx, c, k, j) entries at
        // its start)
        fft_lines(sm, sm + 3 * half * lstride, lstride, 3 * half, group, g.px, g.twx, g.nx, false);
        __syncthreads();
        float2* Sw = Snext;
        StrideDiv wo(R);
        for (int idx = threadIdx.x; idx < 3 * g.Hx * R; idx += blockDim.x, wo.next()) {
            const int r = wo.r;
            const int t = wo.q;
            const int c = byHx.div(t);
            const int kx = t - c * g.Hx;
            const int j = j0 + r;
            if (j >= g.ny) continue;
            const float2* line = sm + (c * half + (r >> 1)) * lstride;
            const float2 zk = line[padi(kx)];
            const float2 zm = line[padi(kx == 0 ? 0 : g.Lx - kx)];
            float2 o;
            if ((r & 1) == 0) o = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            else o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            Sw[(((size_t)kx * 3 + c) * g.nz + k) * g.Jst + j] = o;
        }
    }
}

}  // namespace mmk
