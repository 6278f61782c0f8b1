// demag_passes.cu -- the three per-step kernels of the demag + LLG hot path.
//
// Pass 1  forward x R2C of Mx, My, Mz on the zero-padded length Lx; only the
//         first nx inputs of a row are nonzero (Sec. 2 step (1), Eq. (14)).
//         Two real rows ride in one complex transform.  Output: the
//         half-spectrum kx in [0, Lx/2] written kx-major into S.
// Pass 2  one CTA per kx plane: forward y FFT (ny nonzero inputs), forward
//         z FFT (nz nonzero inputs), the 3x3 product with the real symmetric
//         tensor spectrum (Eq. (13)/(15)), inverse z keeping k < nz, inverse
//         y keeping j < ny (Eq. (16), "discard the latter half").
// Pass 3  inverse x C2R keeping i < nx, then, per cell, H_demag joined with
//         the exchange stencil (Eq. (4), free boundaries), anisotropy
//         (Eq. (5), easy axis x), Zeeman, the LLG right-hand side (Eq. (6)),
//         a forward-Euler step and renormalisation |M| = Ms.  Modes write
//         H_demag, H_eff or M^{n+1}.
#include "mm_internal.h"

namespace mmk {

// ---------------------------------------------------------------- pass 1 --
__global__ void __launch_bounds__(256) k_pass1(Geom g, int R, int group, const float* __restrict__ M,
                                                float2* __restrict__ S) {
    extern __shared__ float2 sm[];
    const int lstride = padded_len(g.Lx);
    const int ntj = (g.ny + R - 1) / R;
    int b = blockIdx.x;
    const int jt = b % ntj;
    b /= ntj;
    const int k = b % g.nz;
    const int c = b / g.nz;
    const int j0 = jt * R;

    const float* Mc = M + (size_t)c * g.N + (size_t)k * g.nx * g.ny;
    for (int idx = threadIdx.x; idx < R * g.nx; idx += blockDim.x) {
        const int r = idx / g.nx;
        const int i = idx - r * g.nx;
        const int j = j0 + r;
        const float v = (j < g.ny) ? __ldg(Mc + (size_t)j * g.nx + i) : 0.f;
        reinterpret_cast<float*>(sm + (r >> 1) * lstride + padi(i))[r & 1] = v;
    }
    fft_lines(sm, sm + (R / 2) * lstride, lstride, R / 2, group, g.px, g.twx, g.nx, false);

    // Split Z = A + iB into the spectra of the two real rows:
    // A[k] = (Z[k] + conj Z[L-k]) / 2, B[k] = -i (Z[k] - conj Z[L-k]) / 2.
    for (int idx = threadIdx.x; idx < g.Hx * R; idx += blockDim.x) {
        const int r = idx % R;
        const int kx = idx / R;
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
__global__ void __launch_bounds__(256) k_pass3(Geom g, int R, int group, LlgCoef cf,
                                                const float2* __restrict__ S, const float* __restrict__ M,
                                                float* __restrict__ out, int* __restrict__ flag) {
    extern __shared__ float2 sm[];
    const int lstride = padded_len(g.Lx);
    const int ntj = (g.ny + R - 1) / R;
    const int jt = blockIdx.x % ntj;
    const int k = blockIdx.x / ntj;
    const int j0 = jt * R;
    const int half = R / 2;

    // Rebuild Z = A + iB for each pair of rows (A: row 2p, B: row 2p+1) on
    // the full length Lx from the stored half-spectrum (Hermitian symmetry).
    for (int idx = threadIdx.x; idx < 3 * g.Hx * half; idx += blockDim.x) {
        const int rp = idx % half;
        const int t = idx / half;
        const int kx = t % g.Hx;
        const int c = t / g.Hx;
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
    for (int idx = threadIdx.x; idx < R * g.nx; idx += blockDim.x) {
        const int r = idx / g.nx;
        const int i = idx - r * g.nx;
        const int j = j0 + r;
        if (j >= g.ny) continue;
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
    }
}

// -------------------------------------------------------------- launchers --
static PlaneFn plane_fn(int Lz) {
    PlaneFn f = plane_fn_small(Lz);
    if (!f) f = plane_fn_mid(Lz);
    if (!f) f = plane_fn_large(Lz);
    return f;
}

bool plane_supported_lz(int Lz) { return plane_fn(Lz) != nullptr; }

cudaError_t configure_pass_kernels(const Geom& g, const Launch& l) {
    cudaError_t e;
    if (l.fx) {
        e = cudaFuncSetAttribute(l.fx->p1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fx->s1);
        for (int m = 0; m < 3 && e == cudaSuccess; ++m)
            e = cudaFuncSetAttribute(l.fx->p3[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fx->s3);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(k_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem1);
        if (e != cudaSuccess) return e;
        for (int m = 0; m < 3 && e == cudaSuccess; ++m)
            e = cudaFuncSetAttribute(m == 0 ? k_pass3<kModeDemag> : m == 1 ? k_pass3<kModeHeff> : k_pass3<kModeStep>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem3);
        if (e != cudaSuccess) return e;
    }
    if (l.split) return configure_split_kernels(g);
    if (l.fp) return cudaFuncSetAttribute(l.fp->pl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fp->s2);
    PlaneFn pf = plane_fn(g.Lz);
    if (!pf) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem2);
}

cudaError_t launch_pass1(const Geom& g, const Launch& l, const float* M, float2* S, cudaStream_t s) {
    if (l.fx) {
        l.fx->p1<<<3 * g.nz * (g.ny / l.fx->r1), l.fx->t1, l.fx->s1, s>>>(g, M, S);
        return cudaGetLastError();
    }
    const int ntj = (g.ny + l.r1 - 1) / l.r1;
    k_pass1<<<3 * g.nz * ntj, l.t1, l.smem1, s>>>(g, l.r1, l.g1, M, S);
    return cudaGetLastError();
}

cudaError_t launch_plane(const Geom& g, const Launch& l, float2* S, cudaStream_t s) {
    if (l.split) return launch_split_plane(g, S, s);
    if (l.fp) {
        l.fp->pl<<<g.Hx, l.fp->t2, l.fp->s2, s>>>(g, S);
        return cudaGetLastError();
    }
    PlaneFn pf = plane_fn(g.Lz);
    if (!pf) return cudaErrorInvalidValue;
    pf<<<g.Hx, l.t2, l.smem2, s>>>(g, l.g2, S);
    return cudaGetLastError();
}

cudaError_t launch_pass3(const Geom& g, const Launch& l, const LlgCoef& c, int mode, const float2* S,
                         const float* M, float* out, int* flag, cudaStream_t s) {
    if (l.fx) {
        l.fx->p3[mode]<<<g.nz * (g.ny / l.fx->r3), l.fx->t3, l.fx->s3, s>>>(g, c, S, M, out, flag);
        return cudaGetLastError();
    }
    const int ntj = (g.ny + l.r3 - 1) / l.r3;
    const int grid = g.nz * ntj;
    switch (mode) {
        case kModeDemag: k_pass3<kModeDemag><<<grid, l.t3, l.smem3, s>>>(g, l.r3, l.g3, c, S, M, out, flag); break;
        case kModeHeff: k_pass3<kModeHeff><<<grid, l.t3, l.smem3, s>>>(g, l.r3, l.g3, c, S, M, out, flag); break;
        default: k_pass3<kModeStep><<<grid, l.t3, l.smem3, s>>>(g, l.r3, l.g3, c, S, M, out, flag); break;
    }
    return cudaGetLastError();
}

}  // namespace mmk
