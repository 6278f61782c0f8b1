// fast_passes.cuh -- the three step kernels specialised at compile time for
// power-of-two grids (nx, ny in 16..1024, nz in {1, 2, 4, 8}).
//
// Same data flow and spectrum layout S[kx][c][k][j] as the generic kernels
// (demag_passes.cu / plane_kernel.cuh): pass 1 forward x R2C (Eq. (14)),
// pass 2 per-kx-plane y/z transforms and the tensor product (Eq. (15)),
// pass 3 inverse x C2R (Eq. (16)) fused with the field and LLG update
// (Eqs. (2)-(6), Euler, renormalisation).  Every padded transform is split
// into two unpadded power-of-two FFTs (fast_fft.cuh) whose lengths, radices
// and twiddle indices are compile-time constants, so the zero half of each
// padded axis is never computed and no integer division runs in the
// butterflies.
#pragma once
#include "fast_fft.cuh"
#include "mm_internal.h"

namespace mmk {

// shared-memory padding of a spectrum line: one slot every 16
__device__ __forceinline__ int pz(int k) { return k + (k >> 4); }
__host__ __device__ constexpr int pzlen(int L) { return L + L / 16 + 1; }

// ---------------------------------------------------------------- pass 1 --
// CTA tile: component c, layer k, rows j0..j0+R-1 (R/2 row pairs, each pair
// one complex line).  Groups of G threads: (pair, half).
// Mcopy (may be null): a second copy of the rows read, e.g. the device copy
// of a state that M points to in host memory.
template <int N, int R>
__global__ void __launch_bounds__(R * Fft2<N>::G) k_pass1_fast(Geom g, const float* __restrict__ M,
                                                                float2* __restrict__ S, float* __restrict__ Mcopy) {
    using F = Fft2<N>;
    constexpr int P = F::P, Q = F::Q, G = F::G, L = 2 * N, ZS = pzlen(2 * N);
    constexpr int T = R * G;                              // the launch's block size
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* ex = tw + L;
    float2* zb = ex + R * F::EX;
    const int ntj = g.ny / R;
    int b = blockIdx.x;
    const int jt = b % ntj;
    b /= ntj;
    const int k = b % g.nz;
    const int c = b / g.nz;
    const int j0 = jt * R;
#pragma unroll
    for (int i = threadIdx.x; i < L; i += T) tw[i] = __ldg(g.twx + i);
    pdl_wait();                           // M and S may belong to the previous kernel
    __syncthreads();

    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int p = grp >> 1, h = grp & 1;
    if (t < Q) {
        const float* ra = M + (size_t)c * g.N + ((size_t)k * g.ny + j0 + 2 * p) * N;
        const float* rb = ra + N;
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = t + Q * q;
            v[q] = make_float2(__ldg(ra + j), __ldg(rb + j));
        }
        if (Mcopy && h == 0) {
            float* ca = Mcopy + (ra - M);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int j = t + Q * q;
                ca[j] = v[q].x;
                ca[N + j] = v[q].y;
            }
        }
        if (h) F::odd_input(v, t, tw);
        F::stepA(v, t, tw, ex + grp * F::EX, false);
    }
    __syncthreads();
    if (t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, false);
#pragma unroll
        for (int q = 0; q < Q; ++q) zb[p * ZS + pz(2 * (t + P * q) + h)] = w[q];
    }
    __syncthreads();
    // A[k] = (Z[k] + conj Z[L-k]) / 2 (even row), B[k] = -i (Z[k] - conj Z[L-k]) / 2
#pragma unroll
    for (int idx = threadIdx.x; idx < (N + 1) * R; idx += T) {
        const int r = idx % R;
        const int kx = idx / R;
        const float2* line = zb + (r >> 1) * ZS;
        const float2 zk = line[pz(kx)];
        const float2 zm = line[pz((L - kx) & (L - 1))];
        float2 o;
        if ((r & 1) == 0) o = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        else o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        S[(((size_t)kx * 3 + c) * g.nz + k) * g.Jst + j0 + r] = o;
    }
}

// ---------------------------------------------------------------- pass 2 --
// z transform of one ky column: forward pruned (NZ nonzero of LZ = 2 NZ)
// by the even/odd split, the tensor product, inverse keeping k < NZ.
// Kp points at the tensor octant slice of this kx ([kz'][ky'][6] floats),
// in global or shared memory.
template <int NZ>
__device__ __forceinline__ void zconv_column(float2 (&m)[3][NZ], const float* __restrict__ Kp, int Hy, int Ly,
                                             int ky, const float2* __restrict__ twz) {
    constexpr int LZ = (NZ == 1) ? 1 : 2 * NZ;
    float2 X[3][LZ];
    if (NZ == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c][0] = m[c][0];
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 e[NZ], o[NZ];
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                e[k] = m[c][k];
                o[k] = (k == 0) ? m[c][k] : cmul(m[c][k], __ldg(twz + k));
            }
            dftp<NZ>(e);
            dftp<NZ>(o);
#pragma unroll
            for (int q = 0; q < NZ; ++q) {
                X[c][2 * q] = e[q];
                X[c][2 * q + 1] = o[q];
            }
        }
    }
    int kyp = ky;
    float sy = 1.f;
    if (2 * ky > Ly) { kyp = Ly - ky; sy = -1.f; }
#pragma unroll
    for (int kz = 0; kz < LZ; ++kz) {
        const int kzp = (2 * kz > LZ) ? LZ - kz : kz;
        const float sz = (2 * kz > LZ) ? -1.f : 1.f;
        const float* kk = Kp + ((size_t)kzp * Hy + kyp) * 6;
        const float2 k01 = *reinterpret_cast<const float2*>(kk);
        const float2 k23 = *reinterpret_cast<const float2*>(kk + 2);
        const float2 k45 = *reinterpret_cast<const float2*>(kk + 4);
        const float kxx = k01.x, kxy = sy * k01.y, kxz = sz * k23.x;
        const float kyy = k23.y, kyz = sy * sz * k45.x, kzz = k45.y;
        const float2 mx = X[0][kz], my = X[1][kz], mz = X[2][kz];
        X[0][kz] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
        X[1][kz] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
        X[2][kz] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
    }
    if (NZ == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) m[c][0] = X[c][0];
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 e[NZ], o[NZ];
#pragma unroll
            for (int q = 0; q < NZ; ++q) {
                e[q] = cconj(X[c][2 * q]);
                o[q] = cconj(X[c][2 * q + 1]);
            }
            dftp<NZ>(e);
            dftp<NZ>(o);
#pragma unroll
            for (int k = 0; k < NZ; ++k) {
                // x[k] = IDFT(X_even)[k] + W_LZ^{-k} IDFT(X_odd)[k]
                float2 ov = cconj(o[k]);
                if (k > 0) ov = cmul(ov, cconj(__ldg(twz + k)));
                m[c][k] = cadd(cconj(e[k]), ov);
            }
        }
    }
}

// CTA = one kx plane of 3*NZ lines of NY (padded to 2 NY).  Groups of G
// threads: (line, half).
template <int NY, int NZ>
__global__ void __launch_bounds__(6 * NZ * Fft2<NY>::G, (6 * NZ * Fft2<NY>::G <= 512) ? 2 : 1) k_plane_fast(Geom g, float2* __restrict__ S) {
    using F = Fft2<NY>;
    constexpr int P = F::P, Q = F::Q, G = F::G, LY = 2 * NY, ZS = pzlen(2 * NY), NL = 3 * NZ;
    constexpr int T = 6 * NZ * G;                         // the launch's block size
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* ex = tw + LY;
    float2* zb = ex + 2 * NL * F::EX;
    const int kx = blockIdx.x;
    float2* plane = S + (size_t)kx * NL * g.Jst;
#pragma unroll
    for (int i = threadIdx.x; i < LY; i += T) tw[i] = __ldg(g.twy + i);
    pdl_wait();                           // S comes from the previous kernel
    __syncthreads();

    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int line = grp >> 1, h = grp & 1;
    // forward y, pruned input
    if (t < Q) {
        const float2* src = plane + (size_t)line * g.Jst;
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = t + Q * q;
            v[q] = src[j];
        }
        if (h) F::odd_input(v, t, tw);
        F::stepA(v, t, tw, ex + grp * F::EX, false);
    }
    __syncthreads();
    if (t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, false);
#pragma unroll
        for (int q = 0; q < Q; ++q) zb[line * ZS + pz(2 * (t + P * q) + h)] = w[q];
    }
    __syncthreads();
    // z transform + tensor product + inverse z, one ky column per thread
    const float* Kp = g.Kt + (size_t)kx * g.Hz * g.Hy * 6;
    for (int ky = threadIdx.x; ky < LY; ky += T) {
        float2 m[3][NZ];
        const int e = pz(ky);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < NZ; ++k) m[c][k] = zb[(c * NZ + k) * ZS + e];
        zconv_column<NZ>(m, Kp, g.Hy, LY, ky, g.twz);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < NZ; ++k) zb[(c * NZ + k) * ZS + e] = m[c][k];
    }
    __syncthreads();
    // inverse y, pruned output: x = IFFT(X_even) + W^{-j} IFFT(X_odd)
    if (t < Q) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = zb[line * ZS + pz(2 * (t + Q * q) + h)];
        F::stepA(v, t, tw, ex + grp * F::EX, true);
    }
    __syncthreads();
    if (t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, true);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int n = t + P * q;
            float2 val = w[q];
            if (h) val = cmul(val, cconj(tw[n]));
            zb[line * ZS + pz(h * NY + n)] = val;
        }
    }
    __syncthreads();
#pragma unroll
    for (int idx = threadIdx.x; idx < NL * NY; idx += T) {
        const int l = idx / NY, n = idx % NY;
        plane[(size_t)l * g.Jst + n] = cadd(zb[l * ZS + pz(n)], zb[l * ZS + pz(NY + n)]);
    }
}

// ---------------------------------------------------------------- pass 3 --
template <int N, int R> __host__ __device__ constexpr int pass3_fast_threads() {
    return 3 * R * Fft2<N>::G > 128 ? 3 * R * Fft2<N>::G : 128;
}
// CTA tile: layer k, rows j0..j0+R-1, all three components: 3R/2 complex
// lines (row pairs), groups (line, half).  Then the per-cell update.
template <int N, int R, int MODE>
__global__ void __launch_bounds__(256) k_pass3_fast(Geom g, LlgCoef cf, const float2* __restrict__ S,
                                                     const float* __restrict__ M, float* __restrict__ out,
                                                     int* __restrict__ flag) {
    using F = Fft2<N>;
    constexpr int P = F::P, Q = F::Q, G = F::G, L = 2 * N, NL = 3 * R / 2, H = N + 1;
    constexpr int T = pass3_fast_threads<N, R>();         // the launch's block size
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* sb = tw + L;                  // staged half-spectrum [c][kx][r]
    float2* ex = sb + 3 * H * R;          // 2*NL exchange buffers
    float2* ob = ex + 2 * NL * F::EX;     // [line][h*N + n]
    const int ntj = g.ny / R;
    const int jt = blockIdx.x % ntj;
    const int k = blockIdx.x / ntj;
    const int j0 = jt * R;
#pragma unroll
    for (int i = threadIdx.x; i < L; i += T) tw[i] = __ldg(g.twx + i);
    pdl_wait();                           // S (and M) come from earlier kernels
#pragma unroll
    for (int idx = threadIdx.x; idx < 3 * H * R; idx += T) {
        const int r = idx % R;
        const int rest = idx / R;
        const int kx = rest % H, c = rest / H;
        sb[idx] = S[(((size_t)kx * 3 + c) * g.nz + k) * g.Jst + j0 + r];
    }
    __syncthreads();

    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int line = grp >> 1, h = grp & 1;
    const int c = line / (R / 2), pr = line % (R / 2);
    if (grp < 2 * NL && t < Q) {
        const float2* base = sb + (size_t)c * H * R + 2 * pr;
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int kk = 2 * (t + Q * q) + h;     // full-length index in [0, L)
            const bool low = kk <= N;
            const int ks = low ? kk : L - kk;
            float2 A = base[ks * R], B = base[ks * R + 1];
            if (ks == 0 || ks == N) { A.y = 0.f; B.y = 0.f; }
            v[q] = low ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
        }
        F::stepA(v, t, tw, ex + grp * F::EX, true);
    }
    __syncthreads();
    if (grp < 2 * NL && t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, true);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int n = t + P * q;
            float2 val = w[q];
            if (h) val = cmul(val, cconj(tw[n]));
            ob[line * (2 * N) + h * N + n] = val;
        }
    }
    __syncthreads();

    const size_t Nc = (size_t)g.N;
#pragma unroll
    for (int idx = threadIdx.x; idx < R * N; idx += T) {
        const int r = idx / N;
        const int i = idx % N;
        const int j = j0 + r;
        float hd[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const int ln = cc * (R / 2) + (r >> 1);
            const float2 z = cadd(ob[ln * (2 * N) + i], ob[ln * (2 * N) + N + i]);
            hd[cc] = (r & 1) ? z.y : z.x;
        }
        const size_t cell = (size_t)i + (size_t)N * ((size_t)j + (size_t)g.ny * k);
        if (MODE == kModeDemag) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) out[cc * Nc + cell] = hd[cc];
            continue;
        }
        const size_t xm = (i > 0) ? cell - 1 : cell;
        const size_t xp = (i + 1 < N) ? cell + 1 : cell;
        const size_t ym = (j > 0) ? cell - N : cell;
        const size_t yp = (j + 1 < g.ny) ? cell + N : cell;
        const size_t sxy = (size_t)N * g.ny;
        const size_t zm = (k > 0) ? cell - sxy : cell;
        const size_t zp = (k + 1 < g.nz) ? cell + sxy : cell;
        float m[3], hh[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const float* Mc = M + cc * Nc;
            const float m0 = __ldg(Mc + cell);
            const float lap = (__ldg(Mc + xp) - 2.f * m0 + __ldg(Mc + xm)) * cf.idx2 +
                              (__ldg(Mc + yp) - 2.f * m0 + __ldg(Mc + ym)) * cf.idy2 +
                              (__ldg(Mc + zp) - 2.f * m0 + __ldg(Mc + zm)) * cf.idz2;
            m[cc] = m0;
            hh[cc] = hd[cc] + cf.pexch * lap;
        }
        hh[0] += cf.hx;
        hh[1] += cf.panis * m[1] + cf.hy;
        hh[2] += cf.panis * m[2] + cf.hz;
        if (MODE == kModeHeff) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) out[cc * Nc + cell] = hh[cc];
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
        const float s = cf.Ms / sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
        const float o0 = n0 * s, o1 = n1 * s, o2 = n2 * s;
        if (!(isfinite(o0) && isfinite(o1) && isfinite(o2))) atomicOr(flag, 1);
        out[cell] = o0;
        out[Nc + cell] = o1;
        out[2 * Nc + cell] = o2;
    }
}

// shared-memory bytes of each fast kernel
template <int N, int R> constexpr size_t pass1_fast_smem() {
    return sizeof(float2) * (2 * N + R * Fft2<N>::EX + (R / 2) * pzlen(2 * N));
}
template <int NY, int NZ> constexpr size_t plane_fast_smem() {
    return sizeof(float2) * (2 * NY + 6 * NZ * Fft2<NY>::EX + 3 * NZ * pzlen(2 * NY));
}
template <int N, int R> constexpr size_t pass3_fast_smem() {
    return sizeof(float2) * (2 * N + 3 * (N + 1) * R + 3 * R * Fft2<N>::EX + (3 * R / 2) * 2 * N);
}

}  // namespace mmk
