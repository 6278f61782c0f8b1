// integrators.cu -- stage update of the explicit Runge-Kutta steppers.
//
// The paper integrates Eq. (6) with forward Euler (Table 1 caption).  Heun
// and the classic fourth-order Runge-Kutta scheme reuse the same field
// evaluation (x R2C -> plane -> x C2R + exchange/anisotropy/Zeeman, writing
// H_eff) once per stage; this kernel then forms the LLG right-hand side at
// the stage state and
//   - accumulates acc = sum_i b_i k_i,
//   - writes the next stage state M_n + a dt k_i (not renormalised), or, on
//     the last stage, M_n + dt acc renormalised to |M| = Ms.
#include "mm_internal.h"

namespace mmk {

__global__ void __launch_bounds__(256) k_rk_stage(int N, LlgCoef cf, float a_next, float b_acc, int kind,
                                                  const float* __restrict__ Mst, const float* __restrict__ H,
                                                  const float* __restrict__ Mb, float* __restrict__ acc,
                                                  float* __restrict__ out, int* __restrict__ flag) {
    const size_t n = (size_t)N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float m0 = Mst[i], m1 = Mst[n + i], m2 = Mst[2 * n + i];
        const float h0 = H[i], h1 = H[n + i], h2 = H[2 * n + i];
        const float p0 = m1 * h2 - m2 * h1;
        const float p1 = m2 * h0 - m0 * h2;
        const float p2 = m0 * h1 - m1 * h0;
        const float q0 = m1 * p2 - m2 * p1;
        const float q1 = m2 * p0 - m0 * p2;
        const float q2 = m0 * p1 - m1 * p0;
        const float f0 = cf.c1 * p0 + cf.c2 * q0;
        const float f1 = cf.c1 * p1 + cf.c2 * q1;
        const float f2 = cf.c1 * p2 + cf.c2 * q2;
        float a0 = b_acc * f0, a1 = b_acc * f1, a2 = b_acc * f2;
        if (kind != 0) {
            a0 += acc[i];
            a1 += acc[n + i];
            a2 += acc[2 * n + i];
        }
        if (kind == 2) {
            const float n0 = Mb[i] + cf.dt * a0;
            const float n1 = Mb[n + i] + cf.dt * a1;
            const float n2 = Mb[2 * n + i] + cf.dt * a2;
            const float s = cf.Ms / sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
            const float o0 = n0 * s, o1 = n1 * s, o2 = n2 * s;
            if (!(isfinite(o0) && isfinite(o1) && isfinite(o2))) atomicOr(flag, 1);
            out[i] = o0;
            out[n + i] = o1;
            out[2 * n + i] = o2;
        } else {
            acc[i] = a0;
            acc[n + i] = a1;
            acc[2 * n + i] = a2;
            const float s = a_next * cf.dt;
            out[i] = Mb[i] + s * f0;
            out[n + i] = Mb[n + i] + s * f1;
            out[2 * n + i] = Mb[2 * n + i] + s * f2;
        }
    }
}

cudaError_t launch_rk_stage(int N, const LlgCoef& cf, float a_next, float b_acc, int kind, const float* Mst,
                            const float* H, const float* Mb, float* acc, float* out, int* flag, cudaStream_t s) {
    int blocks = (N + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_rk_stage<<<blocks, 256, 0, s>>>(N, cf, a_next, b_acc, kind, Mst, H, Mb, acc, out, flag);
    return cudaGetLastError();
}

}  // namespace mmk

// ---------------------------------------------------------------------------
// Adaptive Dormand-Prince RK5(4) (beyond the paper).  Stage states are plain;
// the fifth-order state is renormalised to |M| = Ms; the seventh stage is
// the right-hand side there (it becomes k1 of the next step).
//
// k_dp_combine: out = M + dt sum_{j < nk} w_j k_j (optionally renormalised).
// k_dp_stage:   k_i = f(Y_i, H_i) -> k[i-1]; then out = M + dt sum_{j <= i} w_j k_j,
//               renormalised when `renorm` (the candidate state after k6).
//               out may alias Y (each cell is read, then written, by one
//               thread).  A non-finite candidate sets *flag when flag is
//               non-null; the adaptive driver passes null and lets the
//               infinite error estimate reject the step instead.
// k_dp_error:   k7 = f(Y, H) -> k7out; err = max over cells |dt sum_j e_j k_j| / Ms,
//               folded into *errbits with an unsigned max (non-negative floats
//               order like their bit patterns).

namespace mmk {

__device__ __forceinline__ void llg_f(const LlgCoef& cf, float m0, float m1, float m2, float h0, float h1, float h2,
                                      float& f0, float& f1, float& f2) {
    const float p0 = m1 * h2 - m2 * h1;
    const float p1 = m2 * h0 - m0 * h2;
    const float p2 = m0 * h1 - m1 * h0;
    const float q0 = m1 * p2 - m2 * p1;
    const float q1 = m2 * p0 - m0 * p2;
    const float q2 = m0 * p1 - m1 * p0;
    f0 = cf.c1 * p0 + cf.c2 * q0;
    f1 = cf.c1 * p1 + cf.c2 * q1;
    f2 = cf.c1 * p2 + cf.c2 * q2;
}

__device__ __forceinline__ void dp_store(size_t n, size_t i, float s0, float s1, float s2, const float* M, float dt,
                                         bool renorm, float Ms, float* out, int* flag) {
    float o0 = M[i] + dt * s0, o1 = M[n + i] + dt * s1, o2 = M[2 * n + i] + dt * s2;
    if (renorm) {
        const float s = Ms / sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        o0 *= s;
        o1 *= s;
        o2 *= s;
        if (flag && !(isfinite(o0) && isfinite(o1) && isfinite(o2))) atomicOr(flag, 1);
    }
    out[i] = o0;
    out[n + i] = o1;
    out[2 * n + i] = o2;
}

__global__ void __launch_bounds__(256) k_dp_combine(int N, DpPtrs kp, DpWeights w, int nk, float dt,
                                                    const float* __restrict__ M, float* __restrict__ out) {
    const size_t n = (size_t)N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int j = 0; j < nk; ++j) {
            if (w.w[j] == 0.f) continue;
            const float* k = kp.k[j];
            s0 += w.w[j] * k[i];
            s1 += w.w[j] * k[n + i];
            s2 += w.w[j] * k[2 * n + i];
        }
        dp_store(n, i, s0, s1, s2, M, dt, false, 0.f, out, nullptr);
    }
}

__global__ void __launch_bounds__(256) k_dp_stage(int N, LlgCoef cf, DpPtrs kp, int stage, DpWeights w, int renorm,
                                                  const float* __restrict__ Y, const float* __restrict__ H,
                                                  const float* __restrict__ M, float* __restrict__ out,
                                                  int* __restrict__ flag) {
    const size_t n = (size_t)N;
    float* kout = kp.k[stage - 1];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float f0, f1, f2;
        llg_f(cf, Y[i], Y[n + i], Y[2 * n + i], H[i], H[n + i], H[2 * n + i], f0, f1, f2);
        kout[i] = f0;
        kout[n + i] = f1;
        kout[2 * n + i] = f2;
        const float wi = w.w[stage - 1];
        float s0 = wi * f0, s1 = wi * f1, s2 = wi * f2;
        for (int j = 0; j < stage - 1; ++j) {
            if (w.w[j] == 0.f) continue;
            const float* k = kp.k[j];
            s0 += w.w[j] * k[i];
            s1 += w.w[j] * k[n + i];
            s2 += w.w[j] * k[2 * n + i];
        }
        dp_store(n, i, s0, s1, s2, M, cf.dt, renorm != 0, cf.Ms, out, flag);
    }
}

__global__ void __launch_bounds__(256) k_dp_error(int N, LlgCoef cf, DpPtrs kp, DpWeights e,
                                                  const float* __restrict__ Y, const float* __restrict__ H,
                                                  float* __restrict__ k7out, unsigned* __restrict__ errbits) {
    const size_t n = (size_t)N;
    float emax = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float f0, f1, f2;
        llg_f(cf, Y[i], Y[n + i], Y[2 * n + i], H[i], H[n + i], H[2 * n + i], f0, f1, f2);
        k7out[i] = f0;
        k7out[n + i] = f1;
        k7out[2 * n + i] = f2;
        float d0 = e.w[6] * f0, d1 = e.w[6] * f1, d2 = e.w[6] * f2;
        for (int j = 0; j < 6; ++j) {
            if (e.w[j] == 0.f) continue;
            const float* k = kp.k[j];
            d0 += e.w[j] * k[i];
            d1 += e.w[j] * k[n + i];
            d2 += e.w[j] * k[2 * n + i];
        }
        const float r = fabsf(cf.dt) * sqrtf(d0 * d0 + d1 * d1 + d2 * d2) / cf.Ms;
        emax = (r > emax || r != r) ? r : emax;       // a NaN wins (it fails the step)
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float x = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = (x > emax || x != x) ? x : emax;
    }
    __shared__ float wmax[8];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = wmax[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) b = (wmax[q] > b || wmax[q] != wmax[q]) ? wmax[q] : b;
        if (b != b) b = __int_as_float(0x7f800000);   // NaN -> +inf for the unsigned max
        atomicMax(errbits, __float_as_uint(b));
    }
}

static int dp_blocks(int N) {
    int blocks = (N + 255) / 256;
    return blocks > 152 * 8 ? 152 * 8 : blocks;
}

cudaError_t launch_dp_combine(int N, const DpPtrs& kp, const DpWeights& w, int nk, float dt, const float* M,
                              float* out, cudaStream_t s) {
    k_dp_combine<<<dp_blocks(N), 256, 0, s>>>(N, kp, w, nk, dt, M, out);
    return cudaGetLastError();
}

cudaError_t launch_dp_stage(int N, const LlgCoef& cf, const DpPtrs& kp, int stage, const DpWeights& w, int renorm,
                            const float* Y, const float* H, const float* M, float* out, int* flag, cudaStream_t s) {
    k_dp_stage<<<dp_blocks(N), 256, 0, s>>>(N, cf, kp, stage, w, renorm, Y, H, M, out, flag);
    return cudaGetLastError();
}

cudaError_t launch_dp_error(int N, const LlgCoef& cf, const DpPtrs& kp, const DpWeights& e, const float* Y,
                            const float* H, float* k7out, unsigned* errbits, cudaStream_t s) {
    k_dp_error<<<dp_blocks(N), 256, 0, s>>>(N, cf, kp, e, Y, H, k7out, errbits);
    return cudaGetLastError();
}

}  // namespace mmk
