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
