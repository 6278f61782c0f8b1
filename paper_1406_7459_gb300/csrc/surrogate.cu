// surrogate.cu -- elementwise kernels of the surrogate-assisted stepper.
//
// Between exact demag refreshes the demag field is taken as
// H_ref + Ms r FNO((M - M_ref) / (Ms r)), r the root mean square of
// (M - M_ref) / Ms: H_demag is linear in M, so the network only ever sees
// increments of unit scale, whatever the time since the refresh.  The rest
// of the step is the paper's: exchange (Eq. 4), anisotropy (Eq. 5), Zeeman,
// the LLG right-hand side (Eq. 6), forward Euler and renormalisation.
#include "mm_internal.h"

namespace mmk {

// sum of (a - b)^2 in FP64 into *out (zeroed by the caller)
__global__ void k_sumsq_diff(const float* __restrict__ a, const float* __restrict__ b, long long n,
                             double* __restrict__ out) {
    double d2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        d2 += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_down_sync(0xffffffffu, d2, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, d2);
}

// Ms r = rms(M - M_ref) from the sum of squares over n values (0 when
// M = M_ref)
__device__ __forceinline__ double increment_scale(const double* ss, long long n) { return sqrt(*ss / (double)n); }

// out = (a - b) / (Ms r), the unit-scale increment the network takes
__global__ void k_unit_diff(const float* __restrict__ a, const float* __restrict__ b, const double* __restrict__ ss,
                            long long n, float* __restrict__ out) {
    const double sc = increment_scale(ss, n);
    const float inv = sc > 0.0 ? (float)(1.0 / sc) : 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (a[i] - b[i]) * inv;
}

// out = base + Ms r y: the field of the increment from the network's output
__global__ void k_rescale_add(const float* __restrict__ base, const float* __restrict__ y,
                              const double* __restrict__ ss, long long n, float* __restrict__ out) {
    const float sc = (float)increment_scale(ss, n);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = base[i] + sc * y[i];
}

// sums of (a - b)^2 and b^2 in FP64 (out[0], out[1])
__global__ void k_resid(const float* __restrict__ a, const float* __restrict__ b, long long n, double* __restrict__ out) {
    double d2 = 0.0, b2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        d2 += d * d;
        b2 += (double)b[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, d2);
        atomicAdd(out + 1, b2);
    }
}

// Euler step of Eq. (6) with the demag field given: M^{n+1} from M^n, Hd.
__global__ void k_llg_given_h(Geom g, LlgCoef cf, const float* __restrict__ M, const float* __restrict__ Hd,
                              float* __restrict__ out, int* __restrict__ flag) {
    const size_t N = (size_t)g.N;
    for (size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(cell % g.nx);
        const int j = (int)((cell / g.nx) % g.ny);
        const int k = (int)(cell / ((size_t)g.nx * g.ny));
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
            const float m0 = Mc[cell];
            const float lap = (Mc[xp] - 2.f * m0 + Mc[xm]) * cf.idx2 + (Mc[yp] - 2.f * m0 + Mc[ym]) * cf.idy2 +
                              (Mc[zp] - 2.f * m0 + Mc[zm]) * cf.idz2;
            m[c] = m0;
            h[c] = Hd[c * N + cell] + cf.pexch * lap;
        }
        h[0] += cf.hx;
        h[1] += cf.panis * m[1] + cf.hy;
        h[2] += cf.panis * m[2] + cf.hz;
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

static int nblk(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

cudaError_t sur_unit_diff(const float* a, const float* b, long long n, double* ss, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ss, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_sumsq_diff<<<nblk(n), 256, 0, st>>>(a, b, n, ss);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_unit_diff<<<nblk(n), 256, 0, st>>>(a, b, ss, n, out);
    return cudaGetLastError();
}
cudaError_t sur_rescale_add(const float* base, const float* y, const double* ss, long long n, float* out,
                            cudaStream_t st) {
    k_rescale_add<<<nblk(n), 256, 0, st>>>(base, y, ss, n, out);
    return cudaGetLastError();
}
cudaError_t sur_resid(const float* a, const float* b, long long n, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_resid<<<nblk(n), 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}
cudaError_t sur_llg(const Geom& g, const LlgCoef& cf, const float* M, const float* Hd, float* out, int* flag,
                    cudaStream_t st) {
    k_llg_given_h<<<nblk(g.N), 256, 0, st>>>(g, cf, M, Hd, out, flag);
    return cudaGetLastError();
}

}  // namespace mmk
