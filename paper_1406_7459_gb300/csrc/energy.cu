// energy.cu -- the energy of Eq. (1) summed in FP64.
//
// Per cell: exchange as the link sum |m_i - m_j|^2 / delta^2 over the +x,
// +y, +z neighbours that exist (each link once; the discrete form of
// A (grad m)^2 matching the free-boundary stencil of Eq. (4)), anisotropy
// (M_y^2 + M_z^2)/Ms^2, demag H_d . M and Zeeman H_ext . M.  A fixed grid
// writes one partial per block, and a single block adds the partials in a
// fixed order, so the result is deterministic.
#include "mm_internal.h"

namespace mmk {

constexpr int kEnergyBlocks = 1024;
constexpr int kEnergyThreads = 256;

size_t energy_partials_elems(int) { return (size_t)kEnergyBlocks * 4; }

__device__ inline double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(kEnergyThreads) k_energy_partial(Geom g, double Ms, double hx, double hy,
                                                                    double hz, double idx2, double idy2,
                                                                    double idz2, const float* __restrict__ M,
                                                                    const float* __restrict__ H,
                                                                    double* __restrict__ part) {
    __shared__ double red[kEnergyThreads / 32];
    const size_t N = (size_t)g.N;
    const double inv = 1.0 / Ms;
    double ex = 0, an = 0, de = 0, ze = 0;
    for (size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
         cell += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(cell % g.nx);
        const int j = (int)((cell / g.nx) % g.ny);
        const int k = (int)(cell / ((size_t)g.nx * g.ny));
        double m[3];
        for (int c = 0; c < 3; ++c) m[c] = (double)M[c * N + cell];
        if (i + 1 < g.nx) {
            double s = 0;
            for (int c = 0; c < 3; ++c) { const double d = ((double)M[c * N + cell + 1] - m[c]) * inv; s += d * d; }
            ex += s * idx2;
        }
        if (j + 1 < g.ny) {
            double s = 0;
            for (int c = 0; c < 3; ++c) { const double d = ((double)M[c * N + cell + g.nx] - m[c]) * inv; s += d * d; }
            ex += s * idy2;
        }
        if (k + 1 < g.nz) {
            const size_t st = (size_t)g.nx * g.ny;
            double s = 0;
            for (int c = 0; c < 3; ++c) { const double d = ((double)M[c * N + cell + st] - m[c]) * inv; s += d * d; }
            ex += s * idz2;
        }
        an += (m[1] * m[1] + m[2] * m[2]) * inv * inv;
        de += (double)H[cell] * m[0] + (double)H[N + cell] * m[1] + (double)H[2 * N + cell] * m[2];
        ze += hx * m[0] + hy * m[1] + hz * m[2];
    }
    const double s0 = block_sum(ex, red);
    const double s1 = block_sum(an, red);
    const double s2 = block_sum(de, red);
    const double s3 = block_sum(ze, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 0] = s0;
        part[blockIdx.x * 4 + 1] = s1;
        part[blockIdx.x * 4 + 2] = s2;
        part[blockIdx.x * 4 + 3] = s3;
    }
}

__global__ void __launch_bounds__(kEnergyThreads) k_energy_final(int nblocks, double A, double Ku, double V,
                                                                  const double* __restrict__ part,
                                                                  double* __restrict__ out) {
    __shared__ double red[kEnergyThreads / 32];
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int q = 0; q < 4; ++q) acc[q] += part[b * 4 + q];
    double s[4];
    for (int q = 0; q < 4; ++q) s[q] = block_sum(acc[q], red);
    if (threadIdx.x == 0) {
        const double ex = A * V * s[0];
        const double an = Ku * V * s[1];
        const double de = -0.5 * kMu0 * V * s[2];
        const double ze = -kMu0 * V * s[3];
        out[0] = ex + an + de + ze;
        out[1] = ex;
        out[2] = an;
        out[3] = de;
        out[4] = ze;
    }
}

cudaError_t energy_reduce_full(const Geom& g, double Ms, const double Hext[3], const double cell[3], double A,
                               double Ku, const float* M, const float* Hd, double* partials, double* out_dev,
                               cudaStream_t s) {
    const int nb = kEnergyBlocks;
    k_energy_partial<<<nb, kEnergyThreads, 0, s>>>(g, Ms, Hext[0], Hext[1], Hext[2], 1.0 / (cell[0] * cell[0]),
                                                   1.0 / (cell[1] * cell[1]), 1.0 / (cell[2] * cell[2]), M, Hd,
                                                   partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_final<<<1, kEnergyThreads, 0, s>>>(nb, A, Ku, cell[0] * cell[1] * cell[2], partials, out_dev);
    return cudaGetLastError();
}

}  // namespace mmk
