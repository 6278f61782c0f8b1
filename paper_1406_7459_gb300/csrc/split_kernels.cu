// split_kernels.cu -- pass 2 for thick samples, in three kernels.
//
// When a kx plane (3*nz lines of Ly) does not fit in shared memory (nz > 8,
// or large ny*nz), the y and z transforms of Sec. 3 (Eqs. (14)-(16)) run as
// separate kernels on the spectrum workspace, whose row stride is then Ly:
//   k_yfft  forward y FFT of each (kx, c, k) line in place (ny nonzero
//           inputs), or inverse y (all Ly inputs; rows j < ny are kept);
//   k_zconv per kx and a chunk of W consecutive ky: forward z FFT of the
//           3W z-lines (nz nonzero inputs), the member-wise product with the
//           real symmetric tensor spectrum (Eq. (15)), inverse z, rows
//           k < nz written back (Eq. (16)).
#include "mm_internal.h"

namespace mmk {

__global__ void __launch_bounds__(256) k_yfft(Geom g, int lines_per_cta, int inverse, float2* __restrict__ S) {
    extern __shared__ float2 sm[];
    pdl_wait();
    const int lstride = padded_len(g.Ly);
    const int total = g.Hx * 3 * g.nz;
    const int l0 = blockIdx.x * lines_per_cta;
    const int nl = min(lines_per_cta, total - l0);
    float2* buf = sm;
    float2* scratch = sm + lines_per_cta * lstride;
    const int nin = inverse ? g.Ly : g.ny;
    for (int idx = threadIdx.x; idx < nl * nin; idx += blockDim.x) {
        const int l = idx / nin, j = idx - l * nin;
        buf[l * lstride + padi(j)] = S[(size_t)(l0 + l) * g.Jst + j];
    }
    fft_lines(buf, scratch, lstride, nl, nl, g.py, g.twy, nin, inverse != 0);
    const int nout = inverse ? g.ny : g.Ly;
    for (int idx = threadIdx.x; idx < nl * nout; idx += blockDim.x) {
        const int l = idx / nout, j = idx - l * nout;
        S[(size_t)(l0 + l) * g.Jst + j] = buf[l * lstride + padi(j)];
    }
}

__global__ void __launch_bounds__(256) k_zconv(Geom g, int W, float2* __restrict__ S) {
    extern __shared__ float2 sm[];
    pdl_wait();
    const int nchunk = (g.Ly + W - 1) / W;
    const int kx = blockIdx.x / nchunk;
    const int ky0 = (blockIdx.x % nchunk) * W;
    const int wn = min(W, g.Ly - ky0);
    const int lstride = padded_len(g.Lz);
    const int nz = g.nz;
    float2* buf = sm;                         // line (c*W + w), element kz
    float2* scratch = sm + 3 * W * lstride;
    const float2* base = S + (size_t)kx * 3 * nz * g.Jst;
    for (int idx = threadIdx.x; idx < 3 * nz * W; idx += blockDim.x) {
        const int w = idx % W;
        const int ck = idx / W;               // c*nz + k
        const int c = ck / nz, k = ck - c * nz;
        buf[(c * W + w) * lstride + padi(k)] =
            (w < wn) ? base[(size_t)ck * g.Jst + ky0 + w] : make_float2(0.f, 0.f);
    }
    fft_lines(buf, scratch, lstride, 3 * W, 3 * W, g.pz, g.twz, nz, false);
    const float* Kp = g.Kt + (size_t)kx * g.Hz * g.Hy * 6;
    for (int idx = threadIdx.x; idx < wn * g.Lz; idx += blockDim.x) {
        const int w = idx % wn, kz = idx / wn;
        const int ky = ky0 + w;
        int kyp = ky, kzp = kz;
        float sy = 1.f, sz = 1.f;
        if (2 * ky > g.Ly) { kyp = g.Ly - ky; sy = -1.f; }
        if (2 * kz > g.Lz) { kzp = g.Lz - kz; sz = -1.f; }
        const float* kk = Kp + ((size_t)kzp * g.Hy + kyp) * 6;
        const float kxx = __ldg(kk + 0), kxy = sy * __ldg(kk + 1), kxz = sz * __ldg(kk + 2);
        const float kyy = __ldg(kk + 3), kyz = sy * sz * __ldg(kk + 4), kzz = __ldg(kk + 5);
        const int e = padi(kz);
        const float2 mx = buf[(0 * W + w) * lstride + e];
        const float2 my = buf[(1 * W + w) * lstride + e];
        const float2 mz = buf[(2 * W + w) * lstride + e];
        buf[(0 * W + w) * lstride + e] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
        buf[(1 * W + w) * lstride + e] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
        buf[(2 * W + w) * lstride + e] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
    }
    fft_lines(buf, scratch, lstride, 3 * W, 3 * W, g.pz, g.twz, g.Lz, true);
    for (int idx = threadIdx.x; idx < 3 * nz * wn; idx += blockDim.x) {
        const int w = idx % wn;
        const int ck = idx / wn;
        const int c = ck / nz, k = ck - c * nz;
        S[(size_t)kx * 3 * nz * g.Jst + (size_t)ck * g.Jst + ky0 + w] = buf[(c * W + w) * lstride + padi(k)];
    }
}

static int split_lines_per_cta(const Geom& g) {
    const size_t line = (size_t)padded_len(g.Ly) * sizeof(float2);
    int n = (int)(32768 / (2 * line));
    return n < 1 ? 1 : (n > 16 ? 16 : n);
}

static int split_chunk(const Geom& g) {
    const size_t line = (size_t)padded_len(g.Lz) * sizeof(float2);
    int w = (int)(65536 / (2 * 3 * line));
    return w < 1 ? 1 : (w > 32 ? 32 : w);
}

size_t split_smem_y(const Geom& g) {
    return (size_t)2 * split_lines_per_cta(g) * padded_len(g.Ly) * sizeof(float2);
}
size_t split_smem_z(const Geom& g) { return (size_t)2 * 3 * split_chunk(g) * padded_len(g.Lz) * sizeof(float2); }

cudaError_t configure_split_kernels(const Geom& g) {
    cudaError_t e = cudaFuncSetAttribute(k_yfft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem_y(g));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zconv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem_z(g));
}

cudaError_t launch_split_plane(const Geom& g, float2* S, cudaStream_t s) {
    const int lp = split_lines_per_cta(g);
    const int total = g.Hx * 3 * g.nz;
    const int gy = (total + lp - 1) / lp;
    // programmatic serialisation: both kernels wait on griddepcontrol first
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cy = launch_config(dim3(gy), 256, split_smem_y(g), s, attr);
    cudaError_t e = cudaLaunchKernelEx(&cy, k_yfft, g, lp, 0, S);
    if (e != cudaSuccess) return e;
    const int W = split_chunk(g);
    const int nchunk = (g.Ly + W - 1) / W;
    cudaLaunchConfig_t cz = launch_config(dim3(g.Hx * nchunk), 256, split_smem_z(g), s, attr);
    e = cudaLaunchKernelEx(&cz, k_zconv, g, W, S);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cy, k_yfft, g, lp, 1, S);
}

}  // namespace mmk
