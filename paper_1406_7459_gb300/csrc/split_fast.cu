// split_fast.cu -- pass 2 for thick power-of-two samples with compile-time
// FFTs: the y transforms and the z transform + tensor product of Sec. 3
// (Eqs. (14)-(16)) as three kernels on the spectrum workspace (row stride
// Ly), for ny in 16 ... 1024 and nz in 1, 2, 4, 8 ... 128.
//
//   k_yfwd_fast<NY>  per batch of (kx, c, k) lines: forward y of the ny
//                    nonzero inputs as the two unpadded halves of the padded
//                    length 2 ny (fast_fft.cuh); X[2m + h] is stored at
//                    position h*NY + m of the line, in place.
//   k_zconv_fast<NZ> per kx and W consecutive y positions: forward z of the
//                    3W z-lines (nz nonzero inputs), the member-wise product
//                    with the real symmetric tensor spectrum (Eq. (15)),
//                    inverse z keeping k < nz (Eq. (16)).
//   k_yinv_fast<NY>  per batch of lines: inverse y keeping j < ny, in place.
//
// All three wait on griddepcontrol before touching the spectrum, so they are
// launched with programmatic serialisation like the x passes.
#include "fast_passes.cuh"

namespace mmk {

constexpr int cmax_i(int a, int b) { return a > b ? a : b; }

template <int NY> struct YLayout {
    using F = Fft2<NY>;
    static constexpr int LPC = cmax_i(256 / (2 * F::G), 1);   // lines per CTA
    static constexpr int THREADS = LPC * 2 * F::G;
    static constexpr size_t BYTES = sizeof(float2) * (2 * NY + 2 * LPC * F::EX + LPC * (2 * NY + 2));
};

template <int NY>
__global__ void __launch_bounds__(YLayout<NY>::THREADS) k_yfwd_fast(Geom g, float2* __restrict__ S) {
    using Lay = YLayout<NY>;
    using F = Fft2<NY>;
    constexpr int P = F::P, Q = F::Q, G = F::G, T = Lay::THREADS, LPC = Lay::LPC;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* ex = tw + 2 * NY;
#pragma unroll
    for (int i = threadIdx.x; i < 2 * NY; i += T) tw[i] = __ldg(g.twy + i);
    pdl_wait();
    __syncthreads();
    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int lc = grp >> 1, h = grp & 1;
    const int line = blockIdx.x * LPC + lc;
    const bool on = line < g.Hx * 3 * g.nz;
    float2* ln = S + (size_t)(on ? line : 0) * g.Jst;
    if (on && t < Q) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = ln[t + Q * q];
        if (h) F::odd_input(v, t, tw);
        F::stepA(v, t, tw, ex + grp * F::EX, false);
    }
    __syncthreads();
    if (on && t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, false);
#pragma unroll
        for (int q = 0; q < Q; ++q) ln[h * NY + t + P * q] = w[q];      // X[2 n + h] at h*NY + n
    }
}

template <int NY>
__global__ void __launch_bounds__(YLayout<NY>::THREADS) k_yinv_fast(Geom g, float2* __restrict__ S) {
    using Lay = YLayout<NY>;
    using F = Fft2<NY>;
    constexpr int P = F::P, Q = F::Q, G = F::G, T = Lay::THREADS, LPC = Lay::LPC, LS = 2 * NY + 2;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* ex = tw + 2 * NY;
    float2* ob = ex + 2 * LPC * F::EX;       // [lc][h*NY + n]
#pragma unroll
    for (int i = threadIdx.x; i < 2 * NY; i += T) tw[i] = __ldg(g.twy + i);
    pdl_wait();
    __syncthreads();
    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int lc = grp >> 1, h = grp & 1;
    const int total = g.Hx * 3 * g.nz;
    const int line = blockIdx.x * LPC + lc;
    const bool on = line < total;
    float2* ln = S + (size_t)(on ? line : 0) * g.Jst;
    if (on && t < Q) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = ln[h * NY + t + Q * q];
        F::stepA(v, t, tw, ex + grp * F::EX, true);
    }
    __syncthreads();
    if (on && t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, true);
        if (h) F::odd_output(w, t, tw);
#pragma unroll
        for (int q = 0; q < Q; ++q) ob[lc * LS + h * NY + t + P * q] = w[q];
    }
    __syncthreads();
    // x[j] = (even half)[j] + (odd half)[j], j < ny, written over the line
#pragma unroll
    for (int idx = threadIdx.x; idx < LPC * NY; idx += T) {
        const int l = idx / NY, n = idx % NY;
        const int gl = blockIdx.x * LPC + l;
        if (gl < total) S[(size_t)gl * g.Jst + n] = cadd(ob[l * LS + n], ob[l * LS + NY + n]);
    }
}

template <int NZ> struct ZLayout {
    using F = Fft2<NZ>;
    static constexpr int W = cmax_i(64 / F::G, 1);            // y positions per CTA (384 threads)
    static constexpr int THREADS = 6 * W * F::G;
    static constexpr int ZP = 2 * NZ + 1;                        // z-line stride in shared memory
    static constexpr int MINB = NZ >= 128 ? 3 : 1;               // CTAs per SM the registers must allow
    static constexpr size_t BYTES = sizeof(float2) * (2 * NZ + 3 * W * ZP + 6 * W * F::EX);
};

template <int NZ>
__global__ void __launch_bounds__(ZLayout<NZ>::THREADS, ZLayout<NZ>::MINB) k_zconv_fast(Geom g, const float* __restrict__ Kt, float2* __restrict__ S) {
    using Lay = ZLayout<NZ>;
    using F = Fft2<NZ>;
    constexpr int P = F::P, Q = F::Q, G = F::G, T = Lay::THREADS, W = Lay::W, ZP = Lay::ZP;
    extern __shared__ float2 sm[];
    float2* tw = sm;                          // W_{2NZ}^k
    float2* zs = tw + 2 * NZ;                 // [c*W + w][z], z < 2 NZ
    float2* ex = zs + 3 * W * ZP;
    const int nchunk = g.Ly / W;
    const int kx = blockIdx.x / nchunk;
    const int p0 = (blockIdx.x % nchunk) * W;
    const int NYh = g.Ly / 2;
#pragma unroll
    for (int i = threadIdx.x; i < 2 * NZ; i += T) tw[i] = __ldg(g.twz + i);
    pdl_wait();
    const float2* base = S + (size_t)kx * 3 * NZ * g.Jst + p0;
#pragma unroll
    for (int idx = threadIdx.x; idx < 3 * NZ * W; idx += T) {
        const int w = idx % W, ck = idx / W;          // ck = c*NZ + k
        const int c = ck / NZ, k = ck % NZ;
        zs[(c * W + w) * ZP + k] = base[(size_t)ck * g.Jst + w];
    }
    __syncthreads();
    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    const int zl = grp >> 1, h = grp & 1;              // z-line zl = c*W + w
    float2* zln = zs + zl * ZP;
    // forward z, pruned input: Z[2 m + h] at position h*NZ + m
    if (t < Q) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = zln[t + Q * q];
        if (h) F::odd_input(v, t, tw);
        F::stepA(v, t, tw, ex + grp * F::EX, false);
    }
    __syncthreads();
    if (t < P) {
        float2 w[Q];
        F::stepB(w, t, ex + grp * F::EX, false);
#pragma unroll
        for (int q = 0; q < Q; ++q) zln[h * NZ + t + P * q] = w[q];
    }
    __syncthreads();
    // tensor product per (y position, kz); the y position p holds
    // ky = 2 (p mod ny) + p / ny (the forward y kernel's order)
    const float* Kp = Kt + (size_t)kx * g.Hz * g.Hy * 6;
#pragma unroll
    for (int idx = threadIdx.x; idx < W * 2 * NZ; idx += T) {
        const int w = idx % W, zp = idx / W;
        const int kz = 2 * (zp % NZ) + zp / NZ;
        const int p = p0 + w;
        const int ky = 2 * (p % NYh) + p / NYh;
        int kyp = ky, kzp = kz;
        float sy = 1.f, sz = 1.f;
        if (2 * ky > g.Ly) { kyp = g.Ly - ky; sy = -1.f; }
        if (2 * kz > g.Lz) { kzp = g.Lz - kz; sz = -1.f; }
        const float* kk = Kp + ((size_t)kzp * g.Hy + kyp) * 6;
        const float kxx = __ldg(kk + 0), kxy = sy * __ldg(kk + 1), kxz = sz * __ldg(kk + 2);
        const float kyy = __ldg(kk + 3), kyz = sy * sz * __ldg(kk + 4), kzz = __ldg(kk + 5);
        const float2 mx = zs[(0 * W + w) * ZP + zp];
        const float2 my = zs[(1 * W + w) * ZP + zp];
        const float2 mz = zs[(2 * W + w) * ZP + zp];
        zs[(0 * W + w) * ZP + zp] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
        zs[(1 * W + w) * ZP + zp] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
        zs[(2 * W + w) * ZP + zp] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
    }
    __syncthreads();
    // inverse z, pruned output: x[k] = IFFT(even)[k] + W^{-k} IFFT(odd)[k]
    float2 w[Q];
    if (t < Q) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = zln[h * NZ + t + Q * q];
        F::stepA(v, t, tw, ex + grp * F::EX, true);
    }
    __syncthreads();
    if (t < P) {
        F::stepB(w, t, ex + grp * F::EX, true);
        if (h) F::odd_output(w, t, tw);
    }
    __syncthreads();                          // zs is rewritten below
    if (t < P) {
#pragma unroll
        for (int q = 0; q < Q; ++q) zln[h * NZ + t + P * q] = w[q];
    }
    __syncthreads();
    float2* out = S + (size_t)kx * 3 * NZ * g.Jst + p0;
#pragma unroll
    for (int idx = threadIdx.x; idx < 3 * NZ * W; idx += T) {
        const int w2 = idx % W, ck = idx / W;
        const int c = ck / NZ, k = ck % NZ;
        const float2* l = zs + (c * W + w2) * ZP;
        out[(size_t)ck * g.Jst + w2] = cadd(l[k], l[NZ + k]);
    }
}

// Thin z (nz <= 8): one y position per thread, its 3 nz values held in
// registers through the z transform, the product and the inverse
// (zconv_column); consecutive threads take consecutive positions, so every
// (c, k) row is read and written coalesced, and no barrier is needed.
constexpr int kZcolThreads = 128;

template <int NZ>
__global__ void __launch_bounds__(kZcolThreads) k_zcol_fast(Geom g, const float* __restrict__ Kt, float2* __restrict__ S) {
    pdl_wait();
    const int p = blockIdx.x * kZcolThreads + threadIdx.x;      // y position within the kx plane
    const int kx = blockIdx.y;
    if (p >= g.Ly) return;
    const int NYh = g.Ly / 2;
    const int ky = 2 * (p % NYh) + p / NYh;                      // the forward y kernel's order
    float2* base = S + (size_t)kx * 3 * NZ * g.Jst + p;
    float2 m[3][NZ];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < NZ; ++k) m[c][k] = base[(size_t)(c * NZ + k) * g.Jst];
    zconv_column<NZ>(m, Kt + (size_t)kx * g.Hz * g.Hy * 6, g.Hy, g.Ly, ky, g.twz);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < NZ; ++k) base[(size_t)(c * NZ + k) * g.Jst] = m[c][k];
}

template <int NY> static void fill_y(FastSplitFns* f) {
    f->yf = k_yfwd_fast<NY>;
    f->yi = k_yinv_fast<NY>;
    f->ylpc = YLayout<NY>::LPC;
    f->ty = YLayout<NY>::THREADS;
    f->sy = YLayout<NY>::BYTES;
}
template <int NZ> static void fill_z(FastSplitFns* f) {
    f->zc = k_zconv_fast<NZ>;
    f->zw = ZLayout<NZ>::W;
    f->tz = ZLayout<NZ>::THREADS;
    f->sz = ZLayout<NZ>::BYTES;
}
template <int NZ> static void fill_zcol(FastSplitFns* f) {
    f->zc = k_zcol_fast<NZ>;
    f->zw = 0;                               // marks the one-position-per-thread kernel
    f->tz = kZcolThreads;
    f->sz = 0;
}

bool fast_split_lookup(int ny, int nz, FastSplitFns* f) {
    switch (ny) {
        case 16: fill_y<16>(f); break;
        case 32: fill_y<32>(f); break;
        case 64: fill_y<64>(f); break;
        case 128: fill_y<128>(f); break;
        case 256: fill_y<256>(f); break;
        case 512: fill_y<512>(f); break;
        case 1024: fill_y<1024>(f); break;
        default: return false;
    }
    switch (nz) {
        case 1: fill_zcol<1>(f); break;
        case 2: fill_zcol<2>(f); break;
        case 4: fill_zcol<4>(f); break;
        case 8: fill_zcol<8>(f); break;
        case 16: fill_z<16>(f); break;
        case 32: fill_z<32>(f); break;
        case 64: fill_z<64>(f); break;
        case 128: fill_z<128>(f); break;
        default: return false;
    }
    return true;
}

cudaError_t configure_fast_split(const FastSplitFns& f) {
    cudaError_t e = cudaFuncSetAttribute(f.yf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sy);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f.yi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sy);
    if (e == cudaSuccess && f.sz) e = cudaFuncSetAttribute(f.zc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sz);
    return e;
}

cudaError_t launch_fast_split(const Geom& g, const FastSplitFns& f, const float* Kt, float2* S, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    const int lines = g.Hx * 3 * g.nz;
    const int gy = (lines + f.ylpc - 1) / f.ylpc;
    cudaLaunchConfig_t cy = launch_config(dim3(gy), f.ty, f.sy, s, attr);
    cudaError_t e = cudaLaunchKernelEx(&cy, f.yf, g, S);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cz = f.zw ? launch_config(dim3(g.Hx * (g.Ly / f.zw)), f.tz, f.sz, s, attr)
                                 : launch_config(dim3(1), f.tz, 0, s, attr);
    if (!f.zw) cz.gridDim = dim3((g.Ly + f.tz - 1) / f.tz, g.Hx);
    e = cudaLaunchKernelEx(&cz, f.zc, g, Kt, S);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cy, f.yi, g, S);
}

cudaError_t launch_split_xstep(const Geom& g, const FastSplitFns& f2, const FastStepFns& fs, const LlgCoef& c,
                               int mode, const float* Kt, float2* S, const float* M, float* out, int* flag,
                               cudaStream_t s) {
    cudaError_t e = launch_fast_split(g, f2, Kt, S, s);
    if (e != cudaSuccess) return e;
    // the x-step kernel reads its tile of S (all kx of R rows of a layer)
    // into shared memory before it writes the same tile back: in place
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / fs.rb)), fs.tb, fs.sb, s, attr);
    return cudaLaunchKernelEx(&cfg, fs.kb[mode], g, c, (const float2*)S, mode == kModeStep ? S : (float2*)nullptr,
                              M, out, mode == kModeStep ? flag : (int*)nullptr);
}

}  // namespace mmk
