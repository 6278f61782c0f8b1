// split_fast.cu -- pass 2 for thick power-of-two samples with compile-time
// FFTs: the y transforms and the z transform + tensor product of Sec. 3
// (Eqs. (14)-(16)) as three kernels on the spectrum workspace (row stride
// Ly), for ny in 16 ... 1024 and nz in 1, 2, 4, 8 ... 128.
//
//   k_yfwd_fast<NY>  per batch of (kx, c, k) lines: forward y of the ny
//                    nonzero inputs as the two unpadded halves of the padded
//                    length 2 ny (fast_fft.cuh); X[2m + h] is stored at
//                    position h*NY + m of the line, in place.
//   k_zconv_fast<NZ> per kx and W consecutive y positions (nz >= 16):
//                    forward z of the 3W z-lines (nz nonzero inputs), the
//                    member-wise product with the real symmetric tensor
//                    spectrum (Eq. (15)), inverse z keeping k < nz (Eq. (16));
//   k_zcol_fast<NZ>  the same for nz <= 8, one y position per thread.
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

// NY >= 512: the step B registers of a 32-point DFT would leave one CTA per
// SM; the bound asks for two
template <int NY> constexpr int yinv_min_blocks() { return NY >= 512 ? 2 : 1; }

template <int NY>
__global__ void __launch_bounds__(YLayout<NY>::THREADS, yinv_min_blocks<NY>()) k_yinv_fast(Geom g, float2* __restrict__ S) {
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

// z convolution for nz >= 16.  A CTA takes W consecutive y positions of one
// kx plane and keeps their 3 nz-point z lines in shared memory as [c][z][w]
// (w fastest): every warp reads and writes whole W-wide rows, so no access
// has a bank conflict, and the rows of S are staged with 16-byte copies.
// Each half h of the padded z spectrum (kz = 2m + h) is one unpadded FFT of
// length nz = P Q in the index split of Fft2, done in place:
//   strided items (c, t, w), t < Q: positions t + Q p, DFT_P, twiddle W^{ta};
//   block items (a, w), a < P, all three components: positions a Q + b,
//     DFT_Q gives X[a + P b] (b < Q); the product with the tensor spectrum
//     (Eq. (15)) for the Q wavenumbers kz = 2 (a + P b) + h; then the first
//     step of the inverse on the conjugated product: DFT_Q over b, twiddle
//     W^{s a}, stored at a Q + s;
//   strided items (c, s, w): positions s + Q a, DFT_P and conjugation give
//     the inverse transform at z = s + Q r, in natural order.
// Half 0 works out of the input buffer xb into wb and leaves its inverse in
// wb; half 1 works in xb in place and adds W_{2nz}^{-z} times its inverse to
// wb's (the pruned inverse of Sec. 2, step (5)) on the way out to S.
template <int NZ> struct ZLayout {
    using F = Fft2<NZ>;
    static constexpr int W = (NZ == 16 || NZ == 32) ? 32 : 16;   // y positions per CTA
    static constexpr int NB = F::P * W;                           // block items
    static constexpr int NS = 3 * F::Q * W;                       // strided items
    // one block item per thread where the strided items split evenly over
    // them (P = Q), else one strided item per thread (P = 2Q)
    static constexpr int THREADS = NS % NB == 0 ? NB : NS;
    static constexpr int MINB = NS % NB == 0 ? 512 / THREADS : 2;  // CTAs per SM the registers must allow
    static constexpr int LINE = NZ * W;                           // one component's lines (complex)
    static constexpr size_t BYTES = sizeof(float2) * (2 * NZ + 6 * LINE);
};

template <int NZ>
__global__ void __launch_bounds__(ZLayout<NZ>::THREADS, ZLayout<NZ>::MINB) k_zconv_fast(Geom g, const float* __restrict__ Kt, float2* __restrict__ S) {
    using Lay = ZLayout<NZ>;
    using F = Fft2<NZ>;
    constexpr int P = F::P, Q = F::Q, T = Lay::THREADS, W = Lay::W, LINE = Lay::LINE;
    constexpr int NS = Lay::NS;
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;                          // W_{2NZ}^k, k < 2 NZ
    float2* xb = tw + 2 * NZ;                 // [c][z][w]
    float2* wb = xb + 3 * LINE;
    const int nchunk = g.Ly / W;
    const int kx = blockIdx.x / nchunk;
    const int p0 = (blockIdx.x - kx * nchunk) * W;
    for (int i = threadIdx.x; i < 2 * NZ; i += T) tw[i] = __ldg(g.twz + i);
    pdl_wait();
    float2* plane = S + (size_t)kx * 3 * NZ * g.Jst + p0;
#pragma unroll
    for (int i = threadIdx.x; i < 3 * NZ * (W / 2); i += T) {
        const int ck = i / (W / 2), j = i - ck * (W / 2);
        __pipeline_memcpy_async(xb + ck * W + 2 * j, plane + (size_t)ck * g.Jst + 2 * j, 2 * sizeof(float2));
    }
    __pipeline_commit();
    // this thread's y position (the same in every item: T is a multiple of W)
    const int w = threadIdx.x % W, a = threadIdx.x / W;
    const int NYh = g.Ly / 2;
    const int py = p0 + w;
    const int ky = 2 * (py % NYh) + py / NYh;             // the forward y kernel's order
    int kyp = ky;
    float sy = 1.f;
    if (2 * ky > g.Ly) { kyp = g.Ly - ky; sy = -1.f; }
    const float* Kp = Kt + ((size_t)kx * g.Hz * g.Hy + kyp) * 6;
    __pipeline_wait_prior(0);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2* buf = h ? xb : wb;
        // forward, strided items: xb -> buf
#pragma unroll
        for (int i = threadIdx.x; i < NS; i += T) {
            const int t = (i / W) % Q, c = i / (W * Q);
            float2 v[P];
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = xb[(c * NZ + t + Q * p) * W + w];
            if (h) F::odd_input(v, t, tw);
            F::stepA_reg(v, t, tw, false);
#pragma unroll
            for (int p = 0; p < P; ++p) buf[(c * NZ + t + Q * p) * W + w] = v[p];
        }
        __syncthreads();
        // block items: DFT_Q, tensor product, first inverse step
        if (Lay::NB == T || threadIdx.x < Lay::NB) {
            float2 u[3][Q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int b = 0; b < Q; ++b) u[c][b] = buf[(c * NZ + a * Q + b) * W + w];
                dftp<Q>(u[c]);
            }
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const int kz = 2 * (a + P * b) + h;
                int kzp = kz;
                float sz = 1.f;
                if (kz > NZ) { kzp = 2 * NZ - kz; sz = -1.f; }
                const float2* kk = reinterpret_cast<const float2*>(Kp + (size_t)kzp * g.Hy * 6);
                const float2 k01 = __ldg(kk), k23 = __ldg(kk + 1), k45 = __ldg(kk + 2);
                const float kxx = k01.x, kxy = sy * k01.y, kxz = sz * k23.x;
                const float kyy = k23.y, kyz = sy * sz * k45.x, kzz = k45.y;
                const float2 mx = u[0][b], my = u[1][b], mz = u[2][b];
                // conjugated product: the inverse runs as conj(DFT(conj(.)))
                u[0][b] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, -(kxx * mx.y + kxy * my.y + kxz * mz.y));
                u[1][b] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, -(kxy * mx.y + kyy * my.y + kyz * mz.y));
                u[2][b] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, -(kxz * mx.y + kyz * my.y + kzz * mz.y));
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dftp<Q>(u[c]);
#pragma unroll
                for (int s2 = 0; s2 < Q; ++s2) {
                    const float2 v = s2 ? cmul(u[c][s2], tw[2 * s2 * a]) : u[c][s2];
                    buf[(c * NZ + a * Q + s2) * W + w] = v;
                }
            }
        }
        __syncthreads();
        // inverse, strided items: natural order, conjugated back
#pragma unroll
        for (int i = threadIdx.x; i < NS; i += T) {
            const int s2 = (i / W) % Q, c = i / (W * Q);
            float2 v[P];
#pragma unroll
            for (int r = 0; r < P; ++r) v[r] = buf[(c * NZ + s2 + Q * r) * W + w];
            dftp<P>(v);
            if (h == 0) {
#pragma unroll
                for (int r = 0; r < P; ++r) wb[(c * NZ + s2 + Q * r) * W + w] = cconj(v[r]);
            } else {
                // x[z] = y0[z] + W_{2NZ}^{-z} y1[z],  z = s2 + Q r
                F::odd_input(v, s2, tw);
#pragma unroll
                for (int r = 0; r < P; ++r) {
                    const int z = s2 + Q * r;
                    plane[(size_t)(c * NZ + z) * g.Jst + w] = cadd(wb[(c * NZ + z) * W + w], cconj(v[r]));
                }
            }
        }
        // half 1 reads only xb (untouched by half 0) before its next barrier
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
                               cudaStream_t s, float* Mcopy) {
    cudaError_t e = launch_fast_split(g, f2, Kt, S, s);
    if (e != cudaSuccess) return e;
    // the x-step kernel reads its tile of S (all kx of R rows of a layer)
    // into shared memory before it writes the same tile back: in place
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / fs.rb)), fs.tb, fs.sb, s, attr);
    return cudaLaunchKernelEx(&cfg, fs.kb[mode], g, c, (const float2*)S, mode == kModeStep ? S : (float2*)nullptr,
                              M, out, mode == kModeStep ? flag : (int*)nullptr,
                              mode == kModeStep ? Mcopy : (float*)nullptr);
}

}  // namespace mmk
