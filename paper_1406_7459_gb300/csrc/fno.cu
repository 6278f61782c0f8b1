// fno.cu -- Fourier-neural-operator surrogate of the demag field: BF16
// storage, FP32 accumulation, forward, backward and Adam on the GPU.
//
// Not in the paper.  The network maps a magnetisation increment dM/Ms on an
// H x W film to its demag field H_demag(dM)/Ms (H_demag is linear in M, so
// between exact refreshes H_demag(M) = H_demag(M_ref) + Ms FNO((M-M_ref)/Ms)).
//   v0 = P [x; y/H; x/W] + p (two coordinate channels let the operator see
//   the film's edges);  for l < L: u = W_l v + b_l + S_l(v), v = gelu(u) (not on
//   the last layer);  y = Q v + q;  S_l keeps kx < m and ky in
//   {0..m-1} U {H-m..H-1}, with complex weights R_l[c][o] per mode.
// Dense contractions (the x-direction mode transforms, the channel mixes)
// run on the fifth-generation tensor cores (tcgen05 MMAs with the FP32
// accumulator in tensor memory, gemm_tc.cuh); the small complex transforms along y and the per-mode
// channel mix run as FP32 kernels.  Parameters live as an FP32 master copy
// (Adam moments beside it) and a BF16 copy for the GEMMs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mm.h"
#include "mm_internal.h"
#include "gemm_tc.cuh"

using namespace mmk;

namespace mmk {

// ------------------------------------------------------------ BF16 GEMM --
// The tcgen05 kernel of gemm_tc.cuh; the tile width follows N.  A product
// with fewer rows than a 128-row tile and more columns (the per-sample
// channel mix, C x C times C x HW) runs as its transpose C^T = B^T A^T.
template <int BN> static cudaError_t gemm_launch(const GemmArgs& g, int batch, cudaStream_t s) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + kTcM - 1) / kTcM, batch);
    k_gemm_tc<BN><<<grid, kTcThreads, gemm_tc_smem<BN>(), s>>>(g);
    return cudaGetLastError();
}

static cudaError_t gemm(GemmArgs g, int batch, int* err, cudaStream_t s) {
    g.err = err;
    if (g.M < kTcM && g.N > g.M) {
        GemmArgs t = g;
        t.A = g.B; t.B = g.A; t.M = g.N; t.N = g.M;
        t.sam = g.sbn; t.sak = g.sbk; t.sbk = g.sak; t.sbn = g.sam;
        t.scm = g.scn; t.scn = g.scm; t.zA = g.zB; t.zB = g.zA;
        g = t;
    }
    if (g.N <= 32) return gemm_launch<32>(g, batch, s);
    if (g.N <= 64) return gemm_launch<64>(g, batch, s);
    return gemm_launch<128>(g, batch, s);
}

static cudaError_t gemm_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_tc_smem<32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem<64>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_tc_smem<128>());
    return e;
}

// ------------------------------------------------------ small FP32 kernels --
__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n, float scale) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(scale * in[i]);
}

// 1x1 channel map per pixel: out[b][o][p] = sum_c Wt[o][c] in[b][c][p] + bias[o]
// (trans: Wt stored [c][o], i.e. the transposed map)
__global__ void k_pointwise(const float* __restrict__ in, int cin, const float* __restrict__ Wt,
                            const float* __restrict__ bias, int cout, long long npix, int B, int trans,
                            float* __restrict__ outf) {
    const long long total = (long long)B * npix;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        const long long p = t - (long long)b * npix;
        float x[64];
        for (int c = 0; c < cin; ++c) x[c] = in[((long long)b * cin + c) * npix + p];
        for (int o = 0; o < cout; ++o) {
            float s = bias ? bias[o] : 0.f;
            for (int c = 0; c < cin; ++c) s += (trans ? Wt[c * cout + o] : Wt[o * cin + c]) * x[c];
            outf[((long long)b * cout + o) * npix + p] = s;
        }
    }
}

// y-direction transform of the x-mode coefficients (complex, FP32):
// out[b][c][iy][kx] = sum_y F[iy][y] * A[b][c][y][kx] (+/- conj by sign)
// A: re at [.. y][kx], im at [.. y][m + kx] with row stride ldA (= 2m).
// F: Fre/Fim (ny_out x H).  out: re/im planes [bc][iy][kx].
__global__ void k_ydft(const float* __restrict__ A, int ldA, int H, int m, const float* __restrict__ Fre,
                       const float* __restrict__ Fim, int ny_out, int BC, float* __restrict__ ore,
                       float* __restrict__ oim, float scale, int double_kx) {
    const long long total = (long long)BC * ny_out * m;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(t % m);
        const int iy = (int)((t / m) % ny_out);
        const long long bc = t / ((long long)m * ny_out);
        const float* a = A + bc * H * ldA;
        float sr = 0.f, si = 0.f;
        for (int y = 0; y < H; ++y) {
            const float fr = Fre[iy * H + y], fi = Fim[iy * H + y];
            const float ar = a[y * ldA + kx], ai = a[y * ldA + m + kx];
            sr += fr * ar - fi * ai;
            si += fr * ai + fi * ar;
        }
        const float sc = (double_kx && kx > 0) ? 2.f * scale : scale;
        ore[t] = sc * sr;
        oim[t] = sc * si;
    }
}

// inverse along y: Z[b][o][y][kx] (re), Z[.][.][y][m + kx] (im) =
// sum_iy G[y][iy] * w[b][o][iy][kx]
__global__ void k_yidft(const float* __restrict__ wre, const float* __restrict__ wim, int nky, int m,
                        const float* __restrict__ Gre, const float* __restrict__ Gim, int H, int BC,
                        float* __restrict__ Z) {
    const long long total = (long long)BC * H * m;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(t % m);
        const int y = (int)((t / m) % H);
        const long long bc = t / ((long long)m * H);
        const float* wr = wre + bc * nky * m;
        const float* wi = wim + bc * nky * m;
        float sr = 0.f, si = 0.f;
        for (int iy = 0; iy < nky; ++iy) {
            const float gr = Gre[y * nky + iy], gi = Gim[y * nky + iy];
            sr += gr * wr[iy * m + kx] - gi * wi[iy * m + kx];
            si += gr * wi[iy * m + kx] + gi * wr[iy * m + kx];
        }
        Z[(bc * H + y) * 2 * m + kx] = sr;
        Z[(bc * H + y) * 2 * m + m + kx] = si;
    }
}

// per-mode channel mix: out[b][o][mode] = sum_c R[c][o][mode] in[b][c][mode]
// (conjT: out[b][c][mode] = sum_o conj(R[c][o][mode]) in[b][o][mode])
__global__ void k_modemix(const float* __restrict__ ire, const float* __restrict__ iim, const float* __restrict__ Rre,
                          const float* __restrict__ Rim, int C, int nmode, int B, int conjT, float* __restrict__ ore,
                          float* __restrict__ oim) {
    const long long total = (long long)B * C * nmode;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int md = (int)(t % nmode);
        const int o = (int)((t / nmode) % C);
        const int b = (int)(t / ((long long)nmode * C));
        float sr = 0.f, si = 0.f;
        for (int c = 0; c < C; ++c) {
            const long long ri = conjT ? ((long long)o * C + c) * nmode + md : ((long long)c * C + o) * nmode + md;
            const float rr = Rre[ri], rim = conjT ? -Rim[ri] : Rim[ri];
            const float xr = ire[((long long)b * C + c) * nmode + md], xi = iim[((long long)b * C + c) * nmode + md];
            sr += rr * xr - rim * xi;
            si += rr * xi + rim * xr;
        }
        ore[t] = sr;
        oim[t] = si;
    }
}

// dR[c][o][mode] += sum_b dw[b][o][mode] * conj(vh[b][c][mode])
__global__ void k_dR(const float* __restrict__ dwr, const float* __restrict__ dwi, const float* __restrict__ vr,
                     const float* __restrict__ vi, int C, int nmode, int B, float* __restrict__ gre,
                     float* __restrict__ gim) {
    const long long total = (long long)C * C * nmode;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int md = (int)(t % nmode);
        const int o = (int)((t / nmode) % C);
        const int c = (int)(t / ((long long)nmode * C));
        float sr = 0.f, si = 0.f;
        for (int b = 0; b < B; ++b) {
            const float gr = dwr[((long long)b * C + o) * nmode + md], gi = dwi[((long long)b * C + o) * nmode + md];
            const float ar = vr[((long long)b * C + c) * nmode + md], ai = -vi[((long long)b * C + c) * nmode + md];
            sr += gr * ar - gi * ai;
            si += gr * ai + gi * ar;
        }
        gre[t] += sr;
        gim[t] += si;
    }
}

// lift: out[b][o][p] = sum_{c<3} P[o][c] x[b][c][p] + P[o][3] y/H + P[o][4] x/W + bias[o]
__global__ void k_lift(const float* __restrict__ in, const float* __restrict__ P, const float* __restrict__ bias,
                       int C, int H, int W, int B, float* __restrict__ out) {
    const long long np = (long long)H * W, total = (long long)B * np;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / np);
        const long long p = t - (long long)b * np;
        const float x0 = in[((long long)b * 3 + 0) * np + p], x1 = in[((long long)b * 3 + 1) * np + p];
        const float x2 = in[((long long)b * 3 + 2) * np + p];
        const float cy = (float)(p / W) / (float)H, cx = (float)(p % W) / (float)W;
        for (int o = 0; o < C; ++o)
            out[((long long)b * C + o) * np + p] =
                bias[o] + P[o * 5] * x0 + P[o * 5 + 1] * x1 + P[o * 5 + 2] * x2 + P[o * 5 + 3] * cy + P[o * 5 + 4] * cx;
    }
}

// g[o][c] += sum_p dv[b][o][p] * feature_c(p), features 3 and 4 the coordinates
__global__ void k_outer_lift(const float* __restrict__ a, int C, const float* __restrict__ x, int H, int W, int B,
                             float* __restrict__ g) {
    const int o = blockIdx.y / 5, c = blockIdx.y % 5;
    const long long np = (long long)H * W;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * np;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / np);
        const long long p = t - (long long)b * np;
        const float f = c < 3 ? x[((long long)b * 3 + c) * np + p]
                              : (c == 3 ? (float)(p / W) / (float)H : (float)(p % W) / (float)W);
        acc += a[((long long)b * C + o) * np + p] * f;
    }
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + o * 5 + c, acc);
}

// u[b][o][p] += bias[o]
__global__ void k_add_bias(float* __restrict__ u, const float* __restrict__ bias, int C, long long np, int B) {
    const long long n = (long long)B * C * np;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] += bias[(i / np) % C];
}

// u (FP32) -> v = gelu(u) (BF16) when act, else v = u
__global__ void k_act(const float* __restrict__ u, __nv_bfloat16* __restrict__ v, float* __restrict__ vf, long long n,
                      int act) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = u[i];
        const float y = act ? 0.5f * x * (1.f + erff(x * 0.70710678118654752f)) : x;
        v[i] = __float2bfloat16(y);
        if (vf) vf[i] = y;
    }
}

// du = dv * gelu'(u)
__global__ void k_act_back(const float* __restrict__ u, float* __restrict__ dv, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = u[i];
        const float g = 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.3989422804014327f;
        dv[i] *= g;
    }
}

// loss = mean (y - t)^2 (partial sums, FP64 atomics) and dy = 2 (y - t) / n
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, long long n, float* __restrict__ dy,
                       double* __restrict__ loss) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        dy[i] = 2.f * d / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// sum over pixels of x[b][c][p] into g[c]
__global__ void k_colsum(const float* __restrict__ x, int C, long long npix, int B, float* __restrict__ g) {
    const int c = blockIdx.y;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * npix;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        acc += x[((long long)b * C + c) * npix + (t - (long long)b * npix)];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + c, acc);
}

// g[o][c] += sum_p a[b][o][p] x[b][c][p] (small channel counts, FP32)
__global__ void k_outer(const float* __restrict__ a, int Ca, const float* __restrict__ x, int Cx, long long npix, int B,
                        float* __restrict__ g) {
    const int o = blockIdx.y / Cx, c = blockIdx.y % Cx;
    float acc = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)B * npix;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / npix);
        const long long p = t - (long long)b * npix;
        acc += a[((long long)b * Ca + o) * npix + p] * x[((long long)b * Cx + c) * npix + p];
    }
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if ((threadIdx.x & 31) == 0) atomicAdd(g + o * Cx + c, acc);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float s = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = s;
        w[i] -= lr * (a / c1) / (sqrtf(s / c2) + eps);
    }
}

}  // namespace mmk

// -------------------------------------------------------------- the model --
struct mm_fno {
    int H, W, C, m, L, Bmax;
    long long np;                 // pixels per channel
    cudaStream_t s;
    // parameters: FP32 master, gradient, Adam moments; layout
    // [P (C*5), p (C), R_re (L*C*C*2m*m), R_im, W (L*C*C), b (L*C), Q (3*C), q (3)]
    long long n_params;
    long long oP, op, oRr, oRi, oW, ob, oQ, oq;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16* wb = nullptr;  // BF16 copy of W (per layer C*C)
    int step = 0;
    // mode matrices
    __nv_bfloat16* Fx = nullptr;    // W x 2m: cos | -sin           (forward x, K = W)
    __nv_bfloat16* Gx = nullptr;    // 2m x W: a cos/(HW) | -a sin/(HW) (inverse x)
    __nv_bfloat16* Gxa = nullptr;   // 2m x W: cos | -sin (adjoint of the forward x)
    float *Fyre = nullptr, *Fyim = nullptr;   // 2m x H: exp(-2 pi i ky y / H)
    float *Gyre = nullptr, *Gyim = nullptr;   // H x 2m: exp(+2 pi i ky y / H)
    // activations (per layer): v (bf16 + f32), u (f32), x-modes A1 (f32), vh re/im
    std::vector<float*> vf, u, A1, vhr, vhi;
    std::vector<__nv_bfloat16*> vb;
    float *whr = nullptr, *whi = nullptr, *Z = nullptr, *acc = nullptr, *y = nullptr, *dy = nullptr, *dv = nullptr,
          *du = nullptr, *tmp = nullptr, *dwr = nullptr, *dwi = nullptr;
    __nv_bfloat16 *zb = nullptr, *db16 = nullptr;
    double* dloss = nullptr;
    int* err = nullptr;           // set by a tensor-core GEMM whose wait expired
};

static int fno_fail(int code, const char* msg) { return set_error(code, msg); }

#define FCU(expr)                                                                                    \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) {                                                                     \
            char _m[256];                                                                            \
            snprintf(_m, sizeof(_m), "%s: %s", #expr, cudaGetErrorString(_e));                       \
            return fno_fail(_e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA, _m);             \
        }                                                                                            \
    } while (0)

static int grid1(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// deterministic N(0,1) samples: splitmix64 + Box-Muller
static uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double gauss(uint64_t& st) {
    const double u1 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
}

static void fno_free(mm_fno* f) {
    cudaFree(f->w); cudaFree(f->g); cudaFree(f->m1); cudaFree(f->m2); cudaFree(f->wb);
    cudaFree(f->Fx); cudaFree(f->Gx); cudaFree(f->Gxa);
    cudaFree(f->Fyre); cudaFree(f->Fyim); cudaFree(f->Gyre); cudaFree(f->Gyim);
    for (auto p : f->vf) cudaFree(p);
    for (auto p : f->u) cudaFree(p);
    for (auto p : f->A1) cudaFree(p);
    for (auto p : f->vhr) cudaFree(p);
    for (auto p : f->vhi) cudaFree(p);
    for (auto p : f->vb) cudaFree(p);
    cudaFree(f->whr); cudaFree(f->whi); cudaFree(f->Z); cudaFree(f->acc); cudaFree(f->y); cudaFree(f->dy);
    cudaFree(f->dv); cudaFree(f->du); cudaFree(f->tmp); cudaFree(f->dwr); cudaFree(f->dwi);
    cudaFree(f->zb); cudaFree(f->db16); cudaFree(f->dloss); cudaFree(f->err);
}

extern "C" int mm_fno_create(mm_fno** out, int H, int W, int width, int modes, int layers, int max_batch,
                             unsigned long long seed, void* stream) {
    if (!out) return fno_fail(MM_EINVAL, "out is NULL");
    *out = nullptr;
    if (H < 8 || W < 8 || width < 1 || width > 64 || modes < 1 || 2 * modes > H || 2 * modes >= W || layers < 1 ||
        max_batch < 1)
        return fno_fail(MM_EINVAL, "need H, W >= 8, 1 <= width <= 64, 2 modes <= H, 2 modes < W, layers, batch >= 1");
    mm_fno* f = new (std::nothrow) mm_fno();
    if (!f) return fno_fail(MM_ENOMEM, "host allocation failed");
    f->H = H; f->W = W; f->C = width; f->m = modes; f->L = layers; f->Bmax = max_batch;
    f->np = (long long)H * W;
    f->s = (cudaStream_t)stream;
    const int C = width, m = modes, L = layers;
    const long long nR = (long long)L * C * C * 2 * m * m;
    f->oP = 0; f->op = 5LL * C; f->oRr = f->op + C; f->oRi = f->oRr + nR; f->oW = f->oRi + nR;
    f->ob = f->oW + (long long)L * C * C; f->oQ = f->ob + (long long)L * C; f->oq = f->oQ + 3LL * C;
    f->n_params = f->oq + 3;
    int rc = [&]() -> int {
        const long long n = f->n_params;
        FCU(cudaMalloc(&f->w, 4 * n)); FCU(cudaMalloc(&f->g, 4 * n));
        FCU(cudaMalloc(&f->m1, 4 * n)); FCU(cudaMalloc(&f->m2, 4 * n));
        FCU(cudaMemset(f->m1, 0, 4 * n)); FCU(cudaMemset(f->m2, 0, 4 * n));
        FCU(cudaMalloc(&f->wb, 2LL * L * C * C));
        // seeded initial weights (scale as in the FP64 reference): P ~ N/sqrt5,
        // R ~ N/C, W ~ N/sqrt C, Q ~ N/sqrt C, biases 0
        std::vector<float> h(n, 0.f);
        uint64_t st = seed;
        for (long long i = 0; i < 5LL * C; ++i) h[f->oP + i] = (float)(gauss(st) / std::sqrt(5.0));
        for (long long i = 0; i < 2 * nR; ++i) h[f->oRr + i] = (float)(gauss(st) / C);
        for (long long i = 0; i < (long long)L * C * C; ++i) h[f->oW + i] = (float)(gauss(st) / std::sqrt((double)C));
        for (long long i = 0; i < 3LL * C; ++i) h[f->oQ + i] = (float)(gauss(st) / std::sqrt((double)C));
        FCU(cudaMemcpy(f->w, h.data(), 4 * n, cudaMemcpyHostToDevice));
        // mode matrices (FP64 -> BF16 / FP32)
        const double pi = 3.14159265358979323846;
        std::vector<__nv_bfloat16> fx((size_t)W * 2 * m), gx((size_t)2 * m * W), gxa((size_t)2 * m * W);
        for (int x = 0; x < W; ++x)
            for (int k = 0; k < m; ++k) {
                const double th = 2.0 * pi * k * x / W, a = (k == 0 ? 1.0 : 2.0) / ((double)H * W);
                fx[(size_t)x * 2 * m + k] = __float2bfloat16((float)std::cos(th));
                fx[(size_t)x * 2 * m + m + k] = __float2bfloat16((float)-std::sin(th));
                gx[(size_t)k * W + x] = __float2bfloat16((float)(a * std::cos(th)));
                gx[(size_t)(m + k) * W + x] = __float2bfloat16((float)(-a * std::sin(th)));
                gxa[(size_t)k * W + x] = __float2bfloat16((float)std::cos(th));
                gxa[(size_t)(m + k) * W + x] = __float2bfloat16((float)-std::sin(th));
            }
        std::vector<float> fyr((size_t)2 * m * H), fyi((size_t)2 * m * H), gyr((size_t)H * 2 * m), gyi((size_t)H * 2 * m);
        for (int iy = 0; iy < 2 * m; ++iy) {
            const int ky = iy < m ? iy : H - 2 * m + iy;
            for (int y = 0; y < H; ++y) {
                const double th = 2.0 * pi * ky * y / H;
                fyr[(size_t)iy * H + y] = (float)std::cos(th);
                fyi[(size_t)iy * H + y] = (float)-std::sin(th);
                gyr[(size_t)y * 2 * m + iy] = (float)std::cos(th);
                gyi[(size_t)y * 2 * m + iy] = (float)std::sin(th);
            }
        }
        FCU(cudaMalloc(&f->Fx, 2 * fx.size())); FCU(cudaMemcpy(f->Fx, fx.data(), 2 * fx.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gx, 2 * gx.size())); FCU(cudaMemcpy(f->Gx, gx.data(), 2 * gx.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gxa, 2 * gxa.size())); FCU(cudaMemcpy(f->Gxa, gxa.data(), 2 * gxa.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Fyre, 4 * fyr.size())); FCU(cudaMemcpy(f->Fyre, fyr.data(), 4 * fyr.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Fyim, 4 * fyi.size())); FCU(cudaMemcpy(f->Fyim, fyi.data(), 4 * fyi.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gyre, 4 * gyr.size())); FCU(cudaMemcpy(f->Gyre, gyr.data(), 4 * gyr.size(), cudaMemcpyHostToDevice));
        FCU(cudaMalloc(&f->Gyim, 4 * gyi.size())); FCU(cudaMemcpy(f->Gyim, gyi.data(), 4 * gyi.size(), cudaMemcpyHostToDevice));
        const long long act = (long long)max_batch * C * f->np;
        const long long modes_n = (long long)max_batch * C * 2 * m * m;
        f->vf.resize(L + 1); f->vb.resize(L + 1); f->u.resize(L); f->A1.resize(L); f->vhr.resize(L); f->vhi.resize(L);
        for (int l = 0; l <= L; ++l) {
            FCU(cudaMalloc(&f->vf[l], 4 * act));
            FCU(cudaMalloc(&f->vb[l], 2 * act));
        }
        for (int l = 0; l < L; ++l) {
            FCU(cudaMalloc(&f->u[l], 4 * act));
            FCU(cudaMalloc(&f->A1[l], 4LL * max_batch * C * H * 2 * m));
            FCU(cudaMalloc(&f->vhr[l], 4 * modes_n));
            FCU(cudaMalloc(&f->vhi[l], 4 * modes_n));
        }
        FCU(cudaMalloc(&f->whr, 4 * modes_n)); FCU(cudaMalloc(&f->whi, 4 * modes_n));
        FCU(cudaMalloc(&f->dwr, 4 * modes_n)); FCU(cudaMalloc(&f->dwi, 4 * modes_n));
        FCU(cudaMalloc(&f->Z, 4LL * max_batch * C * H * 2 * m));
        FCU(cudaMalloc(&f->zb, 2LL * max_batch * C * H * 2 * m));
        FCU(cudaMalloc(&f->acc, 4 * act)); FCU(cudaMalloc(&f->dv, 4 * act)); FCU(cudaMalloc(&f->du, 4 * act));
        FCU(cudaMalloc(&f->tmp, 4 * act)); FCU(cudaMalloc(&f->db16, 2 * act));
        FCU(cudaMalloc(&f->y, 4LL * max_batch * 3 * f->np)); FCU(cudaMalloc(&f->dy, 4LL * max_batch * 3 * f->np));
        FCU(cudaMalloc(&f->dloss, 8));
        FCU(cudaMalloc(&f->err, sizeof(int)));
        FCU(cudaMemset(f->err, 0, sizeof(int)));
        FCU(gemm_configure());
        return MM_OK;
    }();
    if (rc != MM_OK) {
        fno_free(f);
        delete f;
        return rc;
    }
    *out = f;
    return MM_OK;
}

extern "C" int mm_fno_destroy(mm_fno* f) {
    if (!f) return MM_OK;
    cudaStreamSynchronize(f->s);
    fno_free(f);
    delete f;
    return MM_OK;
}

extern "C" long long mm_fno_param_count(const mm_fno* f) { return f ? f->n_params : -1; }

extern "C" int mm_fno_set_params(mm_fno* f, const float* p) {
    if (!f || !p) return fno_fail(MM_EINVAL, "null argument");
    FCU(cudaMemcpyAsync(f->w, p, 4 * f->n_params, cudaMemcpyDefault, f->s));
    FCU(cudaMemsetAsync(f->m1, 0, 4 * f->n_params, f->s));
    FCU(cudaMemsetAsync(f->m2, 0, 4 * f->n_params, f->s));
    FCU(cudaStreamSynchronize(f->s));
    f->step = 0;
    return MM_OK;
}

extern "C" int mm_fno_get_params(mm_fno* f, float* p) {
    if (!f || !p) return fno_fail(MM_EINVAL, "null argument");
    FCU(cudaMemcpyAsync(p, f->w, 4 * f->n_params, cudaMemcpyDefault, f->s));
    FCU(cudaStreamSynchronize(f->s));
    return MM_OK;
}

// forward pass of B samples; x (B, 3, H, W) FP32 device; result in f->y
static int fno_forward(mm_fno* f, int B, const float* x) {
    const int C = f->C, m = f->m, L = f->L, H = f->H, W = f->W;
    const long long np = f->np, act = (long long)B * C * np;
    cudaStream_t s = f->s;
    k_to_bf16<<<grid1((long long)L * C * C), 256, 0, s>>>(f->w + f->oW, f->wb, (long long)L * C * C, 1.f);
    k_lift<<<grid1(B * np), 256, 0, s>>>(x, f->w + f->oP, f->w + f->op, C, H, W, B, f->vf[0]);
    k_to_bf16<<<grid1(act), 256, 0, s>>>(f->vf[0], f->vb[0], act, 1.f);
    const int nmode = 2 * m * m;
    for (int l = 0; l < L; ++l) {
        // x modes: A1[(b,c,y)][2m] = v[(b,c,y)][x] . Fx[x][2m]
        GemmArgs g{};
        g.A = f->vb[l]; g.B = f->Fx; g.C = f->A1[l];
        g.M = B * C * H; g.N = 2 * m; g.K = W;
        g.sam = W; g.sak = 1; g.sbk = 2 * m; g.sbn = 1; g.scm = 2 * m; g.scn = 1;
        g.alpha = 1.f; g.beta = 0.f;
        FCU(gemm(g, 1, f->err, s));
        // y modes
        k_ydft<<<grid1((long long)B * C * nmode), 256, 0, s>>>(f->A1[l], 2 * m, H, m, f->Fyre, f->Fyim, 2 * m, B * C,
                                                                f->vhr[l], f->vhi[l], 1.f, 0);
        // mode mix
        k_modemix<<<grid1((long long)B * C * nmode), 256, 0, s>>>(
            f->vhr[l], f->vhi[l], f->w + f->oRr + (long long)l * C * C * nmode, f->w + f->oRi + (long long)l * C * C * nmode,
            C, nmode, B, 0, f->whr, f->whi);
        // back along y: Z[(b,o,y)][2m]
        k_yidft<<<grid1((long long)B * C * H * m), 256, 0, s>>>(f->whr, f->whi, 2 * m, m, f->Gyre, f->Gyim, H, B * C,
                                                                 f->Z);
        k_to_bf16<<<grid1((long long)B * C * H * 2 * m), 256, 0, s>>>(f->Z, f->zb, (long long)B * C * H * 2 * m, 1.f);
        // u = S(v): acc[(b,o,y)][x] = Z . Gx
        GemmArgs g2{};
        g2.A = f->zb; g2.B = f->Gx; g2.C = f->u[l];
        g2.M = B * C * H; g2.N = W; g2.K = 2 * m;
        g2.sam = 2 * m; g2.sak = 1; g2.sbk = W; g2.sbn = 1; g2.scm = W; g2.scn = 1;
        g2.alpha = 1.f; g2.beta = 0.f;
        FCU(gemm(g2, 1, f->err, s));
        // u += W_l v (per sample: (C x C) . (C x np))
        GemmArgs g3{};
        g3.A = f->wb + (long long)l * C * C; g3.B = f->vb[l]; g3.C = f->u[l];
        g3.M = C; g3.N = (int)np; g3.K = C;
        g3.sam = C; g3.sak = 1; g3.sbk = np; g3.sbn = 1; g3.scm = np; g3.scn = 1;
        g3.zA = 0; g3.zB = (long long)C * np; g3.zC = (long long)C * np;
        g3.alpha = 1.f; g3.beta = 1.f;
        FCU(gemm(g3, B, f->err, s));
        // + b_l, activation
        k_add_bias<<<grid1(act), 256, 0, s>>>(f->u[l], f->w + f->ob + (long long)l * C, C, np, B);
        k_act<<<grid1(act), 256, 0, s>>>(f->u[l], f->vb[l + 1], f->vf[l + 1], act, l < L - 1 ? 1 : 0);
    }
    k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->vf[L], C, f->w + f->oQ, f->w + f->oq, 3, np, B, 0, f->y);
    FCU(cudaGetLastError());
    return MM_OK;
}

// backward pass for the batch whose forward pass is in f; t (B, 3, H, W)
// FP32 device; gradients into f->g, loss (FP64) into f->dloss.
static int fno_backward(mm_fno* f, int B, const float* x, const float* t) {
    const int C = f->C, m = f->m, L = f->L, H = f->H, W = f->W;
    const long long np = f->np, act = (long long)B * C * np, ny = (long long)B * 3 * np;
    const int nmode = 2 * m * m;
    cudaStream_t s = f->s;
    FCU(cudaMemsetAsync(f->g, 0, 4 * f->n_params, s));
    FCU(cudaMemsetAsync(f->dloss, 0, 8, s));
    k_loss<<<grid1(ny), 256, 0, s>>>(f->y, t, ny, f->dy, f->dloss);
    const int gx = 64;
    k_outer<<<dim3(gx, 3 * C), 256, 0, s>>>(f->dy, 3, f->vf[L], C, np, B, f->g + f->oQ);
    k_colsum<<<dim3(gx, 3), 256, 0, s>>>(f->dy, 3, np, B, f->g + f->oq);
    k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->dy, 3, f->w + f->oQ, nullptr, C, np, B, 1, f->dv);
    for (int l = L - 1; l >= 0; --l) {
        if (l < L - 1) k_act_back<<<grid1(act), 256, 0, s>>>(f->u[l], f->dv, act);
        // dv now holds du for layer l
        k_colsum<<<dim3(gx, C), 256, 0, s>>>(f->dv, C, np, B, f->g + f->ob + (long long)l * C);
        k_outer<<<dim3(gx, C * C), 256, 0, s>>>(f->dv, C, f->vf[l], C, np, B, f->g + f->oW + (long long)l * C * C);
        k_pointwise<<<grid1(B * np), 256, 0, s>>>(f->dv, C, f->w + f->oW + (long long)l * C * C, nullptr, C, np, B, 1,
                                                   f->tmp);
        // spectral path: dw = (a/(HW)) modes(du); dR += dw conj(vh); dvh = R^H dw
        k_to_bf16<<<grid1(act), 256, 0, s>>>(f->dv, f->db16, act, 1.f);
        GemmArgs g{};
        g.A = f->db16; g.B = f->Fx; g.C = f->Z;
        g.M = B * C * H; g.N = 2 * m; g.K = W;
        g.sam = W; g.sak = 1; g.sbk = 2 * m; g.sbn = 1; g.scm = 2 * m; g.scn = 1;
        g.alpha = 1.f; g.beta = 0.f;
        FCU(gemm(g, 1, f->err, s));
        k_ydft<<<grid1((long long)B * C * nmode), 256, 0, s>>>(f->Z, 2 * m, H, m, f->Fyre, f->Fyim, 2 * m, B * C,
                                                                f->dwr, f->dwi, 1.f / ((float)H * W), 1);
        const long long ro = (long long)l * C * C * nmode;
        k_dR<<<grid1((long long)C * C * nmode), 256, 0, s>>>(f->dwr, f->dwi, f->vhr[l], f->vhi[l], C, nmode, B,
                                                             f->g + f->oRr + ro, f->g + f->oRi + ro);
        k_modemix<<<grid1((long long)B * C * nmode), 256, 0, s>>>(f->dwr, f->dwi, f->w + f->oRr + ro, f->w + f->oRi + ro,
                                                                   C, nmode, B, 1, f->whr, f->whi);
        k_yidft<<<grid1((long long)B * C * H * m), 256, 0, s>>>(f->whr, f->whi, 2 * m, m, f->Gyre, f->Gyim, H, B * C,
                                                                 f->Z);
        k_to_bf16<<<grid1((long long)B * C * H * 2 * m), 256, 0, s>>>(f->Z, f->zb, (long long)B * C * H * 2 * m, 1.f);
        GemmArgs g2{};
        g2.A = f->zb; g2.B = f->Gxa; g2.C = f->tmp;
        g2.M = B * C * H; g2.N = W; g2.K = 2 * m;
        g2.sam = 2 * m; g2.sak = 1; g2.sbk = W; g2.sbn = 1; g2.scm = W; g2.scn = 1;
        g2.alpha = 1.f; g2.beta = 1.f;
        FCU(gemm(g2, 1, f->err, s));
        float* t2 = f->dv;
        f->dv = f->tmp;
        f->tmp = t2;
    }
    k_outer_lift<<<dim3(gx, C * 5), 256, 0, s>>>(f->dv, C, x, H, W, B, f->g + f->oP);
    k_colsum<<<dim3(gx, C), 256, 0, s>>>(f->dv, C, np, B, f->g + f->op);
    FCU(cudaGetLastError());
    return MM_OK;
}

// A tensor-core GEMM whose wait expired left its output incomplete; read
// after the stream has been synchronised.
static int fno_check_tc(const mm_fno* f) {
    int e = 0;
    FCU(cudaMemcpyAsync(&e, f->err, sizeof(int), cudaMemcpyDeviceToHost, f->s));
    FCU(cudaStreamSynchronize(f->s));
    if (e) return fno_fail(MM_ETIMEOUT, "a tensor-core GEMM wait timed out; the result is incomplete");
    return MM_OK;
}

static int fno_check_batch(const mm_fno* f, int B, const void* x, const void* y) {
    if (!f || !x || !y) return fno_fail(MM_EINVAL, "null argument");
    if (B < 1 || B > f->Bmax) return fno_fail(MM_EINVAL, "batch out of range");
    return MM_OK;
}

extern "C" int mm_fno_forward(mm_fno* f, int B, const float* x, float* y) {
    int rc = fno_check_batch(f, B, x, y);
    if (rc != MM_OK) return rc;
    rc = fno_forward(f, B, x);
    if (rc != MM_OK) return rc;
    FCU(cudaMemcpyAsync(y, f->y, 4LL * B * 3 * f->np, cudaMemcpyDeviceToDevice, f->s));
    return MM_OK;
}

extern "C" int mm_fno_grad(mm_fno* f, int B, const float* x, const float* t, double* loss, float* grad) {
    int rc = fno_check_batch(f, B, x, t);
    if (rc != MM_OK) return rc;
    rc = fno_forward(f, B, x);
    if (rc == MM_OK) rc = fno_backward(f, B, x, t);
    if (rc != MM_OK) return rc;
    if (grad) FCU(cudaMemcpyAsync(grad, f->g, 4 * f->n_params, cudaMemcpyDefault, f->s));
    double l = 0.0;
    FCU(cudaMemcpyAsync(&l, f->dloss, 8, cudaMemcpyDeviceToHost, f->s));
    FCU(cudaStreamSynchronize(f->s));
    rc = fno_check_tc(f);
    if (rc != MM_OK) return rc;
    if (loss) *loss = l / (3.0 * B * f->np);
    return MM_OK;
}

extern "C" int mm_fno_train_step(mm_fno* f, int B, const float* x, const float* t, float lr, double* loss) {
    int rc = fno_check_batch(f, B, x, t);
    if (rc != MM_OK) return rc;
    rc = fno_forward(f, B, x);
    if (rc == MM_OK) rc = fno_backward(f, B, x, t);
    if (rc != MM_OK) return rc;
    f->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, f->step), c2 = 1.f - (float)std::pow((double)b2, f->step);
    k_adam<<<grid1(f->n_params), 256, 0, f->s>>>(f->w, f->g, f->m1, f->m2, f->n_params, lr, b1, b2, c1, c2, 1e-8f);
    FCU(cudaGetLastError());
    if (loss) {
        double l = 0.0;
        FCU(cudaMemcpyAsync(&l, f->dloss, 8, cudaMemcpyDeviceToHost, f->s));
        FCU(cudaStreamSynchronize(f->s));
        rc = fno_check_tc(f);
        if (rc != MM_OK) return rc;
        *loss = l / (3.0 * B * f->np);
    }
    return MM_OK;
}

// error word of mm_gemm_bf16 (one per device image of the library)
static __device__ int g_gemm_err;

extern "C" int mm_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, long long sam,
                            long long sak, long long sbk, long long sbn, long long scm, long long scn, int batch,
                            long long zA, long long zB, long long zC, float alpha, float beta, int atomic,
                            void* cuda_stream) {
    if (!C || (K > 0 && (!A || !B))) return fno_fail(MM_EINVAL, "null argument");
    if (M < 1 || N < 1 || K < 0 || batch < 1 || batch > 65535 || M > 65535LL * kTcM || N > 65535LL * kTcM)
        return fno_fail(MM_EINVAL, "need M, N in 1..65535*128, K >= 0, batch in 1..65535");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* errp = nullptr;
    FCU(cudaGetSymbolAddress(&errp, g_gemm_err));
    FCU(gemm_configure());
    FCU(cudaMemsetAsync(errp, 0, sizeof(int), s));
    GemmArgs g{};
    g.A = (const __nv_bfloat16*)A; g.B = (const __nv_bfloat16*)B; g.C = C;
    g.M = M; g.N = N; g.K = K;
    g.sam = sam; g.sak = sak; g.sbk = sbk; g.sbn = sbn; g.scm = scm; g.scn = scn;
    g.zA = zA; g.zB = zB; g.zC = zC;
    g.alpha = alpha; g.beta = beta; g.atomic = atomic ? 1 : 0;
    FCU(gemm(g, batch, (int*)errp, s));
    int e = 0;
    FCU(cudaMemcpyAsync(&e, errp, sizeof(int), cudaMemcpyDeviceToHost, s));
    FCU(cudaStreamSynchronize(s));
    if (e) return fno_fail(MM_ETIMEOUT, "a tensor-core GEMM wait timed out; C is incomplete");
    return MM_OK;
}

namespace mmk {
// Forward of one sample for the surrogate stepper (x, y: 3 * H * W FP32 on
// the device), on stream s.
int fno_apply(mm_fno* f, const float* x, float* y, cudaStream_t s) {
    cudaStream_t keep = f->s;
    f->s = s;
    int rc = fno_forward(f, 1, x);
    if (rc == MM_OK && cudaMemcpyAsync(y, f->y, 4LL * 3 * f->np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = fno_fail(MM_ECUDA, "copy of the surrogate output failed");
    f->s = keep;
    return rc;
}
bool fno_matches(const mm_fno* f, int nx, int ny, int nz) { return f && nz == 1 && f->W == nx && f->H == ny; }
}  // namespace mmk
