// mm_api.cu -- the C ABI of include/mm.h: argument checks, the plan, device
// buffers, CUDA-graph replay of the step and the error channel.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "bulk_copy.cuh"
#include "ctx_internal.h"

using namespace mmk;

static thread_local char g_err[512];

namespace mmk {
int set_error_fmt(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}
}  // namespace mmk

#define fail mmk::set_error_fmt


// ------------------------------------------------------------------ plan --
static bool smooth235(int n) {
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Padded length of an axis with n cells: any L >= 2n-1 gives the exact
// linear convolution; take 2n when n is a power of two (the paper's choice),
// otherwise the smallest 2^a 3^b 5^c >= 2n-1; n = 1 needs no padding.
static int padded_length(int n) {
    if (n == 1) return 1;
    if ((n & (n - 1)) == 0) return 2 * n;
    int L = 2 * n - 1;
    while (!smooth235(L)) ++L;
    return L;
}

static bool make_axis_plan(int L, AxisPlan* p) {
    memset(p, 0, sizeof(*p));
    p->L = L;
    int n = L, a = 0;
    while (n % 2 == 0) { n /= 2; ++a; }
    int st = (a + 3) / 4;               // stages for the power-of-two part
    for (int s = 0; s < st; ++s) {      // spread the bits evenly, <= 4 each
        const int bits = a / st + (s < a % st ? 1 : 0);
        p->rad[p->nst++] = 1 << bits;
    }
    while (n % 5 == 0) { n /= 5; p->rad[p->nst++] = 5; }
    while (n % 3 == 0) { n /= 3; p->rad[p->nst++] = 3; }
    return n == 1 && p->nst <= kMaxStages;
}

static int build_plan(mm_ctx* c) {
    Geom& g = c->g;
    Launch& l = c->l;
    g.nx = c->grid[0];
    g.ny = c->grid[1];
    g.nz = c->grid[2];
    g.N = g.nx * g.ny * g.nz;
    g.Lx = padded_length(g.nx);
    g.Ly = padded_length(g.ny);
    g.Lz = padded_length(g.nz);
    if (g.Lx > kMaxLen || g.Ly > kMaxLen || g.Lz > kMaxLen)
        return fail(MM_EUNSUPPORTED, "padded length exceeds %d", kMaxLen);
    g.Hx = g.Lx / 2 + 1;
    g.Hy = g.Ly / 2 + 1;
    g.Hz = g.Lz / 2 + 1;
    g.Jst = g.ny;
    if (!make_axis_plan(g.Lx, &g.px) || !make_axis_plan(g.Ly, &g.py) || !make_axis_plan(g.Lz, &g.pz))
        return fail(MM_EUNSUPPORTED, "no radix plan for padded lengths %d %d %d", g.Lx, g.Ly, g.Lz);

    // Each pass holds its lines plus a Stockham ping-pong scratch in shared
    // memory (fft_lines); `g*` is the number of lines per scratch group.
    const size_t smem_cap = 227 * 1024;
    const size_t lx_bytes = (size_t)padded_len(g.Lx) * sizeof(float2);
    const size_t ly_bytes = (size_t)padded_len(g.Ly) * sizeof(float2);
    // pass 1: R1/2 complex lines of Lx (+ as many scratch lines), <= ~64 KB
    int lines1 = (int)(32768 / lx_bytes);
    lines1 = lines1 < 1 ? 1 : (lines1 > 4 ? 4 : lines1);
    l.r1 = 2 * lines1;
    if (l.r1 > g.ny + (g.ny & 1)) l.r1 = g.ny + (g.ny & 1);
    l.t1 = 256;
    l.g1 = l.r1 / 2;
    l.smem1 = (size_t)2 * (l.r1 / 2) * lx_bytes;
    // pass 3: 3 * R3/2 lines of Lx (+ scratch)
    int pairs3 = (int)(32768 / (3 * lx_bytes));
    pairs3 = pairs3 < 1 ? 1 : (pairs3 > 2 ? 2 : pairs3);
    // small samples: one row pair per tile when two pairs would leave fewer
    // tiles than two per SM of a 152-SM GPU (the tile is a latency chain)
    if (pairs3 == 2 && (long long)g.nz * ((g.ny + 3) / 4) < 2 * 152) pairs3 = 1;
    l.r3 = 2 * pairs3;
    if (l.r3 > g.ny + (g.ny & 1)) l.r3 = g.ny + (g.ny & 1);
    l.t3 = 256;
    l.g3 = 3 * l.r3 / 2;
    l.smem3 = (size_t)2 * l.g3 * lx_bytes;
    // pass 2: one kx plane of 3*nz lines of Ly in shared memory (+ scratch
    // for g2 of them), or, for thick samples, the split y / z / y kernels
    // with the spectrum row stride widened to Ly.
    const int nl2 = 3 * g.nz;
    l.t2 = (nl2 * g.Ly >= 4096) ? 512 : 256;
    const size_t plane_bytes = (size_t)nl2 * ly_bytes;
    l.split = g.nz > kMaxPlaneNz || !plane_supported_lz(g.Lz) || plane_bytes + 2 * ly_bytes > 200 * 1024;
    if (l.split) {
        g.Jst = g.Ly;
        l.g2 = 0;
        l.smem2 = 0;
        if (split_smem_y(g) > smem_cap || split_smem_z(g) > smem_cap)
            return fail(MM_EUNSUPPORTED, "padded lengths %d, %d too long for the split pass", g.Ly, g.Lz);
    } else {
        size_t fit = (smem_cap - plane_bytes) / ly_bytes;
        l.g2 = (int)(fit < (size_t)nl2 ? fit : (size_t)nl2);
        l.smem2 = plane_bytes + (size_t)l.g2 * ly_bytes;
    }
    if (l.smem1 > smem_cap || l.smem3 > smem_cap)
        return fail(MM_EUNSUPPORTED, "x lines of %zu bytes exceed shared memory", lx_bytes);

    // Power-of-two grids use the compile-time kernels (same spectrum layout).
    const char* nofast = getenv("MM_NO_FAST");
    const bool allow_fast = !(nofast && nofast[0] == '1');
    l.fx = nullptr;
    l.fp = nullptr;
    l.fs2 = nullptr;
    if (allow_fast) {
        FastFns& f = c->fast;
        if (fast_lookup_x(g.nx, &f) && g.ny % f.r1 == 0 && g.ny % f.r3 == 0 && f.s1 <= smem_cap &&
            f.s3 <= smem_cap)
            l.fx = &f;
        bool pl = false;
        switch (g.nz) {
            case 1: pl = fast_lookup_plane_nz1(g.ny, &f); break;
            case 2: pl = fast_lookup_plane_nz2(g.ny, &f); break;
            case 4: pl = fast_lookup_plane_nz4(g.ny, &f); break;
            case 8: pl = fast_lookup_plane_nz8(g.ny, &f); break;
            default: break;
        }
        if (pl && f.s2 <= smem_cap && !l.split) l.fp = &f;
        if (l.split && fast_split_lookup(g.ny, g.nz, &c->fsplit) && c->fsplit.sy <= smem_cap &&
            c->fsplit.sz <= smem_cap)
            l.fs2 = &c->fsplit;
        FastStepFns& s = c->fs;
        bool ok = fast_step_lookup_x(g.nx, &s);
        ok = ok && (fast_step_lookup_plane_a(g.ny, g.nz, &s) || fast_step_lookup_plane_b(g.ny, g.nz, &s));
        ok = ok && l.fx && !l.split && g.ny % s.rb == 0 && s.sa <= smem_cap && s.sb <= smem_cap;
        // the x-step kernel indexes the spectrum and M with 32-bit offsets
        ok = ok && 3.0 * g.Hx * g.nz * g.Jst < (double)INT_MAX && 3.0 * g.N < (double)INT_MAX;
        c->has_fs = ok;
        // thick samples: the compile-time split pass with the x-step kernel
        // (same 32-bit offset limits)
        c->has_ss = !ok && l.split && l.fs2 && s.kb[kModeStep] && g.ny % s.rb == 0 && s.sb <= smem_cap &&
                    3.0 * g.Hx * g.nz * g.Jst < (double)INT_MAX && 3.0 * g.N < (double)INT_MAX;
        if (c->has_ss) s.ka = nullptr;
        c->has_persist = ok && persist_lookup(g.nx, g.ny, g.nz, s.rb, &c->pf);
    }
    if (!c->has_fs && !c->has_ss && !l.fx) {
        c->has_gx = true;
    }
    return MM_OK;
}

// Planning helpers shared with the batched driver (batch.cu).
namespace mmk {
int plan_padded_length(int n) { return padded_length(n); }
bool plan_axis(int L, AxisPlan* p) { return make_axis_plan(L, p); }
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace mmk

static void host_twiddles(int L, float2* out) {
    for (int m = 0; m < L; ++m) {
        const double a = -2.0 * 3.14159265358979323846 * (double)m / (double)L;
        out[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
}

namespace mmk {
void plan_twiddles(int L, float2* out) { host_twiddles(L, out); }
}  // namespace mmk

LlgCoef mmk::make_coef(const mm_ctx* c, double dt) {
    LlgCoef f;
    const double Ms2 = c->Ms * c->Ms;
    const double den = 1.0 + c->alpha * c->alpha;
    f.Ms = (float)c->Ms;
    f.pexch = (float)(2.0 * c->A / (kMu0 * Ms2));
    f.panis = (float)(-2.0 * c->Ku / (kMu0 * Ms2));
    f.c1 = (float)(-c->gamma / den);
    f.c2 = (float)(-c->alpha * c->gamma / (den * c->Ms));
    f.idx2 = (float)(1.0 / (c->cell[0] * c->cell[0]));
    f.idy2 = (float)(1.0 / (c->cell[1] * c->cell[1]));
    f.idz2 = (float)(1.0 / (c->cell[2] * c->cell[2]));
    f.hx = (float)c->Hext[0];
    f.hy = (float)c->Hext[1];
    f.hz = (float)c->Hext[2];
    f.dt = (float)dt;
    return f;
}

static void release(mm_ctx* c) {
    for (int kd = 0; kd < 2; ++kd)
        for (int p = 0; p < 2; ++p)
            if (c->step_exec[kd][p]) cudaGraphExecDestroy(c->step_exec[kd][p]);
    cudaFree(c->Kt);
    cudaFree(c->Kd);
    cudaFree(c->Kd0);
    cudaFree(c->Kt_ex);
    cudaFree(c->S);
    cudaFree(c->Sh);
    for (int q = 0; q < 7; ++q) cudaFree(c->dpk[q]);
    cudaFree(c->dperr);
    cudaFree(c->Mbuf[0]);
    cudaFree(c->Mbuf[1]);
    cudaFree(c->H);
    cudaFree(c->Mst);
    cudaFree(c->acc);
    cudaFree(c->sur);
    cudaFree(c->sur_r);
    cudaFree(c->flag);
    cudaFree(c->partials);
    cudaFree(c->Edev);
    cudaFree(c->tw);
    cudaFree(c->gbar);
    if (c->cap) cudaStreamDestroy(c->cap);
}

// ------------------------------------------------------------------ API --
extern "C" int mm_create(mm_ctx** out, const int grid[3], const double cell[3], double Ms, double A, double Ku,
                         double alpha, double gamma, void* cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(MM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !cell) return fail(MM_EINVAL, "grid or cell is NULL");
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < 1) return fail(MM_EINVAL, "grid[%d] = %d < 1", a, grid[a]);
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a])) return fail(MM_EINVAL, "cell[%d] must be > 0", a);
    }
    if (!(Ms > 0.0) || !std::isfinite(Ms)) return fail(MM_EINVAL, "Ms must be > 0");
    if (!(A >= 0.0) || !std::isfinite(A)) return fail(MM_EINVAL, "A must be >= 0");
    if (!std::isfinite(Ku)) return fail(MM_EINVAL, "Ku must be finite");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(MM_EINVAL, "alpha must be >= 0");
    if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(MM_EINVAL, "gamma must be > 0");
    if ((long long)grid[0] * grid[1] * grid[2] > (1LL << 28)) return fail(MM_EUNSUPPORTED, "grid too large");

    mm_ctx* c = new (std::nothrow) mm_ctx();
    if (!c) return fail(MM_ENOMEM, "host allocation failed");
    for (int a = 0; a < 3; ++a) {
        c->grid[a] = grid[a];
        c->cell[a] = cell[a];
        c->Hext[a] = 0.0;
    }
    c->Ms = Ms;
    c->A = A;
    c->Ku = Ku;
    c->alpha = alpha;
    c->gamma = gamma;
    c->stream = (cudaStream_t)cuda_stream;
    c->use_graphs = !(getenv("MM_NO_GRAPHS") && getenv("MM_NO_GRAPHS")[0] == '1');
    int rc = build_plan(c);
    if (rc != MM_OK) {
        delete c;
        return rc;
    }
    rc = [&]() -> int {
        CU(cudaGetDevice(&c->device));
        CU(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        Geom& g = c->g;
        const size_t N = (size_t)g.N;
        CU(cudaMalloc(&c->Kt, sizeof(float) * 6 * (size_t)g.Hx * g.Hy * g.Hz));
        // the two-kernel step's spectra carry one pad kx plane (the tiled
        // copies of the x-step touch it; nothing reads it)
        const size_t plane = (size_t)3 * g.nz * g.Jst;
        const size_t nS = (size_t)(g.Hx + (c->has_fs ? 1 : 0)) * plane;
        CU(cudaMalloc(&c->S, sizeof(float2) * nS));
        if (c->has_fs) {
            CU(cudaMalloc(&c->Sh, sizeof(float2) * nS));
            CU(cudaMemset(c->S + (size_t)g.Hx * plane, 0, sizeof(float2) * plane));
            CU(cudaMemset(c->Sh + (size_t)g.Hx * plane, 0, sizeof(float2) * plane));
            CU(cudaMalloc(&c->Kd, sizeof(float) * 6 * (size_t)g.Hx * kd_row(g.Hy) * g.nz));
            CU(cudaMalloc(&c->Kd0, sizeof(float) * 6 * (size_t)g.Hx * kd_row(g.Hy) * g.nz));
        }
        if (c->has_ss) CU(cudaMalloc(&c->Kt_ex, sizeof(float) * 6 * (size_t)g.Hx * g.Hy * g.Hz));
        CU(cudaMalloc(&c->Mbuf[0], sizeof(float) * 3 * N));
        CU(cudaMalloc(&c->Mbuf[1], sizeof(float) * 3 * N));
        CU(cudaMalloc(&c->H, sizeof(float) * 3 * N));
        CU(cudaMalloc(&c->flag, sizeof(int)));
        CU(cudaMalloc(&c->partials, sizeof(double) * energy_partials_elems(g.N)));
        CU(cudaMalloc(&c->Edev, sizeof(double) * 5));
        CU(cudaMalloc(&c->tw, sizeof(float2) * (size_t)(g.Lx + g.Ly + g.Lz)));
        {
            float2* h = (float2*)malloc(sizeof(float2) * (size_t)(g.Lx + g.Ly + g.Lz));
            if (!h) return fail(MM_ENOMEM, "host allocation failed");
            host_twiddles(g.Lx, h);
            host_twiddles(g.Ly, h + g.Lx);
            host_twiddles(g.Lz, h + g.Lx + g.Ly);
            cudaError_t e = cudaMemcpy(c->tw, h, sizeof(float2) * (size_t)(g.Lx + g.Ly + g.Lz),
                                       cudaMemcpyHostToDevice);
            free(h);
            CU(e);
        }
        g.twx = c->tw;
        g.twy = c->tw + g.Lx;
        g.twz = c->tw + g.Lx + g.Ly;
        g.Kt = c->Kt;
        g.Kd = c->Kd;
        g.Kd0 = c->Kd0;
        CU(configure_pass_kernels(g, c->l));
        if (c->has_fs || c->has_ss) CU(configure_step_kernels(c->fs));
        if (c->has_fs) {
            int sms = 0;
            CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
            c->fs.early = fast_step_early_trigger(g, sms);
            encode_xstep_maps(g, &c->fs, c->Sh, c->S);   // per-thread copies where no map applies
        }
        if (c->has_persist) {
            bool usable = false;
            CU(persist_configure(g, c->fs.rb, &c->pf, &usable));
            c->has_persist = usable;
            if (usable) CU(persist_alloc_bar(&c->gbar));
        }

        // tensor set-up in FP64
        const int L[3] = {g.Lx, g.Ly, g.Lz};
        double *Nd = nullptr, *w1 = nullptr, *w2 = nullptr;
        const size_t wn = tensor_work_elems(c->grid, L);
        cudaError_t e = cudaMalloc(&Nd, sizeof(double) * 6 * N);
        if (e == cudaSuccess) e = cudaMalloc(&w1, sizeof(double) * wn);
        if (e == cudaSuccess) e = cudaMalloc(&w2, sizeof(double) * wn);
        if (e == cudaSuccess) e = tensor_octant_fp64(c->grid, c->cell, Nd, c->stream);
        ExchangeFold exf{};
        exf.on = c->has_fs ? 1 : 0;
        exf.nx = g.nx;
        exf.ny = g.ny;
        exf.Lx = g.Lx;
        exf.Ly = g.Ly;
        exf.pexch = 2.0 * c->A / (kMu0 * c->Ms * c->Ms);
        exf.idx2 = 1.0 / (c->cell[0] * c->cell[0]);
        exf.idy2 = 1.0 / (c->cell[1] * c->cell[1]);
        exf.idz2 = 1.0 / (c->cell[2] * c->cell[2]);
        if (e == cudaSuccess) e = tensor_spectrum(c->grid, L, Nd, c->Kt, w1, w2, c->stream, c->Kd, exf, c->Kd0);
        if (e == cudaSuccess && c->has_ss) {
            ExchangeFold ex3 = exf;
            ex3.on = 1;
            e = tensor_fold_exchange3(c->g, ex3, c->Kt, c->Kt_ex, c->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(Nd);
        cudaFree(w1);
        cudaFree(w2);
        CU(e);

        // initial state: uniform +x
        float* h = (float*)malloc(sizeof(float) * 3 * N);
        if (!h) return fail(MM_ENOMEM, "host allocation failed");
        for (size_t i = 0; i < N; ++i) {
            h[i] = (float)Ms;
            h[N + i] = 0.f;
            h[2 * N + i] = 0.f;
        }
        e = cudaMemcpy(c->Mbuf[0], h, sizeof(float) * 3 * N, cudaMemcpyHostToDevice);
        free(h);
        CU(e);
        CU(cudaMemset(c->flag, 0, sizeof(int)));
        CU(cudaDeviceSynchronize());
        return MM_OK;
    }();
    if (rc != MM_OK) {
        release(c);
        delete c;
        return rc;
    }
    *out = c;
    return MM_OK;
}

extern "C" int mm_destroy(mm_ctx* c) {
    if (!c) return MM_OK;
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
    return MM_OK;
}

extern "C" int mm_set_integrator(mm_ctx* c, int method) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (method != MM_INTEGRATOR_EULER && method != MM_INTEGRATOR_HEUN && method != MM_INTEGRATOR_RK4)
        return fail(MM_EINVAL, "unknown integrator %d", method);
    if (method != MM_INTEGRATOR_EULER && !c->Mst) {
        const size_t n = 3 * (size_t)c->g.N;
        CU(cudaMalloc(&c->Mst, sizeof(float) * n));
        CU(cudaMalloc(&c->acc, sizeof(float) * n));
    }
    if (method != c->method) {
        c->method = method;
        c->ver++;                               // re-capture the step graphs
        c->spec_valid = false;
    }
    return MM_OK;
}

extern "C" int mm_set_field(mm_ctx* c, const double H_ext[3]) {
    if (!c || !H_ext) return fail(MM_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(H_ext[a])) return fail(MM_EINVAL, "H_ext must be finite");
    for (int a = 0; a < 3; ++a) c->Hext[a] = H_ext[a];
    c->ver++;
    return MM_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int mm_set_m(mm_ctx* c, const float* M) {
    if (!c || !M) return fail(MM_EINVAL, "null argument");
    CU(cudaMemcpyAsync(c->Mbuf[c->cur], M, sizeof(float) * 3 * (size_t)c->g.N, cudaMemcpyDefault, c->stream));
    CU(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    c->spec_valid = false;
    if (!is_device_ptr(M)) CU(cudaStreamSynchronize(c->stream));
    return MM_OK;
}

extern "C" int mm_get_m(mm_ctx* c, float* M) {
    if (!c || !M) return fail(MM_EINVAL, "null argument");
    CU(cudaMemcpyAsync(M, c->Mbuf[c->cur], sizeof(float) * 3 * (size_t)c->g.N, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(M)) CU(cudaStreamSynchronize(c->stream));
    return MM_OK;
}

// The three-pass evaluation on the spectrum workspace S (which also holds
// the two-kernel step's spectrum, so it invalidates a pending one).
int mmk::run_passes(mm_ctx* c, int mode, const float* M, float* out, double dt, cudaStream_t s) {
    const LlgCoef cf = make_coef(c, dt);
    c->spec_valid = false;
    CU(launch_pass1(c->g, c->l, M, c->S, s));
    if (c->has_fs && c->fs.ta <= 512 && (mode == kModeDemag || mode == kModeHeff)) {
        // power-of-two films: the step's plane kernel and the field-only
        // variant of its x-step kernel (where the plane kernel runs at most
        // 512 threads: larger ones are register-starved, and the three-pass
        // plane kernel serves them better)
        CU(launch_field_pdl(c->g, c->fs, cf, mode, mode == kModeDemag ? c->Kd0 : c->Kd, c->S, c->Sh, M, out, c->flag,
                            s));
        return MM_OK;
    }
    if (c->has_ss && (mode == kModeDemag || mode == kModeHeff)) {
        CU(launch_split_xstep(c->g, c->fsplit, c->fs, cf, mode, mode == kModeDemag ? c->Kt : c->Kt_ex, c->S, M,
                              out, nullptr, s));
        return MM_OK;
    }
    CU(launch_plane(c->g, c->l, c->S, s));
    CU(launch_pass3(c->g, c->l, cf, mode, c->S, M, out, c->flag, s));
    return MM_OK;
}

static bool overlap(const float* a, const float* b, size_t n) { return a < b + n && b < a + n; }

extern "C" int mm_demag_field(mm_ctx* c, const float* M, float* H) {
    if (!c || !M || !H) return fail(MM_EINVAL, "null argument");
    if (overlap(M, H, 3 * (size_t)c->g.N)) return fail(MM_EINVAL, "M and H overlap");
    return run_passes(c, kModeDemag, M, H, 0.0, c->stream);
}

extern "C" int mm_effective_field(mm_ctx* c, const float* M, float* H) {
    if (!c || !M || !H) return fail(MM_EINVAL, "null argument");
    if (overlap(M, H, 3 * (size_t)c->g.N)) return fail(MM_EINVAL, "M and H overlap");
    return run_passes(c, kModeHeff, M, H, 0.0, c->stream);
}

// One step from parity p (M[p] -> M[1-p]).  Two-kernel path: K_A from S
// into Sh, K_B from Sh into S (the spectrum of M[1-p]), programmatic
// dependent launch between them.  Generic path: the three passes on S.
// One explicit Runge-Kutta step (Heun or classic RK4) from parity p: per
// stage a field evaluation into H, then the stage update.
static int enqueue_rk_step(mm_ctx* c, int p, double dt, cudaStream_t s) {
    static const float heun_a[2] = {1.f, 0.f}, heun_b[2] = {0.5f, 0.5f};
    static const float rk4_a[4] = {0.5f, 0.5f, 1.f, 0.f};
    static const float rk4_b[4] = {1.f / 6.f, 1.f / 3.f, 1.f / 3.f, 1.f / 6.f};
    const int ns = c->method == MM_INTEGRATOR_HEUN ? 2 : 4;
    const float* av = ns == 2 ? heun_a : rk4_a;
    const float* bv = ns == 2 ? heun_b : rk4_b;
    const LlgCoef cf = make_coef(c, dt);
    for (int st = 0; st < ns; ++st) {
        const float* Min = st == 0 ? c->Mbuf[p] : c->Mst;
        int rc = run_passes(c, kModeHeff, Min, c->H, dt, s);
        if (rc != MM_OK) return rc;
        const int kind = st == 0 ? 0 : (st == ns - 1 ? 2 : 1);
        float* out = kind == 2 ? c->Mbuf[1 - p] : c->Mst;
        CU(launch_rk_stage(c->g.N, cf, av[st], bv[st], kind, Min, c->H, c->Mbuf[p], c->acc, out, c->flag, s));
    }
    return MM_OK;
}

static int enqueue_step(mm_ctx* c, int p, double dt, cudaStream_t s) {
    if (c->method != MM_INTEGRATOR_EULER) return enqueue_rk_step(c, p, dt, s);
    if (c->has_fs) {
        CU(launch_step_pdl(c->g, c->fs, make_coef(c, dt), c->S, c->Sh, c->Mbuf[p], c->Mbuf[1 - p],
                           c->flag, s, true));
        return MM_OK;
    }
    if (c->has_ss) {
        CU(launch_split_xstep(c->g, c->fsplit, c->fs, make_coef(c, dt), kModeStep, c->Kt_ex, c->S, c->Mbuf[p],
                              c->Mbuf[1 - p], c->flag, s));
        return MM_OK;
    }
    if (c->has_gx) {
        // S holds the x spectrum of M[p]: plane pass, then the update that
        // also forms the x spectrum of M[1-p]
        CU(launch_plane(c->g, c->l, c->S, s));
        CU(launch_pass3(c->g, c->l, make_coef(c, dt), kModeStepX, c->S, c->Mbuf[p], c->Mbuf[1 - p], c->flag, s));
        return MM_OK;
    }
    return run_passes(c, kModeStep, c->Mbuf[p], c->Mbuf[1 - p], dt, s);
}

// Steps per multi-step graph (even, so that it ends on the parity it starts
// from).  Inside one graph consecutive steps keep their programmatic
// launch edges, so a step's first kernel starts while the previous one drains.
constexpr int kGraphSteps = 16;

// Capture one step (kind 0) or kGraphSteps steps (kind 1) from parity p on
// the private stream into a graph.
static int capture_step(mm_ctx* c, int kind, int p, double dt) {
    cudaGraphExec_t& ex = c->step_exec[kind][p];
    if (ex) {
        cudaGraphExecDestroy(ex);
        ex = nullptr;
    }
    CU(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int rc = MM_OK;
    const int ns = kind ? kGraphSteps : 1;
    for (int s = 0; s < ns && rc == MM_OK; ++s) rc = enqueue_step(c, (p + s) & 1, dt, c->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
    if (rc != MM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CU(e);
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    CU(e);
    c->step_dt[kind][p] = dt;
    c->step_ver[kind][p] = c->ver;
    return MM_OK;
}

// Form S[cur] from M[cur] when the two-kernel step needs it.
static int ensure_spectrum(mm_ctx* c) {
    if (!(c->has_fs || c->has_ss || c->has_gx) || c->spec_valid || c->method != MM_INTEGRATOR_EULER) return MM_OK;
    CU(launch_pass1(c->g, c->l, c->Mbuf[c->cur], c->S, c->stream));
    c->spec_valid = true;
    return MM_OK;
}

// Steps per launch of the persistent step.
constexpr int kPersistChunk = 1024;

// mm_step takes the persistent kernel for Euler steps only when asked to
// (MM_STEP_PERSISTENT): on GB300 the two-kernel graph step is faster (the
// persistent kernel's 384-thread blocks, two per SM, cap both phases at 80
// registers, which the x-step phase exceeds).
static bool uses_persist(const mm_ctx* c) {
    return c->has_persist && c->method == MM_INTEGRATOR_EULER && c->step_path == MM_STEP_PERSISTENT;
}

extern "C" int mm_set_step_path(mm_ctx* c, int path) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (path != MM_STEP_AUTO && path != MM_STEP_GRAPH && path != MM_STEP_PERSISTENT)
        return fail(MM_EINVAL, "unknown step path %d", path);
    if (path == MM_STEP_PERSISTENT && !c->has_persist)
        return fail(MM_EUNSUPPORTED, "no persistent step for this grid and device");
    c->step_path = path;
    return MM_OK;
}

extern "C" int mm_get_step_path(const mm_ctx* c) {
    if (!c) return fail(MM_EINVAL, "null context");
    return uses_persist(c) ? MM_STEP_PERSISTENT : MM_STEP_GRAPH;
}

extern "C" int mm_set_tiled_copies(mm_ctx* c, int mask) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (mask & ~(MM_TILED_GATHER | MM_TILED_SCATTER)) return fail(MM_EINVAL, "unknown tiled-copy bits %d", mask);
    if (mask && !(c->has_fs && c->fs.tma))
        return fail(MM_EUNSUPPORTED, "no tiled x-step copies for this grid");
    if (c->fs.tma_use != mask) {
        c->fs.tma_use = mask;
        c->ver++;                               // re-capture the step graphs
    }
    return MM_OK;
}

extern "C" int mm_get_tiled_copies(const mm_ctx* c) {
    if (!c) return fail(MM_EINVAL, "null context");
    return c->has_fs && c->fs.tma ? c->fs.tma_use : 0;
}

extern "C" int mm_set_wait_limit(mm_ctx* c, long long polls) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (polls < 0) return fail(MM_EINVAL, "polls must be >= 0");
    c->wait_limit = polls;
    return MM_OK;
}

extern "C" int mm_step(mm_ctx* c, int n, double dt) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (n < 0) return fail(MM_EINVAL, "n must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MM_EINVAL, "dt must be > 0");
    if (n == 0) return MM_OK;
    int rc = ensure_spectrum(c);
    if (rc != MM_OK) return rc;
    if (uses_persist(c)) {
        // n steps per launch (in chunks, so that one launch stays short)
        const LlgCoef cf = make_coef(c, dt);
        for (int s = 0; s < n;) {
            const int m = std::min(n - s, kPersistChunk);
            const int p = c->cur, q = (p + m) & 1;
            CU(launch_persist(c->g, c->pf, cf, c->Kd, c->S, c->Sh, c->Mbuf[p], c->Mbuf[q], m, c->flag, c->gbar,
                              c->wait_limit, c->stream));
            c->cur = q;
            s += m;
        }
        return MM_OK;
    }
    for (int s = 0; s < n;) {
        const int p = c->cur;
        // single steps of the two-kernel path launch directly: a flushed
        // 256x256x4 step measured 23.2-23.5 us so against 24.7 us as a
        // one-step graph; runs of kGraphSteps replay their graph (17.0
        // against 17.3 us per L2-resident step launched one by one)
        if (c->use_graphs && (n - s >= kGraphSteps || !c->has_fs)) {
            const int kind = n - s >= kGraphSteps ? 1 : 0;
            if (!c->step_exec[kind][p] || c->step_dt[kind][p] != dt || c->step_ver[kind][p] != c->ver) {
                rc = capture_step(c, kind, p, dt);
                if (rc != MM_OK) return rc;
            }
            CU(cudaGraphLaunch(c->step_exec[kind][p], c->stream));
            if (!kind) c->cur = 1 - p;
            s += kind ? kGraphSteps : 1;
        } else {
            rc = enqueue_step(c, p, dt, c->stream);
            if (rc != MM_OK) return rc;
            c->cur = 1 - p;
            ++s;
        }
    }
    return MM_OK;
}

// A host buffer's address as kernels may use it: page-locked memory mapped
// into the device's address space, or, where the device reaches pageable
// host memory coherently (cudaDevAttrPageableMemoryAccess, e.g. over a
// cache-coherent chip-to-chip link), the address itself; nullptr otherwise
// (the caller then stages the data with copies).
// What a caller's pointer is, from one attribute query: device (or managed)
// memory, and for host memory the address kernels may use for it (nullptr
// when they cannot reach it).
struct PtrKind {
    bool device = false;
    void* view = nullptr;
};
static PtrKind ptr_kind(void* p) {
    PtrKind k;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return k;
    }
    k.device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) k.view = a.devicePointer;
    if (a.type == cudaMemoryTypeUnregistered) {
        int dev = 0, pageable = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess && pageable)
            k.view = p;
        cudaGetLastError();
    }
    return k;
}

extern "C" int mm_step_host(mm_ctx* c, const float* M_in, int n, double dt, float* M_out) {
    if (!c || !M_in || !M_out) return fail(MM_EINVAL, "null argument");
    if (n < 0) return fail(MM_EINVAL, "n must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MM_EINVAL, "dt must be > 0");
    const size_t bytes = sizeof(float) * 3 * (size_t)c->g.N;
    const PtrKind kin = ptr_kind(const_cast<float*>(M_in)), kout = ptr_kind(M_out);
    const bool fast = c->has_fs && c->method == MM_INTEGRATOR_EULER && !uses_persist(c) && n > 0 && !kin.device &&
                      !kout.device;
    if (!fast) {
        // copies around the ordinary step, one synchronisation at the end
        CU(cudaMemcpyAsync(c->Mbuf[c->cur], M_in, bytes, cudaMemcpyDefault, c->stream));
        CU(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
        c->spec_valid = false;
        int rc = mm_step(c, n, dt);
        if (rc != MM_OK) return rc;
        CU(cudaMemcpyAsync(M_out, c->Mbuf[c->cur], bytes, cudaMemcpyDefault, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        return MM_OK;
    }
    const float* in = (const float*)kin.view;
    float* out = (float*)kout.view;
    if (!in) {
        CU(cudaMemcpyAsync(c->Mbuf[c->cur], M_in, bytes, cudaMemcpyHostToDevice, c->stream));
        in = c->Mbuf[c->cur];
    }
    CU(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    // the x transform of the starting state reads it where it lies and
    // leaves a device copy for the updates; the last step's update writes
    // the new state to the context and to the caller's buffer
    float* cp = in == c->Mbuf[c->cur] ? nullptr : c->Mbuf[c->cur];
    CU(launch_pass1(c->g, c->l, in, c->S, c->stream, cp));
    const LlgCoef cf = make_coef(c, dt);
    int p = c->cur;
    for (int s = 0; s < n; ++s) {
        const float* Mn = c->Mbuf[p];
        float* copy = (s == n - 1) ? out : nullptr;
        CU(launch_step_pdl(c->g, c->fs, cf, c->S, c->Sh, Mn, c->Mbuf[1 - p], c->flag, c->stream, true, copy));
        p = 1 - p;
    }
    c->cur = p;
    c->spec_valid = true;
    if (!out) CU(cudaMemcpyAsync(M_out, c->Mbuf[p], bytes, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return MM_OK;
}

static int read_flag(mm_ctx* c) {
    int f = 0;
    CU(cudaMemcpy(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & kFlagTimeout) return fail(MM_ETIMEOUT, "a device-side wait gave up; the state is incomplete");
    if (f) return fail(MM_ENONFINITE, "a step produced a non-finite magnetisation");
    return MM_OK;
}

extern "C" int mm_sync(mm_ctx* c) {
    if (!c) return fail(MM_EINVAL, "null context");
    CU(cudaStreamSynchronize(c->stream));
    return read_flag(c);
}

extern "C" int mm_energy(mm_ctx* c, double E[5]) {
    if (!c || !E) return fail(MM_EINVAL, "null argument");
    int rc = run_passes(c, kModeDemag, c->Mbuf[c->cur], c->H, 0.0, c->stream);
    if (rc != MM_OK) return rc;
    CU(energy_reduce_full(c->g, c->Ms, c->Hext, c->cell, c->A, c->Ku, c->Mbuf[c->cur], c->H, c->partials,
                          c->Edev, c->stream));
    double h[5];
    CU(cudaMemcpyAsync(h, c->Edev, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    rc = read_flag(c);
    if (rc != MM_OK) return rc;
    for (int q = 0; q < 5; ++q) E[q] = h[q];
    return MM_OK;
}

extern "C" const char* mm_last_error(const mm_ctx*) { return g_err; }

extern "C" int mm_plan_info(const mm_ctx* c, int L[3]) {
    if (!c) return fail(MM_EINVAL, "null context");
    if (L) {
        L[0] = c->g.Lx;
        L[1] = c->g.Ly;
        L[2] = c->g.Lz;
    }
    if (c->has_gx) return c->l.split ? 4 : 2;
    return c->has_fs ? 2 : (c->has_ss ? 4 : (c->l.split ? 5 : 3));
}

extern "C" int mm_tensor_octant(mm_ctx* c, double* out) {
    if (!c || !out) return fail(MM_EINVAL, "null argument");
    const size_t n = (size_t)6 * c->g.N;
    double* Nd = nullptr;
    CU(cudaMalloc(&Nd, sizeof(double) * n));
    cudaError_t e = tensor_octant_fp64(c->grid, c->cell, Nd, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, Nd, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(Nd);
    CU(e);
    return MM_OK;
}

extern "C" int mm_kernel_spectrum(mm_ctx* c, float* out) {
    if (!c || !out) return fail(MM_EINVAL, "null argument");
    const size_t n = (size_t)6 * c->g.Hx * c->g.Hy * c->g.Hz;
    CU(cudaMemcpyAsync(out, c->Kt, sizeof(float) * n, cudaMemcpyDefault, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return MM_OK;
}

extern "C" int mm_time_passes(mm_ctx* c, int reps, double dt, void* flush, unsigned long long flush_bytes,
                              float ms[3]) {
    if (!c || !ms || reps < 1) return fail(MM_EINVAL, "null argument or reps < 1");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MM_EINVAL, "dt must be > 0");
    cudaEvent_t ev[4];
    for (int q = 0; q < 4; ++q) CU(cudaEventCreate(&ev[q]));
    double acc[3] = {0, 0, 0};
    int rc = MM_OK;
    const LlgCoef cf = make_coef(c, dt);
    for (int r = 0; r < reps && rc == MM_OK; ++r) {
        rc = [&]() -> int {
            const int p = c->cur;
            if (flush) CU(cudaMemsetAsync(flush, r & 0xff, (size_t)flush_bytes, c->stream));
            CU(cudaEventRecord(ev[0], c->stream));
            if (c->has_fs) {
                // pass 1 alone (the two-kernel step folds it into K_B), then K_A, K_B
                CU(launch_pass1(c->g, c->l, c->Mbuf[p], c->S, c->stream));
                CU(cudaEventRecord(ev[1], c->stream));
                CU(launch_step_a(c->g, c->fs, c->Kd, c->S, c->Sh, c->flag, c->stream, false, 0));
                CU(cudaEventRecord(ev[2], c->stream));
                CU(launch_step_b(c->g, c->fs, cf, c->Sh, c->S, c->Mbuf[p], c->Mbuf[1 - p], c->flag,
                                 c->stream, false));
                c->spec_valid = true;
            } else {
                c->spec_valid = false;            // S no longer holds a step's x spectrum
                CU(launch_pass1(c->g, c->l, c->Mbuf[p], c->S, c->stream));
                CU(cudaEventRecord(ev[1], c->stream));
                CU(launch_plane(c->g, c->l, c->S, c->stream));
                CU(cudaEventRecord(ev[2], c->stream));
                CU(launch_pass3(c->g, c->l, cf, kModeStep, c->S, c->Mbuf[p], c->Mbuf[1 - p], c->flag, c->stream));
            }
            CU(cudaEventRecord(ev[3], c->stream));
            CU(cudaEventSynchronize(ev[3]));
            for (int q = 0; q < 3; ++q) {
                float t = 0.f;
                CU(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
                acc[q] += t;
            }
            c->cur = 1 - p;
            return MM_OK;
        }();
    }
    for (int q = 0; q < 4; ++q) cudaEventDestroy(ev[q]);
    if (rc != MM_OK) return rc;
    for (int q = 0; q < 3; ++q) ms[q] = (float)(acc[q] / reps);
    return MM_OK;
}

// ----------------------------------------------------- no-allocation entry --
// Callers that may not allocate device memory (a host that runs with a fixed
// memory budget, code that executes where cudaMalloc is forbidden or would
// synchronise the device) evaluate the demag field through
// mm_demag_field_noalloc.  Its only workspace is this file-scope device
// array: every GPU that loads the library holds it until the process exits.
// Layout per call: twiddles W_Lx, W_Ly, W_Lz, then the spectrum workspace.
static constexpr size_t kNoAllocComplex = (size_t)1 << 20;    // 8 MiB of float2
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocComplex];

static std::mutex g_noalloc_mu;
static float2* g_noalloc_ptr[64] = {nullptr};     // device address per device ordinal

__global__ void k_noalloc_twiddles(int Lx, int Ly, int Lz, float2* tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    int L, e;
    if (m < Lx) { L = Lx; e = m; }
    else if (m < Lx + Ly) { L = Ly; e = m - Lx; }
    else if (m < Lx + Ly + Lz) { L = Lz; e = m - Lx - Ly; }
    else return;
    double s, c;
    sincospi(-2.0 * e / L, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
}

extern "C" int mm_demag_field_noalloc(const int grid[3], const float* Kt_dev, long long kt_elems,
                                      const float* M_dev, float* H_dev, void* cuda_stream) {
    if (!grid || !Kt_dev || !M_dev || !H_dev) return fail(MM_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1) return fail(MM_EINVAL, "grid[%d] = %d < 1", a, grid[a]);
    if ((long long)grid[0] * grid[1] * grid[2] > (1LL << 28)) return fail(MM_EUNSUPPORTED, "grid too large");
    // plan on a stack context: no device or host allocation
    mm_ctx tmp;
    for (int a = 0; a < 3; ++a) tmp.grid[a] = grid[a];
    int rc = build_plan(&tmp);
    if (rc != MM_OK) return rc;
    Geom g = tmp.g;
    const size_t N = (size_t)g.N;
    if (overlap(M_dev, H_dev, 3 * N)) return fail(MM_EINVAL, "M and H overlap");
    const size_t ntw = (size_t)g.Lx + g.Ly + g.Lz;
    const size_t nspec = (size_t)g.Hx * 3 * g.nz * g.Jst;
    const size_t need = ((ntw + 31) & ~(size_t)31) + nspec;
    if (need > kNoAllocComplex)
        return fail(MM_EUNSUPPORTED,
                    "grid %dx%dx%d needs %zu bytes of workspace; the static workspace holds %zu bytes",
                    grid[0], grid[1], grid[2], need * sizeof(float2), kNoAllocComplex * sizeof(float2));
    const long long kt_need = 6LL * g.Hx * g.Hy * g.Hz;
    if (kt_elems != kt_need)
        return fail(MM_EINVAL, "Kt holds %lld floats; the spectrum of grid %dx%dx%d has %lld", kt_elems, grid[0],
                    grid[1], grid[2], kt_need);
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(MM_EUNSUPPORTED, "device ordinal %d out of range", dev);
    float2* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_ptr[dev] = (float2*)p;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float2* tw = base;
    float2* S = base + ((ntw + 31) & ~(size_t)31);
    g.twx = tw;
    g.twy = tw + g.Lx;
    g.twz = tw + g.Lx + g.Ly;
    g.Kt = Kt_dev;
    g.Kd = nullptr;
    g.Kd0 = nullptr;
    CU(configure_pass_kernels(g, tmp.l));
    k_noalloc_twiddles<<<(unsigned)((ntw + 255) / 256), 256, 0, s>>>(g.Lx, g.Ly, g.Lz, tw);
    CU(cudaGetLastError());
    // every workspace element the passes read is written earlier in this call
    const LlgCoef cf{};
    CU(launch_pass1(g, tmp.l, M_dev, S, s));
    CU(launch_plane(g, tmp.l, S, s));
    CU(launch_pass3(g, tmp.l, cf, kModeDemag, S, M_dev, H_dev, nullptr, s));
    return MM_OK;
}

