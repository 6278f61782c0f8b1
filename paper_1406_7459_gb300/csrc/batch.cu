// batch.cu -- many independent samples of uneven size stepped together.
//
// Each sample is a complete problem of its own (grid, cell, material, field)
// with its own tensor spectrum; the step of every sample is the paper's
// three phases (Sec. 3: forward FFTs, member-wise product, inverse FFTs,
// then the field and Euler update).  All samples advance in lock step: one
// batched kernel per pass covers the tiles of every sample, each CTA
// finding its (sample, tile) in a prefix table over a per-sample
// descriptor array, and the three launches of a step replay from one CUDA
// graph.  Or (MM_STEP_PERSISTENT) one cooperative launch runs many steps,
// captured once in a CUDA graph and replayed on later calls:
// its blocks take (sample, tile) items from a work queue per pass, passes
// separated by bounded grid barriers, the x R2C of the next step fused into
// the update pass.  The tile shapes (rows per CTA in the x passes, threads
// per CTA) come from an autotuner that times candidate shapes on the batch
// itself.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mm.h"
#include "bulk_copy.cuh"
#include "grid_sync.cuh"
#include "pass_bodies.cuh"
#include "plane_kernel.cuh"

using namespace mmk;

namespace mmk {

struct BatchDesc {
    Geom g;
    LlgCoef cf;
    float* M0;
    float* M1;
    float2* S;
    int r1, r3;
    int r2;                                   // kx planes per plane-pass CTA
};

__device__ __forceinline__ int find_sample(const int* __restrict__ pre, int ns, int b) {
    int lo = 0, hi = ns - 1;                  // largest s with pre[s] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_pass1(const BatchDesc* __restrict__ d, const int* __restrict__ pre,
                                                      int ns, int par) {
    const int s = find_sample(pre, ns, blockIdx.x);
    const BatchDesc& b = d[s];
    pass1_body(b.g, b.r1, b.r1 / 2, par ? b.M1 : b.M0, b.S, blockIdx.x - __ldg(pre + s));
}

// plane-pass tile `tile` of a sample: r2 consecutive kx planes (fewer at
// the end), all their lines transformed together
__device__ __forceinline__ void batch_plane_tile(const BatchDesc& b, int tile) {
    const int kx0 = tile * b.r2;
    const int np = min(b.r2, b.g.Hx - kx0);
    const int nl = 3 * b.g.nz * np;
    switch (b.g.Lz) {
        case 1: plane_body_multi<1>(b.g, nl, b.S, kx0, np); break;
        case 4: plane_body_multi<4>(b.g, nl, b.S, kx0, np); break;
        case 5: plane_body_multi<5>(b.g, nl, b.S, kx0, np); break;
        default: plane_body_multi<8>(b.g, nl, b.S, kx0, np); break;
    }
}

__global__ void __launch_bounds__(256) k_batch_plane(const BatchDesc* __restrict__ d, const int* __restrict__ pre,
                                                      int ns) {
    const int s = find_sample(pre, ns, blockIdx.x);
    batch_plane_tile(d[s], blockIdx.x - __ldg(pre + s));
}

// The update pass; it also forms the x spectra of the new states in place
// (kModeStepX: a tile reads exactly the spectrum entries it writes), the
// first pass of the next step.
__global__ void __launch_bounds__(256) k_batch_pass3(const BatchDesc* __restrict__ d, const int* __restrict__ pre,
                                                      int ns, int par, float dt, int* __restrict__ flag) {
    const int s = find_sample(pre, ns, blockIdx.x);
    const BatchDesc& b = d[s];
    LlgCoef cf = b.cf;
    cf.dt = dt;
    pass3_body<kModeStepX>(b.g, b.r3, 3 * b.r3 / 2, cf, b.S, par ? b.M1 : b.M0, par ? b.M0 : b.M1, flag,
                           blockIdx.x - __ldg(pre + s), b.S);
}

// n steps of every sample in one cooperative launch.  Work queue 0 holds
// the pass-1 tiles (the x R2C of the starting state; only when the spectra
// are not already those of that state), queue 1 the plane tiles, queue 2
// the update tiles, which also form the next step's x spectra (kModeStepX,
// in place: a tile reads exactly the spectrum entries it writes).  The
// state goes M[par0] -> M[par0 ^ 1] -> ...  A grid-barrier wait that runs
// out of polls sets kFlagTimeout.
__global__ void __launch_bounds__(256) k_batch_persist(const BatchDesc* __restrict__ d, const int* __restrict__ pre,
                                                        int ns, int t1, int t2, int t3, int par0, int nsteps,
                                                        float dt, int first_x, int* __restrict__ flag,
                                                        GridBar* __restrict__ gb, long long limit) {
    __shared__ int slot;
    const int P = ns + 1;
    unsigned bar = 0;
    bool ok = true;
    if (first_x) {
        for (int i; (i = queue_next(gb, 0, t1, 0, &slot)) >= 0;) {
            const int s = find_sample(pre, ns, i);
            const BatchDesc& b = d[s];
            pass1_body(b.g, b.r1, b.r1 / 2, par0 ? b.M1 : b.M0, b.S, i - __ldg(pre + s));
        }
        ok = grid_sync(gb, bar++, limit);
    }
    for (int st = 0; ok && st < nsteps; ++st) {
        const int par = (par0 + st) & 1;
        for (int i; (i = queue_next(gb, 1, t2, st, &slot)) >= 0;) {
            const int s = find_sample(pre + P, ns, i);
            batch_plane_tile(d[s], i - __ldg(pre + P + s));
        }
        ok = grid_sync(gb, bar++, limit);
        if (!ok) break;
        for (int i; (i = queue_next(gb, 2, t3, st, &slot)) >= 0;) {
            const int s = find_sample(pre + 2 * P, ns, i);
            const BatchDesc& b = d[s];
            LlgCoef cf = b.cf;
            cf.dt = dt;
            pass3_body<kModeStepX>(b.g, b.r3, 3 * b.r3 / 2, cf, b.S, par ? b.M1 : b.M0, par ? b.M0 : b.M1, flag,
                                   i - __ldg(pre + 2 * P + s), b.S);
        }
        if (st + 1 < nsteps) ok = grid_sync(gb, bar++, limit);
    }
    if (!ok && threadIdx.x == 0) atomicOr(flag, kFlagTimeout);
    grid_exit(gb);
}

}  // namespace mmk

// Steps per launch of the persistent batch step.
static constexpr int kBatchChunk = 1024;

struct mm_batch {
    int ns = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<int> grid;                     // 3 per sample
    std::vector<double> cell, Ms, A, Ku, alpha, gamma, Hext;
    std::vector<BatchDesc> desc;               // host copy
    std::vector<size_t> moff;                  // float offset of each sample's M
    size_t mtotal = 0;                         // floats per M buffer (sum 3 N_s)
    long long cells = 0;
    float* M0 = nullptr;
    float* M1 = nullptr;
    float2* S = nullptr;
    float* Kt = nullptr;
    float2* tw = nullptr;
    BatchDesc* d_desc = nullptr;
    int* d_pre = nullptr;                      // 3 prefix arrays of ns + 1
    int* flag = nullptr;
    int tiles[3] = {0, 0, 0};
    size_t smem[3] = {0, 0, 0};
    int threads = 256, r1 = 4, r3 = 2, r2 = 1;
    int par = 0;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    double exec_dt[2] = {0, 0};
    unsigned long long exec_ver[2] = {0, 0};
    unsigned long long ver = 1;
    // persistent step: counters, co-resident grid, shared memory, choice
    GridBar* gb = nullptr;
    int pgrid = 0;
    size_t psmem = 0;
    int path = MM_STEP_AUTO;
    long long wait_limit = kGridWaitLimit;
    bool spec_valid = false;                   // S holds the x spectra of the current state
    // the persistent launch captured in a graph, for the arguments it was
    // captured with; pgraph_ok false once a capture failed (direct launches)
    cudaGraphExec_t pexec = nullptr;
    int pexec_m = 0, pexec_par = 0, pexec_first = 0;
    double pexec_dt = 0;
    long long pexec_limit = 0;
    unsigned long long pexec_ver = 0;
    bool pgraph_ok = true;
    int form = -1;                             // mm_batch_launch_form of the last step
};

#define BCU(expr)                                                                                    \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) {                                                                     \
            char _m[256];                                                                            \
            snprintf(_m, sizeof(_m), "%s: %s", #expr, cudaGetErrorString(_e));                       \
            return set_error(_e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA, _m);            \
        }                                                                                            \
    } while (0)

static LlgCoef batch_coef(const mm_batch* b, int s) {
    LlgCoef f;
    const double Ms = b->Ms[s], Ms2 = Ms * Ms, al = b->alpha[s], den = 1.0 + al * al;
    const double mu0 = 4.0e-7 * 3.14159265358979323846;
    f.Ms = (float)Ms;
    f.pexch = (float)(2.0 * b->A[s] / (mu0 * Ms2));
    f.panis = (float)(-2.0 * b->Ku[s] / (mu0 * Ms2));
    f.c1 = (float)(-b->gamma[s] / den);
    f.c2 = (float)(-al * b->gamma[s] / (den * Ms));
    f.idx2 = (float)(1.0 / (b->cell[3 * s] * b->cell[3 * s]));
    f.idy2 = (float)(1.0 / (b->cell[3 * s + 1] * b->cell[3 * s + 1]));
    f.idz2 = (float)(1.0 / (b->cell[3 * s + 2] * b->cell[3 * s + 2]));
    f.hx = (float)b->Hext[3 * s];
    f.hy = (float)b->Hext[3 * s + 1];
    f.hz = (float)b->Hext[3 * s + 2];
    f.dt = 0.f;
    return f;
}

// Tile counts, prefix tables, shared-memory sizes and descriptors for the
// current shape choice (r1, r3, threads); uploads them.
static int batch_layout(mm_batch* b) {
    std::vector<int> pre(3 * (b->ns + 1));
    size_t sm[3] = {0, 0, 0};
    int acc[3] = {0, 0, 0};
    for (int s = 0; s < b->ns; ++s) {
        BatchDesc& d = b->desc[s];
        const Geom& g = d.g;
        d.r1 = b->r1;
        d.r3 = b->r3;
        d.r2 = b->r2;
        d.cf = batch_coef(b, s);
        const int t1 = 3 * g.nz * ((g.ny + b->r1 - 1) / b->r1);
        const int t2 = (g.Hx + b->r2 - 1) / b->r2;
        const int t3 = g.nz * ((g.ny + b->r3 - 1) / b->r3);
        pre[0 * (b->ns + 1) + s] = acc[0];
        pre[1 * (b->ns + 1) + s] = acc[1];
        pre[2 * (b->ns + 1) + s] = acc[2];
        acc[0] += t1;
        acc[1] += t2;
        acc[2] += t3;
        const size_t lx = (size_t)padded_len(g.Lx) * sizeof(float2), ly = (size_t)padded_len(g.Ly) * sizeof(float2);
        const size_t a1 = 2 * (size_t)(b->r1 / 2) * lx, a2 = 2 * (size_t)3 * g.nz * b->r2 * ly,
                     a3 = 2 * (size_t)(3 * b->r3 / 2) * lx;
        sm[0] = a1 > sm[0] ? a1 : sm[0];
        sm[1] = a2 > sm[1] ? a2 : sm[1];
        sm[2] = a3 > sm[2] ? a3 : sm[2];
    }
    for (int q = 0; q < 3; ++q) {
        pre[q * (b->ns + 1) + b->ns] = acc[q];
        b->tiles[q] = acc[q];
        b->smem[q] = sm[q];
        if (sm[q] > 227 * 1024) return set_error(MM_EUNSUPPORTED, "batch sample exceeds shared memory");
    }
    BCU(cudaFuncSetAttribute(k_batch_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[0]));
    BCU(cudaFuncSetAttribute(k_batch_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[1]));
    BCU(cudaFuncSetAttribute(k_batch_pass3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[2]));
    {
        size_t ps = sm[0] > sm[1] ? sm[0] : sm[1];
        ps = ps > sm[2] ? ps : sm[2];
        b->psmem = ps;
        BCU(cudaFuncSetAttribute(k_batch_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps));
        int dev = 0, sms = 0, per_sm = 0;
        BCU(cudaGetDevice(&dev));
        BCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persist, b->threads, ps));
        b->pgrid = per_sm * sms;
    }
    BCU(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(BatchDesc) * b->ns, cudaMemcpyHostToDevice));
    BCU(cudaMemcpy(b->d_pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    b->ver++;
    return MM_OK;
}

// x R2C of every sample's state M[par] into its spectrum
static int batch_pass1(mm_batch* b, int par, cudaStream_t s) {
    k_batch_pass1<<<b->tiles[0], b->threads, b->smem[0], s>>>(b->d_desc, b->d_pre, b->ns, par);
    BCU(cudaGetLastError());
    return MM_OK;
}

// One step from spectra that hold the x transforms of M[par]: the plane
// pass, then the update, which leaves the x transforms of M[par ^ 1].
static int batch_enqueue(mm_batch* b, int par, double dt, cudaStream_t s) {
    const int P = b->ns + 1;
    k_batch_plane<<<b->tiles[1], b->threads, b->smem[1], s>>>(b->d_desc, b->d_pre + P, b->ns);
    BCU(cudaGetLastError());
    k_batch_pass3<<<b->tiles[2], b->threads, b->smem[2], s>>>(b->d_desc, b->d_pre + 2 * P, b->ns, par, (float)dt,
                                                              b->flag);
    BCU(cudaGetLastError());
    return MM_OK;
}

static void batch_release(mm_batch* b) {
    for (int p = 0; p < 2; ++p)
        if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    cudaFree(b->M0);
    cudaFree(b->M1);
    cudaFree(b->S);
    cudaFree(b->Kt);
    cudaFree(b->tw);
    cudaFree(b->d_desc);
    cudaFree(b->d_pre);
    cudaFree(b->flag);
    cudaFree(b->gb);
    if (b->cap) cudaStreamDestroy(b->cap);
}

extern "C" int mm_batch_create(mm_batch** out, int n, const int* grids, const double* cells, const double* Ms,
                               const double* A, const double* Ku, const double* alpha, const double* gamma,
                               void* cuda_stream) {
    if (!out) return set_error(MM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !cells || !Ms || !A || !Ku || !alpha || !gamma)
        return set_error(MM_EINVAL, "n < 1 or null array");
    mm_batch* b = new (std::nothrow) mm_batch();
    if (!b) return set_error(MM_ENOMEM, "host allocation failed");
    b->ns = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->grid.assign(grids, grids + 3 * n);
    b->cell.assign(cells, cells + 3 * n);
    b->Ms.assign(Ms, Ms + n);
    b->A.assign(A, A + n);
    b->Ku.assign(Ku, Ku + n);
    b->alpha.assign(alpha, alpha + n);
    b->gamma.assign(gamma, gamma + n);
    b->Hext.assign(3 * n, 0.0);
    b->desc.resize(n);
    b->moff.resize(n);
    int rc = [&]() -> int {
        size_t mt = 0, st = 0, kt = 0, tt = 0, wmax = 0, nmax = 0;
        std::vector<size_t> soff(n), koff(n), toff(n);
        for (int s = 0; s < n; ++s) {
            const int nx = grids[3 * s], ny = grids[3 * s + 1], nz = grids[3 * s + 2];
            if (nx < 1 || ny < 1 || nz < 1) return set_error(MM_EINVAL, "grid entries must be >= 1");
            for (int a = 0; a < 3; ++a)
                if (!(cells[3 * s + a] > 0.0)) return set_error(MM_EINVAL, "cell sizes must be > 0");
            if (!(Ms[s] > 0.0) || !(A[s] >= 0.0) || !(alpha[s] >= 0.0) || !(gamma[s] > 0.0) || !std::isfinite(Ku[s]))
                return set_error(MM_EINVAL, "bad material value");
            Geom& g = b->desc[s].g;
            memset(&g, 0, sizeof(g));
            g.nx = nx;
            g.ny = ny;
            g.nz = nz;
            g.N = nx * ny * nz;
            g.Lx = plan_padded_length(nx);
            g.Ly = plan_padded_length(ny);
            g.Lz = plan_padded_length(nz);
            if (g.Lx > kMaxLen || g.Ly > kMaxLen || g.Lz > 8)
                return set_error(MM_EUNSUPPORTED, "batch samples need padded lengths <= 4096 and nz <= 4");
            g.Hx = g.Lx / 2 + 1;
            g.Hy = g.Ly / 2 + 1;
            g.Hz = g.Lz / 2 + 1;
            g.Jst = ny;
            if (!plan_axis(g.Lx, &g.px) || !plan_axis(g.Ly, &g.py) || !plan_axis(g.Lz, &g.pz))
                return set_error(MM_EUNSUPPORTED, "no radix plan");
            b->moff[s] = mt;
            mt += 3 * (size_t)g.N;
            soff[s] = st;
            st += (size_t)g.Hx * 3 * nz * ny;
            koff[s] = kt;
            kt += (size_t)6 * g.Hx * g.Hy * g.Hz;
            toff[s] = tt;
            tt += (size_t)(g.Lx + g.Ly + g.Lz);
            const int L[3] = {g.Lx, g.Ly, g.Lz};
            const size_t w = tensor_work_elems(&grids[3 * s], L);
            wmax = w > wmax ? w : wmax;
            nmax = (size_t)g.N > nmax ? (size_t)g.N : nmax;
            b->cells += g.N;
        }
        b->mtotal = mt;
        BCU(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        BCU(cudaMalloc(&b->M0, sizeof(float) * mt));
        BCU(cudaMalloc(&b->M1, sizeof(float) * mt));
        BCU(cudaMalloc(&b->S, sizeof(float2) * st));
        BCU(cudaMalloc(&b->Kt, sizeof(float) * kt));
        BCU(cudaMalloc(&b->tw, sizeof(float2) * tt));
        BCU(cudaMalloc(&b->d_desc, sizeof(BatchDesc) * n));
        BCU(cudaMalloc(&b->d_pre, sizeof(int) * 3 * (n + 1)));
        BCU(cudaMalloc(&b->flag, sizeof(int)));
        BCU(cudaMemset(b->flag, 0, sizeof(int)));
        BCU(cudaMalloc(&b->gb, sizeof(GridBar)));
        BCU(cudaMemset(b->gb, 0, sizeof(GridBar)));
        std::vector<float2> htw(tt);
        std::vector<float> hm(mt);
        for (int s = 0; s < n; ++s) {
            Geom& g = b->desc[s].g;
            float2* t = htw.data() + toff[s];
            plan_twiddles(g.Lx, t);
            plan_twiddles(g.Ly, t + g.Lx);
            plan_twiddles(g.Lz, t + g.Lx + g.Ly);
            g.twx = b->tw + toff[s];
            g.twy = g.twx + g.Lx;
            g.twz = g.twy + g.Ly;
            g.Kt = b->Kt + koff[s];
            g.Kd = nullptr;
            g.Kd0 = nullptr;
            b->desc[s].M0 = b->M0 + b->moff[s];
            b->desc[s].M1 = b->M1 + b->moff[s];
            b->desc[s].S = b->S + soff[s];
            for (int i = 0; i < g.N; ++i) {
                hm[b->moff[s] + i] = (float)Ms[s];
                hm[b->moff[s] + g.N + i] = 0.f;
                hm[b->moff[s] + 2 * (size_t)g.N + i] = 0.f;
            }
        }
        BCU(cudaMemcpy(b->tw, htw.data(), sizeof(float2) * tt, cudaMemcpyHostToDevice));
        BCU(cudaMemcpy(b->M0, hm.data(), sizeof(float) * mt, cudaMemcpyHostToDevice));
        // per-sample FP64 tensor set-up into each sample's spectrum slice
        double *Nd = nullptr, *w1 = nullptr, *w2 = nullptr;
        cudaError_t e = cudaMalloc(&Nd, sizeof(double) * 6 * nmax);
        if (e == cudaSuccess) e = cudaMalloc(&w1, sizeof(double) * wmax);
        if (e == cudaSuccess) e = cudaMalloc(&w2, sizeof(double) * wmax);
        for (int s = 0; s < n && e == cudaSuccess; ++s) {
            const Geom& g = b->desc[s].g;
            const int L[3] = {g.Lx, g.Ly, g.Lz};
            e = tensor_octant_fp64(&grids[3 * s], &cells[3 * s], Nd, b->stream);
            if (e == cudaSuccess) e = tensor_spectrum(&grids[3 * s], L, Nd, b->Kt + koff[s], w1, w2, b->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        cudaFree(Nd);
        cudaFree(w1);
        cudaFree(w2);
        BCU(e);
        return batch_layout(b);
    }();
    if (rc != MM_OK) {
        batch_release(b);
        delete b;
        return rc;
    }
    *out = b;
    return MM_OK;
}

extern "C" int mm_batch_destroy(mm_batch* b) {
    if (!b) return MM_OK;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
    return MM_OK;
}

extern "C" int mm_batch_set_field(mm_batch* b, const double* H) {
    if (!b || !H) return set_error(MM_EINVAL, "null argument");
    for (int i = 0; i < 3 * b->ns; ++i) {
        if (!std::isfinite(H[i])) return set_error(MM_EINVAL, "H_ext must be finite");
        b->Hext[i] = H[i];
    }
    return batch_layout(b);
}

extern "C" int mm_batch_set_m(mm_batch* b, const float* M) {
    if (!b || !M) return set_error(MM_EINVAL, "null argument");
    BCU(cudaMemcpyAsync(b->par ? b->M1 : b->M0, M, sizeof(float) * b->mtotal, cudaMemcpyDefault, b->stream));
    BCU(cudaMemsetAsync(b->flag, 0, sizeof(int), b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    b->spec_valid = false;
    return MM_OK;
}

extern "C" int mm_batch_get_m(mm_batch* b, float* M) {
    if (!b || !M) return set_error(MM_EINVAL, "null argument");
    BCU(cudaMemcpyAsync(M, b->par ? b->M1 : b->M0, sizeof(float) * b->mtotal, cudaMemcpyDefault, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return MM_OK;
}

// The persistent batch step is taken when asked for (MM_STEP_PERSISTENT)
// and when every block of its grid fits on the device at once.
static bool batch_uses_persist(const mm_batch* b) { return b->path == MM_STEP_PERSISTENT && b->pgrid > 0; }

extern "C" int mm_batch_set_path(mm_batch* b, int path) {
    if (!b) return set_error(MM_EINVAL, "null batch");
    if (path != MM_STEP_AUTO && path != MM_STEP_GRAPH && path != MM_STEP_PERSISTENT)
        return set_error(MM_EINVAL, "unknown step path");
    if (path == MM_STEP_PERSISTENT && b->pgrid < 1)
        return set_error(MM_EUNSUPPORTED, "the persistent batch step does not fit on this device");
    b->path = path;
    return MM_OK;
}

extern "C" int mm_batch_set_wait_limit(mm_batch* b, long long polls) {
    if (!b) return set_error(MM_EINVAL, "null batch");
    if (polls < 0) return set_error(MM_EINVAL, "polls must be >= 0");
    b->wait_limit = polls;
    return MM_OK;
}

// One cooperative launch of m steps on stream s.
static cudaError_t batch_launch_persist(const mm_batch* b, int m, double dt, int first, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->pgrid);
    cfg.blockDim = dim3(b->threads);
    cfg.dynamicSmemBytes = b->psmem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_persist, (const BatchDesc*)b->d_desc, (const int*)b->d_pre, b->ns,
                              b->tiles[0], b->tiles[1], b->tiles[2], b->par, m, (float)dt, first, b->flag, b->gb,
                              b->wait_limit);
}

// The launch of m steps as a graph replay: captured (on the capture stream)
// the first time and again whenever its arguments change.  A capture or
// instantiation the runtime refuses switches the batch to direct launches.
static cudaError_t batch_replay_persist(mm_batch* b, int m, double dt, int first) {
    const bool same = b->pexec && b->pexec_m == m && b->pexec_dt == dt && b->pexec_par == b->par &&
                      b->pexec_first == first && b->pexec_limit == b->wait_limit && b->pexec_ver == b->ver;
    if (!same) {
        if (b->pexec) {
            cudaGraphExecDestroy(b->pexec);
            b->pexec = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t el = batch_launch_persist(b, m, dt, first, b->cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap, &graph);
        if (el != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return el != cudaSuccess ? el : e;
        }
        e = cudaGraphInstantiate(&b->pexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->pexec = nullptr;
            return e;
        }
        b->pexec_m = m;
        b->pexec_dt = dt;
        b->pexec_par = b->par;
        b->pexec_first = first;
        b->pexec_limit = b->wait_limit;
        b->pexec_ver = b->ver;
    }
    return cudaGraphLaunch(b->pexec, b->stream);
}

static int batch_step_persist(mm_batch* b, int n, double dt) {
    for (int s = 0; s < n;) {
        const int m = n - s < kBatchChunk ? n - s : kBatchChunk;
        const int first = b->spec_valid ? 0 : 1;
        cudaError_t e = cudaErrorNotSupported;
        if (b->pgraph_ok) {
            e = batch_replay_persist(b, m, dt, first);
            if (e != cudaSuccess) {
                cudaGetLastError();                       // a refused capture leaves no sticky error
                b->pgraph_ok = false;
            }
        }
        if (e != cudaSuccess) BCU(batch_launch_persist(b, m, dt, first, b->stream));
        b->form = e == cudaSuccess ? 1 : 2;
        b->par = (b->par + m) & 1;
        b->spec_valid = true;
        s += m;
    }
    return MM_OK;
}

extern "C" int mm_batch_step(mm_batch* b, int n, double dt) {
    if (!b) return set_error(MM_EINVAL, "null batch");
    if (n < 0 || !(dt > 0.0) || !std::isfinite(dt)) return set_error(MM_EINVAL, "n >= 0 and dt > 0 required");
    if (n == 0) return MM_OK;
    if (batch_uses_persist(b)) return batch_step_persist(b, n, dt);
    if (!b->spec_valid) {
        int rc = batch_pass1(b, b->par, b->stream);
        if (rc != MM_OK) return rc;
        b->spec_valid = true;
    }
    for (int s = 0; s < n; ++s) {
        const int p = b->par;
        if (!b->exec[p] || b->exec_dt[p] != dt || b->exec_ver[p] != b->ver) {
            if (b->exec[p]) {
                cudaGraphExecDestroy(b->exec[p]);
                b->exec[p] = nullptr;
            }
            BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            int rc = batch_enqueue(b, p, dt, b->cap);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
            if (rc != MM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            BCU(e);
            e = cudaGraphInstantiate(&b->exec[p], graph, 0);
            cudaGraphDestroy(graph);
            BCU(e);
            b->exec_dt[p] = dt;
            b->exec_ver[p] = b->ver;
        }
        BCU(cudaGraphLaunch(b->exec[p], b->stream));
        b->form = 0;
        b->par = 1 - p;
    }
    return MM_OK;
}

extern "C" int mm_batch_sync(mm_batch* b) {
    if (!b) return set_error(MM_EINVAL, "null batch");
    BCU(cudaStreamSynchronize(b->stream));
    int f = 0;
    BCU(cudaMemcpy(&f, b->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & kFlagTimeout) return set_error(MM_ETIMEOUT, "a grid-barrier wait of the batch step gave up");
    if (f) return set_error(MM_ENONFINITE, "a batch step produced a non-finite magnetisation");
    return MM_OK;
}

extern "C" long long mm_batch_cells(const mm_batch* b) { return b ? b->cells : -1; }

extern "C" int mm_batch_launch_form(const mm_batch* b) { return b ? b->form : -1; }

extern "C" int mm_batch_autotune(mm_batch* b, double dt, int choice[4], float* ms_out) {
    if (!b || !(dt > 0.0)) return set_error(MM_EINVAL, "null batch or dt <= 0");
    // keep the state: tuning steps run on a saved copy
    float* save = nullptr;
    BCU(cudaMalloc(&save, sizeof(float) * b->mtotal));
    float* cur = b->par ? b->M1 : b->M0;
    BCU(cudaMemcpyAsync(save, cur, sizeof(float) * b->mtotal, cudaMemcpyDeviceToDevice, b->stream));
    static const int cand[][3] = {{2, 2, 128}, {4, 2, 128}, {8, 2, 128}, {2, 4, 128}, {4, 4, 128}, {8, 4, 128},
                                  {2, 2, 256}, {4, 2, 256}, {8, 2, 256}, {2, 4, 256}, {4, 4, 256}, {8, 4, 256}};
    const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bi = 0;
    int rc = MM_OK;
    b->r2 = 1;
    for (int c = 0; c < nc && rc == MM_OK; ++c) {
        b->r1 = cand[c][0];
        b->r3 = cand[c][1];
        b->threads = cand[c][2];
        rc = batch_layout(b);
        if (rc != MM_OK) break;
        rc = batch_pass1(b, b->par, b->stream);
        if (rc == MM_OK) rc = batch_enqueue(b, b->par, dt, b->stream);   // warm-up
        if (rc != MM_OK) break;
        b->par = 1 - b->par;
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 3 && rc == MM_OK; ++k) {
            rc = batch_enqueue(b, b->par, dt, b->stream);
            b->par = 1 - b->par;
        }
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms_out) ms_out[c] = ms;
        if (ms < best) {
            best = ms;
            bi = c;
        }
    }
    // second stage: kx planes per plane-pass CTA with the best x-pass shapes
    static const int cand2[] = {1, 2, 4, 8};
    int b2 = 0;
    float best2 = 1e30f;
    for (int c = 0; c < 4 && rc == MM_OK; ++c) {
        b->r1 = cand[bi][0];
        b->r3 = cand[bi][1];
        b->threads = cand[bi][2];
        b->r2 = cand2[c];
        rc = batch_layout(b);
        if (rc != MM_OK) break;
        rc = batch_pass1(b, b->par, b->stream);
        if (rc == MM_OK) rc = batch_enqueue(b, b->par, dt, b->stream);   // warm-up
        if (rc != MM_OK) break;
        b->par = 1 - b->par;
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 3 && rc == MM_OK; ++k) {
            rc = batch_enqueue(b, b->par, dt, b->stream);
            b->par = 1 - b->par;
        }
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms_out) ms_out[nc + c] = ms;
        if (ms < best2) {
            best2 = ms;
            b2 = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == MM_OK) {
        b->r1 = cand[bi][0];
        b->r3 = cand[bi][1];
        b->threads = cand[bi][2];
        b->r2 = cand2[b2];
        rc = batch_layout(b);
    }
    cudaMemcpyAsync(b->par ? b->M1 : b->M0, save, sizeof(float) * b->mtotal, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemsetAsync(b->flag, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(save);
    b->spec_valid = false;
    if (rc != MM_OK) return rc;
    if (choice) {
        choice[0] = b->r1;
        choice[1] = b->r3;
        choice[2] = b->threads;
        choice[3] = b->r2;
    }
    return MM_OK;
}
