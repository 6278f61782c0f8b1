// mm_internal.h -- context, plan and launcher declarations shared by the
// translation units of libmm.so.  Not part of the public ABI (include/mm.h).
#pragma once
#include <cuda.h>   // CUtensorMap (type only)
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "fft_device.cuh"

namespace mmk {

constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;   // exact SI value
constexpr int kMaxLen = 4096;          // largest padded length per axis
constexpr int kMaxPlaneNz = 8;         // fused y/z plane kernel handles nz <= 8

// Geometry of the padded convolution.  Spectrum element (kx, c, k, j) of the
// workspace S sits at ((kx*3 + c)*nz + k)*Jst + j: kx slowest, so one kx
// plane (3*nz*ny complex) is contiguous for the plane kernel.
struct Geom {
    int nx, ny, nz, N;
    int Lx, Ly, Lz;
    int Hx, Hy, Hz;            // L/2 + 1: stored half-spectrum / octant extents
    int Jst;                   // stride of j in S (= ny)
    AxisPlan px, py, pz;
    const float2* twx;         // W_Lx^m, m < Lx (FP32, from FP64)
    const float2* twy;
    const float2* twz;
    const float* Kt;           // tensor spectrum [kx][kz'][ky'][6], scaled
    const float* Kd0;          // the same without the exchange stencil (demag-only evaluations)
    const float* Kd;           // 2-D (x, y) tensor spectrum per z offset [kx][dz][6][ky'], rows of
                               // kd_row(Hy) floats, scaled,
                               // with the zero-padded exchange stencil folded into xx, yy, zz;
                               // used by the direct-z plane kernel of the power-of-two step
};

#ifdef __CUDACC__
// Programmatic dependent launch: a kernel launched with the programmatic-
// serialisation attribute may start while its predecessor drains; it must
// call pdl_wait() before it reads or writes anything the predecessor may
// touch (a no-op when launched without the attribute).  pdl_trigger() lets
// the successor launch early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

// Launch configuration for cudaLaunchKernelEx, with programmatic stream
// serialisation when `pdl` (the kernel must then call pdl_wait() before it
// touches data of earlier kernels).  attr: storage for one attribute that
// must outlive the launch call.
inline cudaLaunchConfig_t launch_config(dim3 grid, int threads, size_t smem, cudaStream_t s,
                                        cudaLaunchAttribute* attr, bool pdl = true) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cfg;
}

// Row length (floats) of the 2-D spectrum Kd: Hy rounded up to 16 bytes.
inline __host__ __device__ constexpr int kd_row(int Hy) { return (Hy + 3) & ~3; }

// Field and LLG coefficients in FP32 (computed in FP64 on the host).
struct LlgCoef {
    float Ms;
    float pexch;               // 2A / (mu0 Ms^2)
    float panis;               // -2 Ku / (mu0 Ms^2)
    float c1;                  // -gamma / (1 + alpha^2)
    float c2;                  // -alpha gamma / ((1 + alpha^2) Ms)
    float idx2, idy2, idz2;    // 1 / delta^2
    float hx, hy, hz;          // H_ext
    float dt;
};

struct FastFns;
struct FastSplitFns;

// Launch shapes chosen at plan time.
struct Launch {
    int r1, t1, g1;            // pass 1: rows per tile, threads, line group
    int t2, g2;                // pass 2 (plane): threads, line group
    int r3, t3, g3;            // pass 3: rows per tile, threads, line group
    size_t smem1, smem2, smem3;
    const FastFns* fx = nullptr;     // compile-time x passes, if the grid has them
    const FastFns* fp = nullptr;     // compile-time plane kernel, if available
    bool split = false;              // pass 2 as y / z / y kernels (thick samples)
    const FastSplitFns* fs2 = nullptr;  // compile-time split kernels, if the grid has them
};

// kModeStepX (generic kernels only): the Euler step followed by the forward
// x R2C of the new rows into S, the first pass of the next step.
enum Pass3Mode { kModeDemag = 0, kModeHeff = 1, kModeStep = 2, kModeStepX = 3 };

// Planning helpers (mm_api.cu), shared with the batched driver.
int plan_padded_length(int n);
bool plan_axis(int L, AxisPlan* p);
void plan_twiddles(int L, float2* out);
int set_error(int code, const char* msg);

// Launchers (demag_passes.cu).  All asynchronous on `s`.
// Mcopy (compile-time x passes only, may be null): also copy M there.
cudaError_t launch_pass1(const Geom& g, const Launch& l, const float* M, float2* S, cudaStream_t s,
                         float* Mcopy = nullptr);
cudaError_t launch_plane(const Geom& g, const Launch& l, float2* S, cudaStream_t s);
cudaError_t launch_pass3(const Geom& g, const Launch& l, const LlgCoef& c, int mode, const float2* S,
                         const float* M, float* out, int* flag, cudaStream_t s);
cudaError_t configure_pass_kernels(const Geom& g, const Launch& l);
bool plane_supported_lz(int Lz);
typedef void (*PlaneFn)(Geom, int, float2*);
PlaneFn plane_fn_small(int Lz);   // plane_small.cu
PlaneFn plane_fn_mid(int Lz);     // plane_mid.cu

// Compile-time specialised kernels for power-of-two grids (fast_*.cu).
struct FastFns {
    void (*p1)(Geom, const float*, float2*, float*) = nullptr;
    int r1 = 0, t1 = 0;
    size_t s1 = 0;
    void (*pl)(Geom, float2*) = nullptr;
    int t2 = 0;
    size_t s2 = 0;
    void (*p3[3])(Geom, LlgCoef, const float2*, const float*, float*, int*) = {nullptr, nullptr, nullptr};
    int r3 = 0, t3 = 0;
    size_t s3 = 0;
};
// Compile-time split pass 2 (split_fast.cu): power-of-two ny in 16..1024,
// nz in 1..128 (zw = 0: one y position per thread for nz <= 8).
struct FastSplitFns {
    void (*yf)(Geom, float2*) = nullptr;
    void (*yi)(Geom, float2*) = nullptr;
    void (*zc)(Geom, const float*, float2*) = nullptr;
    int ylpc = 0, ty = 0, zw = 0, tz = 0;
    size_t sy = 0, sz = 0;
};
bool fast_split_lookup(int ny, int nz, FastSplitFns* f);
cudaError_t configure_fast_split(const FastSplitFns& f);
// y forward, z transform + product with the tensor spectrum Kt (g.Kt, or
// the exchange-folded copy for the split step), y inverse; in place on S.
cudaError_t launch_fast_split(const Geom& g, const FastSplitFns& f, const float* Kt, float2* S, cudaStream_t s);

bool fast_lookup_x(int nx, FastFns* f);
bool fast_lookup_plane_nz1(int ny, FastFns* f);
bool fast_lookup_plane_nz2(int ny, FastFns* f);
bool fast_lookup_plane_nz4(int ny, FastFns* f);
bool fast_lookup_plane_nz8(int ny, FastFns* f);

// Two-kernel step for power-of-two grids (fast_step*.cu): K_A = plane
// kernel from S into Sh (2-D spectrum given per launch: exchange-folded for
// the step and H_eff, plain for H_demag); K_B = inverse x + LLG + forward x
// from Sh into S, or its field-only variants.
struct FastStepFns {
    void (*ka)(Geom, const float*, const float2*, float2*, int*, int) = nullptr;
    int early = 0;             // K_A triggers K_B right after its wait (fast_step_early_trigger)
    int ta = 0;
    size_t sa = 0;
    // x-step kernels by Pass3Mode: demag field, effective field, Euler step
    void (*kb[3])(Geom, LlgCoef, const float2*, float2*, const float*, float*, int*, float*) = {nullptr, nullptr,
                                                                                               nullptr};
    // the same with the spectrum gather / scatter as tiled tensor copies
    // (nx <= 256), through the maps below when `tma` (maps encoded) and
    // `tma_use` (mm_set_tiled_copies) are set
    void (*kbt[3])(Geom, LlgCoef, const float2*, float2*, const float*, float*, int*, float*, CUtensorMap,
                   CUtensorMap, int) = {nullptr, nullptr, nullptr};
    int rb = 0, tb = 0;
    size_t sb = 0;
    bool tma = false;
    int tma_use = 0;                           // bit 0: tiled gather, bit 1: tiled scatter (opt-in:
                                               // measured slower than the per-thread copies)
    CUtensorMap tin{}, tout{};                 // gather map over tin_buf, scatter map over tout_buf
    const float2* tin_buf = nullptr;
    const float2* tout_buf = nullptr;
};
// Encode f->tin / f->tout for the x-step's gather from Sh and scatter to S
// (each buffer one kx plane longer than the spectrum: the box's unused
// odd-parity row falls there).  False, with f->tma cleared, where the box
// does not fit a map (nx > 256) or the CUDA driver's tensor-map encoder is
// unavailable.
bool encode_xstep_maps(const Geom& g, FastStepFns* f, const float2* Sh, const float2* S);
bool fast_step_lookup_x(int nx, FastStepFns* f);
bool fast_step_lookup_plane_a(int ny, int nz, FastStepFns* f);
bool fast_step_lookup_plane_b(int ny, int nz, FastStepFns* f);
// K_A reads the x half-spectrum S and writes its output to Sh; K_B reads Sh
// and writes the next step's S.
cudaError_t launch_step_pdl(const Geom& g, const FastStepFns& f, const LlgCoef& c, float2* S, float2* Sh,
                            const float* M, float* Mout, int* flag, cudaStream_t s, bool pdl,
                            float* Mcopy = nullptr);
cudaError_t configure_step_kernels(const FastStepFns& f);
int fast_step_early_trigger(const Geom& g, int sms);
cudaError_t launch_step_a(const Geom& g, const FastStepFns& f, const float* Kd, const float2* S, float2* Sh,
                          int* flag, cudaStream_t s, bool pdl, int early);
// The two-kernel evaluation of H_demag (mode kModeDemag, plain 2-D spectrum
// Kd0) or H_eff (kModeHeff, exchange-folded Kd) of M into out, after
// launch_pass1 has formed S from M.
cudaError_t launch_field_pdl(const Geom& g, const FastStepFns& f, const LlgCoef& c, int mode, const float* Kd,
                             float2* S, float2* Sh, const float* M, float* out, int* flag, cudaStream_t s);
// Persistent Euler step (step_persist.cu): K_A phase, grid barrier, K_B
// phase for n steps in one cooperative launch, for the square power-of-two
// films it is instantiated for.
struct GridBar;
struct PersistFns {
    void (*k)(Geom, LlgCoef, const float*, float2*, float2*, const float*, float*, int, int*, GridBar*,
              long long) = nullptr;
    int t = 0, grid = 0;
    size_t smem = 0;
};
bool persist_lookup(int nx, int ny, int nz, int R, PersistFns* f);
cudaError_t persist_configure(const Geom& g, int R, PersistFns* f, bool* usable);
cudaError_t persist_alloc_bar(GridBar** gb);
// n steps from M^n (Min, with S its x spectrum) to M^{n+n} in Mout; S ends as
// the spectrum of the new state.  limit: polls a grid-barrier wait makes
// before it gives up (kFlagTimeout in *flag).
cudaError_t launch_persist(const Geom& g, const PersistFns& f, const LlgCoef& c, const float* Kd, float2* S,
                           float2* Sh, const float* Min, float* Mout, int n, int* flag, GridBar* gb, long long limit,
                           cudaStream_t s);
// Default poll limit of a grid-barrier wait (of the order of a second).
constexpr long long kGridWaitLimit = 1LL << 20;

// Thick-sample step / field: launch_fast_split with Kt, then the x-step
// kernel of mode `mode` in place on S (S -> S, M -> out).
cudaError_t launch_split_xstep(const Geom& g, const FastSplitFns& f2, const FastStepFns& fs, const LlgCoef& c,
                               int mode, const float* Kt, float2* S, const float* M, float* out, int* flag,
                               cudaStream_t s, float* Mcopy = nullptr);
cudaError_t launch_step_b(const Geom& g, const FastStepFns& f, const LlgCoef& c, const float2* Sh, float2* S,
                          const float* M, float* Mout, int* flag, cudaStream_t s, bool pdl, float* Mcopy = nullptr);

// Pass 2 for thick samples (split_kernels.cu); the spectrum row stride is Ly.
cudaError_t launch_split_plane(const Geom& g, float2* S, cudaStream_t s);
cudaError_t configure_split_kernels(const Geom& g);
size_t split_smem_y(const Geom& g);
size_t split_smem_z(const Geom& g);

// Runge-Kutta stage update (integrators.cu).  kind: 0 first stage, 1 middle
// stage, 2 last stage (writes the renormalised new state).
cudaError_t launch_rk_stage(int N, const LlgCoef& cf, float a_next, float b_acc, int kind, const float* Mst,
                            const float* H, const float* Mb, float* acc, float* out, int* flag, cudaStream_t s);

// Adaptive Dormand-Prince stages (integrators.cu).
struct DpPtrs {
    float* k[7];
};
struct DpWeights {
    float w[7];
};
cudaError_t launch_dp_combine(int N, const DpPtrs& kp, const DpWeights& w, int nk, float dt, const float* M,
                              float* out, cudaStream_t s);
cudaError_t launch_dp_stage(int N, const LlgCoef& cf, const DpPtrs& kp, int stage, const DpWeights& w, int renorm,
                            const float* Y, const float* H, const float* M, float* out, int* flag, cudaStream_t s);
cudaError_t launch_dp_error(int N, const LlgCoef& cf, const DpPtrs& kp, const DpWeights& e, const float* Y,
                            const float* H, float* k7out, unsigned* errbits, cudaStream_t s);

}  // namespace mmk
struct mm_fno;
namespace mmk {
// FNO surrogate (fno.cu): one-sample forward on a stream; grid check.
int fno_apply(mm_fno* f, const float* x, float* y, cudaStream_t s);
bool fno_matches(const mm_fno* f, int nx, int ny, int nz);

// Surrogate-assisted stepping (surrogate.cu).
cudaError_t sur_resid(const float* a, const float* b, long long n, double* out, cudaStream_t st);
// out = (a - b) / rms(a - b) (the sum of squares of a - b left in ss,
// device); and out = base + rms(a - b) y from that sum.
cudaError_t sur_unit_diff(const float* a, const float* b, long long n, double* ss, float* out, cudaStream_t st);
cudaError_t sur_rescale_add(const float* base, const float* y, const double* ss, long long n, float* out,
                            cudaStream_t st);
cudaError_t sur_llg(const Geom& g, const LlgCoef& cf, const float* M, const float* Hd, float* out, int* flag,
                    cudaStream_t st);

// Tensor set-up (tensor_setup.cu).  Writes N (FP64 octant) and/or Kt.
cudaError_t tensor_octant_fp64(const int grid[3], const double cell[3], double* N_dev, cudaStream_t s);
// Exchange stencil folded into the 2-D spectrum of the two-kernel step.
struct ExchangeFold {
    int on;
    int nx, ny, Lx, Ly;
    double pexch, idx2, idy2, idz2;
};
cudaError_t tensor_spectrum(const int grid[3], const int L[3], const double* N_dev, float* Kt_dev,
                            double* work1, double* work2, cudaStream_t s, float* Kd_dev = nullptr,
                            ExchangeFold ex = ExchangeFold{}, float* Kd0_dev = nullptr);
// Kt_ex = Kt plus the zero-padded 7-point exchange stencil's symbol on the
// diagonal (the 3-D counterpart of the fold into Kd).
cudaError_t tensor_fold_exchange3(const Geom& g, ExchangeFold ex, const float* Kt, float* Kt_ex, cudaStream_t s);
size_t tensor_work_elems(const int grid[3], const int L[3]);

// Energy (energy.cu): E[0..4] into out_dev (5 doubles, device); partials is
// device scratch of energy_partials_elems(N) doubles.
size_t energy_partials_elems(int N);
cudaError_t energy_reduce_full(const Geom& g, double Ms, const double Hext[3], const double cell[3], double A,
                               double Ku, const float* M, const float* Hd, double* partials, double* out_dev,
                               cudaStream_t s);

}  // namespace mmk
