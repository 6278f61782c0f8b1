// ctx_internal.h -- the solver context behind the C ABI, shared by the
// translation units that implement include/mm.h (mm_api.cu, adaptive.cu,
// step_surrogate.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/mm.h"
#include "mm_internal.h"

namespace mmk {

// Record a message for mm_last_error() and return `code`.
int set_error_fmt(int code, const char* fmt, ...);

}  // namespace mmk

#define CU(expr)                                                                               \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return mmk::set_error_fmt(_e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA,   \
                                      "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                                      __LINE__);                                               \
    } while (0)

// internal header of the ABI translation units: the kernels' types unqualified
using namespace mmk;

struct mm_ctx {
    int grid[3];
    double cell[3];
    double Ms, A, Ku, alpha, gamma;
    double Hext[3];
    cudaStream_t stream;
    cudaStream_t cap;          // private stream used only for graph capture
    int device;
    Geom g;
    Launch l;
    float* Kt = nullptr;
    float* Kd = nullptr;       // 2-D spectrum per z offset, exchange folded in (two-kernel step)
    float* Kd0 = nullptr;      // the same without exchange (two-kernel demag evaluation)
    float2* S = nullptr;
    float* Mbuf[2] = {nullptr, nullptr};
    int cur = 0;
    float* H = nullptr;
    int* flag = nullptr;
    double* partials = nullptr;
    double* Edev = nullptr;
    float2* tw = nullptr;      // twiddles of x, y, z back to back
    // step graphs [kind][parity]: kind 0 one step, kind 1 kGraphSteps steps
    cudaGraphExec_t step_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double step_dt[2][2] = {{0, 0}, {0, 0}};
    unsigned long long step_ver[2][2] = {{0, 0}, {0, 0}};
    unsigned long long ver = 1;   // bumped when H_ext changes
    bool use_graphs = true;
    FastFns fast;              // compile-time kernels (when the grid has them)
    FastStepFns fs;            // two-kernel step (power-of-two grids)
    FastSplitFns fsplit;       // compile-time split pass 2 (thick power-of-two samples)
    bool has_fs = false;
    bool has_ss = false;       // thick power-of-two samples: split pass 2 + the x-step kernel
    bool has_gx = false;       // generic x passes: the step's pass 3 also forms the next x spectrum
    float* Kt_ex = nullptr;    // tensor spectrum with the exchange stencil folded in (has_ss)
    float2* Sh = nullptr;      // plane-kernel output of the two-kernel step (layout of S)
    int method = MM_INTEGRATOR_EULER;
    float* Mst = nullptr;      // Runge-Kutta stage state
    float* acc = nullptr;      // Runge-Kutta weighted slope sum
    float* sur = nullptr;      // surrogate stepper: M_ref, H_ref, x, y, H_d (5 x 3N)
    double* sur_r = nullptr;   // residual sums
    bool spec_valid = false;   // S holds the x half-spectrum of M[cur] (two-kernel step)
    float* dpk[7] = {};        // Dormand-Prince stage slopes (adaptive runs), 3*N each
    unsigned* dperr = nullptr; // error estimate of the last trial step (float bits)
    PersistFns pf;             // persistent step (square power-of-two films it is built for)
    bool has_persist = false;  // the persistent step fits this grid and device
    int step_path = MM_STEP_AUTO;
    long long wait_limit = kGridWaitLimit;   // polls of a grid-barrier wait
    GridBar* gbar = nullptr;   // grid-barrier counters of the persistent step
};

namespace mmk {

// Field and LLG coefficients of the context for a step of size dt.
LlgCoef make_coef(const mm_ctx* c, double dt);
// x R2C, plane, x C2R (+ field / step per mode) of M into out on stream s;
// invalidates a pending step spectrum.
int run_passes(mm_ctx* c, int mode, const float* M, float* out, double dt, cudaStream_t s);

}  // namespace mmk
