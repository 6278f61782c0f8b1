// adaptive.cu -- mm_run_adaptive: Eq. (6) integrated with the embedded
// Dormand-Prince RK5(4) pair and step-size control (beyond the paper, whose
// scheme is forward Euler).  Stage kernels in integrators.cu; the controller
// runs here on the host on the GPU's error estimate.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx_internal.h"

#define fail mmk::set_error_fmt

// ------------------------------------------------ adaptive Dormand-Prince --
// Dormand-Prince RK5(4) (Dormand and Prince, J. Comput. Appl. Math. 6 (1980)
// 19-26): stage rows a (row s forms stage s + 1), fifth-order weights b and
// e = b - b_hat, b_hat the embedded fourth-order weights.
static const double kDpA[6][6] = {
    {0.0},
    {1.0 / 5.0},
    {3.0 / 40.0, 9.0 / 40.0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0}};
static const double kDpB[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double kDpE[7] = {71.0 / 57600.0,      0.0,          -71.0 / 16695.0, 71.0 / 1920.0,
                               -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};
// Controller: accept when err <= tol; next step h * clamp(0.9 (tol/err)^(1/5),
// 0.2, 5), no growth right after a rejection.
static double dp_factor(double err, double tol, bool after_reject) {
    double fac = err <= 0.0 ? 5.0 : 0.9 * std::pow(tol / err, 0.2);
    fac = std::min(5.0, std::max(0.2, fac));
    return after_reject ? std::min(fac, 1.0) : fac;
}

static DpWeights dp_row(const double* w, int n) {
    DpWeights r{};
    for (int j = 0; j < n; ++j) r.w[j] = (float)w[j];
    return r;
}

extern "C" int mm_run_adaptive(mm_ctx* c, double t_span, double* dt_io, double tol, int max_steps,
                               double stats[4]) {
    if (!c || !dt_io) return fail(MM_EINVAL, "null argument");
    if (!(t_span >= 0.0) || !std::isfinite(t_span)) return fail(MM_EINVAL, "t_span must be finite and >= 0");
    if (!(*dt_io > 0.0) || !std::isfinite(*dt_io)) return fail(MM_EINVAL, "dt must be > 0");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(MM_EINVAL, "tol must be > 0");
    if (max_steps < 1) return fail(MM_EINVAL, "max_steps must be >= 1");
    const size_t n3 = 3 * (size_t)c->g.N;
    if (!c->Mst) CU(cudaMalloc(&c->Mst, sizeof(float) * n3));
    for (int q = 0; q < 7; ++q)
        if (!c->dpk[q]) CU(cudaMalloc(&c->dpk[q], sizeof(float) * n3));
    if (!c->dperr) CU(cudaMalloc(&c->dperr, sizeof(unsigned)));
    cudaStream_t s = c->stream;
    DpPtrs kp;
    for (int q = 0; q < 7; ++q) kp.k[q] = c->dpk[q];
    const DpWeights we = dp_row(kDpE, 7);
    double t = 0.0, dt = *dt_io;
    long long acc = 0, rej = 0, nev = 0;
    bool after_reject = false, k1_valid = false;
    int rc = MM_OK;
    c->spec_valid = false;
    while (t_span - t > 1e-12 * t_span && acc + rej < max_steps) {
        const int p = c->cur;
        const double h = std::min(dt, t_span - t);
        const LlgCoef cf = make_coef(c, h);
        const float* M = c->Mbuf[p];
        float* cand = c->Mbuf[1 - p];
        // stage 2 state (and k1 = f(M) on the first step; later k1 is the
        // previous step's seventh stage)
        if (!k1_valid) {
            rc = run_passes(c, kModeHeff, M, c->H, 0.0, s);
            if (rc != MM_OK) return rc;
            CU(launch_dp_stage(c->g.N, cf, kp, 1, dp_row(kDpA[1], 1), 0, M, c->H, M, c->Mst, nullptr, s));
            nev += 1;
            k1_valid = true;
        } else {
            CU(launch_dp_combine(c->g.N, kp, dp_row(kDpA[1], 1), 1, (float)h, M, c->Mst, s));
        }
        for (int st = 2; st <= 6; ++st) {
            rc = run_passes(c, kModeHeff, c->Mst, c->H, 0.0, s);
            if (rc != MM_OK) return rc;
            const bool last = st == 6;
            const DpWeights w = last ? dp_row(kDpB, 6) : dp_row(kDpA[st], st);
            CU(launch_dp_stage(c->g.N, cf, kp, st, w, last ? 1 : 0, c->Mst, c->H, M, last ? cand : c->Mst, nullptr,
                               s));
        }
        rc = run_passes(c, kModeHeff, cand, c->H, 0.0, s);
        if (rc != MM_OK) return rc;
        CU(cudaMemsetAsync(c->dperr, 0, sizeof(unsigned), s));
        CU(launch_dp_error(c->g.N, cf, kp, we, cand, c->H, kp.k[6], c->dperr, s));
        unsigned bits = 0;
        CU(cudaMemcpyAsync(&bits, c->dperr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        nev += 6;
        float errf;
        std::memcpy(&errf, &bits, sizeof(float));
        const double err = (double)errf;
        if (err <= tol) {
            t += h;
            c->cur = 1 - p;
            std::swap(kp.k[0], kp.k[6]);
            ++acc;
            dt = h * dp_factor(err, tol, after_reject);
            after_reject = false;
        } else {
            ++rej;
            dt = h * dp_factor(std::isfinite(err) ? err : 1e300, tol, true);
            after_reject = true;
        }
    }
    for (int q = 0; q < 7; ++q) c->dpk[q] = kp.k[q];
    *dt_io = dt;
    if (stats) {
        stats[0] = (double)acc;
        stats[1] = (double)rej;
        stats[2] = (double)nev;
        stats[3] = t;
    }
    if (t_span - t > 1e-12 * t_span) return fail(MM_ELIMIT, "max_steps reached before t_span was covered");
    return MM_OK;
}

