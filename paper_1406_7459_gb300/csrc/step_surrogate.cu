// step_surrogate.cu -- mm_step_surrogate: Euler steps whose demag field
// comes from the FNO surrogate between exact refreshes (beyond the paper).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx_internal.h"

#define fail mmk::set_error_fmt

// ------------------------------------------------- surrogate-assisted step --
extern "C" int mm_step_surrogate(mm_ctx* c, mm_fno* f, int n, double dt, int refresh, double tol, double stats[4]) {
    if (!c || !f) return fail(MM_EINVAL, "null context or surrogate");
    if (n < 0 || refresh < 1 || !(dt > 0.0) || !(tol > 0.0)) return fail(MM_EINVAL, "bad n, refresh, dt or tol");
    if (!fno_matches(f, c->g.nx, c->g.ny, c->g.nz))
        return fail(MM_EINVAL, "surrogate grid does not match the film (nz must be 1)");
    const size_t N3 = 3 * (size_t)c->g.N;
    if (!c->sur) {
        CU(cudaMalloc(&c->sur, sizeof(float) * 5 * N3));
        CU(cudaMalloc(&c->sur_r, 3 * sizeof(double)));
    }
    float *Mref = c->sur, *Href = c->sur + N3, *x = c->sur + 2 * N3, *y = c->sur + 3 * N3, *Hd = c->sur + 4 * N3;
    const LlgCoef cf = make_coef(c, dt);
    double n_sur = 0, n_exact = 0, max_res = 0;
    bool fallback = false, have_ref = false;
    for (int s = 0; s < n; ++s) {
        const int p = c->cur;
        if (s % refresh == 0 || fallback) {
            int rc = run_passes(c, kModeDemag, c->Mbuf[p], Hd, 0.0, c->stream);
            if (rc != MM_OK) return rc;
            if (have_ref && !fallback) {
                // surrogate's prediction at this state against the exact field
                CU(sur_unit_diff(c->Mbuf[p], Mref, (long long)N3, c->sur_r + 2, x, c->stream));
                rc = fno_apply(f, x, y, c->stream);
                if (rc != MM_OK) return rc;
                CU(sur_rescale_add(Href, y, c->sur_r + 2, (long long)N3, x, c->stream));
                CU(sur_resid(x, Hd, (long long)N3, c->sur_r, c->stream));
                double r[2];
                CU(cudaMemcpyAsync(r, c->sur_r, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
                CU(cudaStreamSynchronize(c->stream));
                const double res = r[1] > 0 ? std::sqrt(r[0] / r[1]) : 0.0;
                if (res > max_res) max_res = res;
                if (res > tol) fallback = true;
            }
            CU(cudaMemcpyAsync(Mref, c->Mbuf[p], sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream));
            CU(cudaMemcpyAsync(Href, Hd, sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream));
            have_ref = true;
            n_exact += 1;
        } else {
            CU(sur_unit_diff(c->Mbuf[p], Mref, (long long)N3, c->sur_r + 2, x, c->stream));
            int rc = fno_apply(f, x, y, c->stream);
            if (rc != MM_OK) return rc;
            CU(sur_rescale_add(Href, y, c->sur_r + 2, (long long)N3, Hd, c->stream));
            n_sur += 1;
        }
        CU(sur_llg(c->g, cf, c->Mbuf[p], Hd, c->Mbuf[1 - p], c->flag, c->stream));
        c->cur = 1 - p;
    }
    c->spec_valid = false;
    if (stats) {
        stats[0] = n_sur;
        stats[1] = n_exact;
        stats[2] = max_res;
        stats[3] = fallback ? 1.0 : 0.0;
    }
    return MM_OK;
}
