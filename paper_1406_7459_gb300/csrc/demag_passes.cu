// demag_passes.cu -- the three per-step kernels of the demag + LLG hot path.
//
// Pass 1  forward x R2C of Mx, My, Mz on the zero-padded length Lx; only the
//         first nx inputs of a row are nonzero (Sec. 2 step (1), Eq. (14)).
//         Two real rows ride in one complex transform.  Output: the
//         half-spectrum kx in [0, Lx/2] written kx-major into S.
// Pass 2  one CTA per kx plane: forward y FFT (ny nonzero inputs), forward
//         z FFT (nz nonzero inputs), the 3x3 product with the real symmetric
//         tensor spectrum (Eq. (13)/(15)), inverse z keeping k < nz, inverse
//         y keeping j < ny (Eq. (16), "discard the latter half").
// Pass 3  inverse x C2R keeping i < nx, then, per cell, H_demag joined with
//         the exchange stencil (Eq. (4), free boundaries), anisotropy
//         (Eq. (5), easy axis x), Zeeman, the LLG right-hand side (Eq. (6)),
//         a forward-Euler step and renormalisation |M| = Ms.  Modes write
//         H_demag, H_eff or M^{n+1}.
#include "pass_bodies.cuh"

namespace mmk {

__global__ void __launch_bounds__(256) k_pass1(Geom g, int R, int group, const float* __restrict__ M,
                                                float2* __restrict__ S) {
    pdl_wait();
    pass1_body(g, R, group, M, S, blockIdx.x);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_pass3(Geom g, int R, int group, LlgCoef cf,
                                                const float2* S, const float* __restrict__ M,
                                                float* __restrict__ out, int* __restrict__ flag) {
    pdl_wait();
    // kModeStepX writes the next step's x spectrum back over S
    pass3_body<MODE>(g, R, group, cf, S, M, out, flag, blockIdx.x,
                     MODE == kModeStepX ? const_cast<float2*>(S) : nullptr);
}

// -------------------------------------------------------------- launchers --
// Generic plane kernels exist for padded z lengths 1, 4, 5, 8, 9 (nz <= 5);
// thicker samples take the split y / z / y pass.
static PlaneFn plane_fn(int Lz) {
    PlaneFn f = plane_fn_small(Lz);
    if (!f) f = plane_fn_mid(Lz);
    return f;
}

bool plane_supported_lz(int Lz) { return plane_fn(Lz) != nullptr; }

cudaError_t configure_pass_kernels(const Geom& g, const Launch& l) {
    cudaError_t e;
    if (l.fx) {
        e = cudaFuncSetAttribute(l.fx->p1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fx->s1);
        for (int m = 0; m < 3 && e == cudaSuccess; ++m)
            e = cudaFuncSetAttribute(l.fx->p3[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fx->s3);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(k_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem1);
        if (e != cudaSuccess) return e;
        for (int m = 0; m < 4 && e == cudaSuccess; ++m)
            e = cudaFuncSetAttribute(m == 0   ? k_pass3<kModeDemag>
                                     : m == 1 ? k_pass3<kModeHeff>
                                     : m == 2 ? k_pass3<kModeStep>
                                              : k_pass3<kModeStepX>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem3);
        if (e != cudaSuccess) return e;
    }
    if (l.split && l.fs2) return configure_fast_split(*l.fs2);
    if (l.split) return configure_split_kernels(g);
    if (l.fp) return cudaFuncSetAttribute(l.fp->pl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.fp->s2);
    PlaneFn pf = plane_fn(g.Lz);
    if (!pf) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem2);
}
cudaError_t launch_pass1(const Geom& g, const Launch& l, const float* M, float2* S, cudaStream_t s, float* Mcopy) {
    if (l.fx) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = launch_config(dim3(3 * g.nz * (g.ny / l.fx->r1)), l.fx->t1, l.fx->s1, s, attr);
        return cudaLaunchKernelEx(&cfg, l.fx->p1, g, M, S, Mcopy);
    }
    if (Mcopy) return cudaErrorInvalidValue;      // the generic pass keeps no copy
    const int ntj = (g.ny + l.r1 - 1) / l.r1;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(3 * g.nz * ntj), l.t1, l.smem1, s, attr);
    return cudaLaunchKernelEx(&cfg, k_pass1, g, l.r1, l.g1, M, S);
}

cudaError_t launch_plane(const Geom& g, const Launch& l, float2* S, cudaStream_t s) {
    if (l.split && l.fs2) return launch_fast_split(g, *l.fs2, g.Kt, S, s);
    if (l.split) return launch_split_plane(g, S, s);
    if (l.fp) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = launch_config(dim3(g.Hx), l.fp->t2, l.fp->s2, s, attr);
        return cudaLaunchKernelEx(&cfg, l.fp->pl, g, S);
    }
    PlaneFn pf = plane_fn(g.Lz);
    if (!pf) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.Hx), l.t2, l.smem2, s, attr);
    return cudaLaunchKernelEx(&cfg, pf, g, l.g2, S);
}

cudaError_t launch_pass3(const Geom& g, const Launch& l, const LlgCoef& c, int mode, const float2* S,
                         const float* M, float* out, int* flag, cudaStream_t s) {
    if (l.fx) {
        if (mode == kModeStepX) return cudaErrorInvalidValue;      // generic kernels only
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / l.fx->r3)), l.fx->t3, l.fx->s3, s, attr);
        return cudaLaunchKernelEx(&cfg, l.fx->p3[mode], g, c, S, M, out, flag);
    }
    const int ntj = (g.ny + l.r3 - 1) / l.r3;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * ntj), l.t3, l.smem3, s, attr);
    switch (mode) {
        case kModeDemag: return cudaLaunchKernelEx(&cfg, k_pass3<kModeDemag>, g, l.r3, l.g3, c, S, M, out, flag);
        case kModeHeff: return cudaLaunchKernelEx(&cfg, k_pass3<kModeHeff>, g, l.r3, l.g3, c, S, M, out, flag);
        case kModeStepX: return cudaLaunchKernelEx(&cfg, k_pass3<kModeStepX>, g, l.r3, l.g3, c, S, M, out, flag);
        default: return cudaLaunchKernelEx(&cfg, k_pass3<kModeStep>, g, l.r3, l.g3, c, S, M, out, flag);
    }
}

}  // namespace mmk
