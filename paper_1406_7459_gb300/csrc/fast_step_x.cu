// fast_step_x.cu -- instantiations of the fused inverse-x + LLG + forward-x
// kernel (second kernel of the power-of-two step) for nx = 16 ... 1024, and
// of its field-only variants (H_demag, H_eff) that close the two-kernel
// field evaluation.
#include <cstdlib>

#include "fast_step.cuh"

namespace mmk {

template <int N>
static void fill_xstep(FastStepFns* f) {
    // four-row tiles where their shared memory fits comfortably, else two
    constexpr int R = XstepLayout<N, kStepRows>::BYTES <= 200 * 1024 ? kStepRows : 2;
    f->kb[kModeDemag] = k_xstep_pdl<N, R, kModeDemag>;
    f->kb[kModeHeff] = k_xstep_pdl<N, R, kModeHeff>;
    f->kb[kModeStep] = k_xstep_pdl<N, R, kModeStep>;
    f->rb = R;
    f->tb = XstepLayout<N, R>::THREADS;
    f->sb = XstepLayout<N, R>::BYTES;
}

bool fast_step_lookup_x(int nx, FastStepFns* f) {
    switch (nx) {
        case 16: fill_xstep<16>(f); return true;
        case 32: fill_xstep<32>(f); return true;
        case 64: fill_xstep<64>(f); return true;
        case 128: fill_xstep<128>(f); return true;
        case 256: fill_xstep<256>(f); return true;
        case 512: fill_xstep<512>(f); return true;
        case 1024: fill_xstep<1024>(f); return true;
        default: return false;
    }
}

}  // namespace mmk

namespace mmk {

// Early trigger for the step where the plane grid already covers every SM
// (Hx > SMs): the x-step blocks that start early then sit beside single
// plane blocks (measured per flushed step: 64x64x4 11.1 vs 11.9 us late,
// 128x128x4 19.2 vs 15.4, 256x256x4 25.4 vs 25.4, 1024x1024x1 90.8 vs 92.9;
// the field evaluations keep the late trigger, 23.2 vs 25.0 us at 256).
// MM_EARLY_TRIGGER=0/1 overrides the choice (for measurements).
int fast_step_early_trigger(const Geom& g, int sms) {
    const char* e = getenv("MM_EARLY_TRIGGER");
    if (e && (e[0] == '0' || e[0] == '1') && e[1] == 0) return e[0] == '1';
    return g.Hx > sms ? 1 : 0;
}

cudaError_t configure_step_kernels(const FastStepFns& f) {
    cudaError_t e = f.ka ? cudaFuncSetAttribute(f.ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sa)
                         : cudaSuccess;                   // x-step only (thick samples)
    for (int m = 0; m < 3 && e == cudaSuccess; ++m)
        e = cudaFuncSetAttribute(f.kb[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sb);
    return e;
}

cudaError_t launch_step_a(const Geom& g, const FastStepFns& f, const float* Kd, const float2* S, float2* Sh,
                          int* flag, cudaStream_t s, bool pdl, int early) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.Hx), f.ta, f.sa, s, attr, pdl);
    return cudaLaunchKernelEx(&cfg, f.ka, g, Kd, S, Sh, flag, early);
}

cudaError_t launch_step_b(const Geom& g, const FastStepFns& f, const LlgCoef& c, const float2* Sh, float2* S,
                          const float* M, float* Mout, int* flag, cudaStream_t s, bool pdl, float* Mcopy) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / f.rb)), f.tb, f.sb, s, attr, pdl);
    return cudaLaunchKernelEx(&cfg, f.kb[kModeStep], g, c, Sh, S, M, Mout, flag, Mcopy);
}

cudaError_t launch_field_pdl(const Geom& g, const FastStepFns& f, const LlgCoef& c, int mode, const float* Kd,
                             float2* S, float2* Sh, const float* M, float* out, int* flag, cudaStream_t s) {
    cudaError_t e = launch_step_a(g, f, Kd, S, Sh, flag, s, true, 0);   // late: measured faster here
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / f.rb)), f.tb, f.sb, s, attr, true);
    return cudaLaunchKernelEx(&cfg, f.kb[mode], g, c, (const float2*)Sh, (float2*)nullptr, M, out, (int*)nullptr,
                              (float*)nullptr);
}

// K_A then K_B; with `pdl` both carry the programmatic-serialisation launch
// attribute so each may start while its predecessor drains (each kernel
// waits on griddepcontrol before reading what the predecessor wrote).
cudaError_t launch_step_pdl(const Geom& g, const FastStepFns& f, const LlgCoef& c, float2* S, float2* Sh,
                            const float* M, float* Mout, int* flag, cudaStream_t s, bool pdl, float* Mcopy) {
    cudaError_t e = launch_step_a(g, f, g.Kd, S, Sh, flag, s, pdl, f.early);
    if (e != cudaSuccess) return e;
    return launch_step_b(g, f, c, Sh, S, M, Mout, flag, s, pdl, Mcopy);
}

}  // namespace mmk
