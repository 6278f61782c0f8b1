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
    if constexpr (XstepLayout<N, R>::HM <= 256) {      // the box's kx / 2 extent
        f->kbt[kModeDemag] = k_xstep_tma<N, R, kModeDemag>;
        f->kbt[kModeHeff] = k_xstep_tma<N, R, kModeHeff>;
        f->kbt[kModeStep] = k_xstep_tma<N, R, kModeStep>;
    }
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
    for (int m = 0; m < 3 && e == cudaSuccess; ++m) {
        e = cudaFuncSetAttribute(f.kb[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sb);
        if (e == cudaSuccess && f.kbt[m])
            e = cudaFuncSetAttribute(f.kbt[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.sb);
    }
    return e;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tiled_encoder() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The spectrum as a 4-D float array for the x-step tiles: dimension 0 the
// floats of the (k, j) rows of one (kx, c) line (contiguous, 2 nz Jst),
// 1 m = kx / 2 (HM values), 2 the parity of kx, 3 the component c.  A
// tile's box is 2R floats (rows j0 .. j0 + R - 1 of layer k) of every
// (m, parity, c): 3 * 2 * HM runs of 8R bytes, landing in shared memory as
// [c][parity][m][2R floats].  Whether the kernels use the maps is
// f->tma_use (mm_set_tiled_copies); by default they keep the per-thread
// 16-byte copies and plain stores, which measured faster on the 256 x 256 x 4
// film (24.5-24.7 against 25.2-25.5 us per flushed step: one thread's box of
// 772 rows of 32 bytes against 192 threads' requests in flight).
bool encode_xstep_maps(const Geom& g, FastStepFns* f, const float2* Sh, const float2* S) {
    f->tma = false;
    const int R = f->rb;
    const int HM = g.nx / 2 + 1;
    EncodeTiledFn enc = tiled_encoder();
    if (!enc || !f->kbt[kModeStep] || HM > 256 || g.Hx != g.nx + 1 || (2LL * g.nz * g.Jst) % 4 != 0) return false;
    const cuuint64_t s_c = (cuuint64_t)g.nz * g.Jst * sizeof(float2), s_kx = 3 * s_c;
    const cuuint64_t dims[4] = {(cuuint64_t)2 * g.nz * g.Jst, (cuuint64_t)HM, 2, 3};
    const cuuint64_t strides[3] = {2 * s_kx, s_kx, s_c};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * R), (cuuint32_t)HM, 2, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int i = 0; i < 2; ++i) {
        CUtensorMap* m = i == 0 ? &f->tin : &f->tout;
        void* base = const_cast<float2*>(i == 0 ? Sh : S);
        if (enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    f->tin_buf = Sh;
    f->tout_buf = S;
    f->tma = true;
    return true;
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
    if (f.tma && f.tma_use && Sh == f.tin_buf && S == f.tout_buf)
        return cudaLaunchKernelEx(&cfg, f.kbt[kModeStep], g, c, Sh, S, M, Mout, flag, Mcopy, f.tin, f.tout,
                                  f.tma_use);
    return cudaLaunchKernelEx(&cfg, f.kb[kModeStep], g, c, Sh, S, M, Mout, flag, Mcopy);
}

cudaError_t launch_field_pdl(const Geom& g, const FastStepFns& f, const LlgCoef& c, int mode, const float* Kd,
                             float2* S, float2* Sh, const float* M, float* out, int* flag, cudaStream_t s) {
    cudaError_t e = launch_step_a(g, f, Kd, S, Sh, flag, s, true, 0);   // late: measured faster here
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(dim3(g.nz * (g.ny / f.rb)), f.tb, f.sb, s, attr, true);
    if (f.tma && f.tma_use && Sh == f.tin_buf)
        return cudaLaunchKernelEx(&cfg, f.kbt[mode], g, c, (const float2*)Sh, (float2*)nullptr, M, out, flag,
                                  (float*)nullptr, f.tin, f.tout, f.tma_use);
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
