// fast_x.cu -- instantiations of the power-of-two x passes (pass 1 and
// pass 3, three output modes) for nx = 16 ... 1024.
#include "fast_passes.cuh"

namespace mmk {

template <int N>
static void fill_x(FastFns* f) {
    constexpr int R1 = 8, R3 = 2;
    f->p1 = k_pass1_fast<N, R1>;
    f->r1 = R1;
    f->t1 = R1 * Fft2<N>::G;
    f->s1 = pass1_fast_smem<N, R1>();
    f->p3[kModeDemag] = k_pass3_fast<N, R3, kModeDemag>;
    f->p3[kModeHeff] = k_pass3_fast<N, R3, kModeHeff>;
    f->p3[kModeStep] = k_pass3_fast<N, R3, kModeStep>;
    f->r3 = R3;
    f->t3 = pass3_fast_threads<N, R3>();
    f->s3 = pass3_fast_smem<N, R3>();
}

bool fast_lookup_x(int nx, FastFns* f) {
    switch (nx) {
        case 16: fill_x<16>(f); return true;
        case 32: fill_x<32>(f); return true;
        case 64: fill_x<64>(f); return true;
        case 128: fill_x<128>(f); return true;
        case 256: fill_x<256>(f); return true;
        case 512: fill_x<512>(f); return true;
        case 1024: fill_x<1024>(f); return true;
        default: return false;
    }
}

}  // namespace mmk
