// fast_step_plane_a.cu -- instantiations of the PDL plane kernel (first
// kernel of the power-of-two step) for nz in {1, 2}.
#include "fast_step.cuh"

namespace mmk {

template <int NY, int NZ>
static void fill_plane_pdl(FastStepFns* f) {
    f->ka = k_plane_pdl<NY, NZ>;
    f->ta = PlaneLayout<NY, NZ>::THREADS;
    f->sa = PlaneLayout<NY, NZ>::BYTES;
}

bool fast_step_lookup_plane_a(int ny, int nz, FastStepFns* f) {
    if (nz == 1) {
        switch (ny) {
            case 16: fill_plane_pdl<16, 1>(f); return true;
            case 32: fill_plane_pdl<32, 1>(f); return true;
            case 64: fill_plane_pdl<64, 1>(f); return true;
            case 128: fill_plane_pdl<128, 1>(f); return true;
            case 256: fill_plane_pdl<256, 1>(f); return true;
            case 512: fill_plane_pdl<512, 1>(f); return true;
            case 1024: fill_plane_pdl<1024, 1>(f); return true;
            default: return false;
        }
    }
    if (nz == 2) {
        switch (ny) {
            case 16: fill_plane_pdl<16, 2>(f); return true;
            case 32: fill_plane_pdl<32, 2>(f); return true;
            case 64: fill_plane_pdl<64, 2>(f); return true;
            case 128: fill_plane_pdl<128, 2>(f); return true;
            case 256: fill_plane_pdl<256, 2>(f); return true;
            case 512: fill_plane_pdl<512, 2>(f); return true;
            case 1024: fill_plane_pdl<1024, 2>(f); return true;
            default: return false;
        }
    }
    return false;
}

}  // namespace mmk
