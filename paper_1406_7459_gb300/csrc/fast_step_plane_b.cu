// fast_step_plane_b.cu -- instantiations of the PDL plane kernel (first
// kernel of the power-of-two step) for nz in {4, 8}.
#include "fast_step.cuh"

namespace mmk {

template <int NY, int NZ>
static void fill_plane_pdl(FastStepFns* f) {
    f->ka = k_plane_pdl<NY, NZ>;
    f->ta = PlaneLayout<NY, NZ>::THREADS;
    f->sa = PlaneLayout<NY, NZ>::BYTES;
}

bool fast_step_lookup_plane_b(int ny, int nz, FastStepFns* f) {
    if (nz == 4) {
        switch (ny) {
            case 16: fill_plane_pdl<16, 4>(f); return true;
            case 32: fill_plane_pdl<32, 4>(f); return true;
            case 64: fill_plane_pdl<64, 4>(f); return true;
            case 128: fill_plane_pdl<128, 4>(f); return true;
            case 256: fill_plane_pdl<256, 4>(f); return true;
            case 512: fill_plane_pdl<512, 4>(f); return true;
            default: return false;
        }
    }
    if (nz == 8) {
        switch (ny) {
            case 16: fill_plane_pdl<16, 8>(f); return true;
            case 32: fill_plane_pdl<32, 8>(f); return true;
            case 64: fill_plane_pdl<64, 8>(f); return true;
            case 128: fill_plane_pdl<128, 8>(f); return true;
            case 256: fill_plane_pdl<256, 8>(f); return true;
            default: return false;
        }
    }
    return false;
}

}  // namespace mmk
