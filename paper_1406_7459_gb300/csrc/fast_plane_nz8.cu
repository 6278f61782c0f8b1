// fast_plane_nz8.cu -- instantiations of the power-of-two plane kernel
// (pass 2) for nz = 8, ny = 16, 32, 64, 128, 256.
#include "fast_passes.cuh"

namespace mmk {

template <int NY>
static void fill_plane(FastFns* f) {
    f->pl = k_plane_fast<NY, 8>;
    f->t2 = 6 * 8 * Fft2<NY>::G;
    f->s2 = plane_fast_smem<NY, 8>();
}

bool fast_lookup_plane_nz8(int ny, FastFns* f) {
    switch (ny) {
        case 16: fill_plane<16>(f); return true;
        case 32: fill_plane<32>(f); return true;
        case 64: fill_plane<64>(f); return true;
        case 128: fill_plane<128>(f); return true;
        case 256: fill_plane<256>(f); return true;
        default: return false;
    }
}

}  // namespace mmk
