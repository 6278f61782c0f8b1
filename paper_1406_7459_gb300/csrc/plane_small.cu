// plane_small.cu -- plane-kernel instantiations for padded z lengths 1, 4, 5.
#include "plane_kernel.cuh"

namespace mmk {

PlaneFn plane_fn_small(int Lz) {
    switch (Lz) {
        case 1: return k_plane<1>;
        case 4: return k_plane<4>;
        case 5: return k_plane<5>;
        default: return nullptr;
    }
}

}  // namespace mmk
