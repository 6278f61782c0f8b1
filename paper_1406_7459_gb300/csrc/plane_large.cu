// plane_large.cu -- plane-kernel instantiations for padded z lengths 12, 15, 16.
#include "plane_kernel.cuh"

namespace mmk {

PlaneFn plane_fn_large(int Lz) {
    switch (Lz) {
        case 12: return k_plane<12>;
        case 15: return k_plane<15>;
        case 16: return k_plane<16>;
        default: return nullptr;
    }
}

}  // namespace mmk
