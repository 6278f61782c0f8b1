// plane_mid.cu -- plane-kernel instantiations for padded z lengths 8, 9.
#include "plane_kernel.cuh"

namespace mmk {

PlaneFn plane_fn_mid(int Lz) {
    switch (Lz) {
        case 8: return k_plane<8>;
        case 9: return k_plane<9>;
        default: return nullptr;
    }
}

}  // namespace mmk
