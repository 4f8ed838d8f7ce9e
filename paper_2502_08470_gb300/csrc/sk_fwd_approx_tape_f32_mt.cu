// Instantiations of the approximation-scheme forward wavefront that records the tape of output
// derivatives read by the tape adjoint (float cell updates, tiled M; the orders bwd_tape_kernel supports).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_approx_tape_ptr_f32_mt(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 2, 2, false, 1, true, true>);
        case 3: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 3, 3, false, 1, true, true>);
        case 4: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 4, 4, false, 1, true, true>);
        case 5: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 5, 5, false, 1, true, true>);
        case 6: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 6, 6, false, 1, true, true>);
        case 7: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 7, 7, false, 1, true, true>);
        case 8: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 8, 8, false, 1, true, true>);
        case 9: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 9, 9, false, 1, true, true>);
        case 10: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 10, 10, false, 1, true, true>);
        case 12: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 12, 12, false, 1, true, true>);
        default: return nullptr;
    }
}

}  // namespace sk
