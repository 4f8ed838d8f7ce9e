// Instantiations of the cooperative-block (strip pipeline) polynomial-approximation forward wavefront (float cell updates).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_approx_coop_ptr_f32(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 2, 2, false, kCoopWarps, false>);
        case 3: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 3, 3, false, kCoopWarps, false>);
        case 4: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 4, 4, false, kCoopWarps, false>);
        case 5: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 5, 5, false, kCoopWarps, false>);
        case 6: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 6, 6, false, kCoopWarps, false>);
        case 7: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 7, 7, false, kCoopWarps, false>);
        case 8: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 8, 8, false, kCoopWarps, false>);
        case 9: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 9, 9, false, kCoopWarps, false>);
        case 10: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 10, 10, false, kCoopWarps, false>);
        case 11: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 11, 11, false, kCoopWarps, false>);
        case 12: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 12, 12, false, kCoopWarps, false>);
        case 13: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 13, 13, false, kCoopWarps, false>);
        case 14: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 14, 14, false, kCoopWarps, false>);
        case 15: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 15, 15, false, kCoopWarps, false>);
        case 16: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 16, 16, false, kCoopWarps, false>);
        default: return nullptr;
    }
}

}  // namespace sk
