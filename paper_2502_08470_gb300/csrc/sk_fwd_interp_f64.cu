// Instantiations of the polynomial-interpolation forward wavefront (double cell updates).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_ptr_f64(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 2, 2 + sk::kJF64, true>);
        case 3: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 3, 3 + sk::kJF64, true>);
        case 4: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 4, 4 + sk::kJF64, true>);
        case 5: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 5, 5 + sk::kJF64, true>);
        case 6: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 6, 6 + sk::kJF64, true>);
        case 7: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 7, 7 + sk::kJF64, true>);
        case 8: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 8, 8 + sk::kJF64, true>);
        case 9: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 9, 9 + sk::kJF64, true>);
        case 10: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 10, 10 + sk::kJF64, true>);
        case 11: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 11, 11 + sk::kJF64, true>);
        case 12: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 12, 12 + sk::kJF64, true>);
        default: return nullptr;
    }
}

}  // namespace sk
