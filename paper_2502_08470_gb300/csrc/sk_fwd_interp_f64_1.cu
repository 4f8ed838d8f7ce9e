// Instantiations of the polynomial-interpolation forward wavefront (double cell updates), orders 7..8 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_ptr_f64_1(int N) {
    switch (N) {
        case 7: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 7, 7 + sk::kJF64, true, 1, false>);
        case 8: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 8, 8 + sk::kJF64, true, 1, false>);
        default: return nullptr;
    }
}

}  // namespace sk
