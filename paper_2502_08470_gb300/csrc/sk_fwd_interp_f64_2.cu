// Instantiations of the polynomial-interpolation forward wavefront (double cell updates), orders 9..10 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_ptr_f64_2(int N) {
    switch (N) {
        case 9: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 9, 9 + sk::kJF64, true, 1, false>);
        case 10: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 10, 10 + sk::kJF64, true, 1, false>);
        default: return nullptr;
    }
}

}  // namespace sk
