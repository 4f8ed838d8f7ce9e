// Instantiations of the polynomial-interpolation forward wavefront (double cell updates), orders 12..12 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_ptr_f64_4(int N) {
    switch (N) {
        case 12: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 12, 12 + sk::kJF64, true, 1, false>);
        default: return nullptr;
    }
}

}  // namespace sk
