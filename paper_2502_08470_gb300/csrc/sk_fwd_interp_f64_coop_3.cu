// Instantiations of the cooperative-block (strip pipeline) polynomial-interpolation forward wavefront (double cell updates), orders 11..11 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_coop_ptr_f64_3(int N) {
    switch (N) {
        case 11: return reinterpret_cast<const void*>(&fwd_poly_kernel<double, 11, 11 + sk::kJF64, true, kCoopWarps, false>);
        default: return nullptr;
    }
}

}  // namespace sk
