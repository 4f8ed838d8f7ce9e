// Instantiations of the cooperative-block (strip pipeline) polynomial-interpolation forward wavefront (float cell updates), orders 7..8 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_coop_ptr_f32_1(int N) {
    switch (N) {
        case 7: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 7, 7 + sk::kJF32, true, kCoopWarps, false>);
        case 8: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 8, 8 + sk::kJF32, true, kCoopWarps, false>);
        default: return nullptr;
    }
}

}  // namespace sk
