// Instantiations of the cooperative-block (strip pipeline) polynomial-interpolation forward wavefront (float cell updates), orders 2..6 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_coop_ptr_f32_0(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 2, 2 + sk::kJF32, true, kCoopWarps, false>);
        case 3: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 3, 3 + sk::kJF32, true, kCoopWarps, false>);
        case 4: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 4, 4 + sk::kJF32, true, kCoopWarps, false>);
        case 5: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 5, 5 + sk::kJF32, true, kCoopWarps, false>);
        case 6: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 6, 6 + sk::kJF32, true, kCoopWarps, false>);
        default: return nullptr;
    }
}

}  // namespace sk
