// Instantiations of the cooperative-block (strip pipeline) tiled-M polynomial-interpolation forward wavefront (float cell updates), orders 11..11 (one unit per group of orders so that the units compile in parallel).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* fwd_interp_coop_mt_ptr_f32_3(int N) {
    switch (N) {
        case 11: return reinterpret_cast<const void*>(&fwd_poly_kernel<float, 11, 11 + sk::kJF32, true, kCoopWarps, true>);
        default: return nullptr;
    }
}

}  // namespace sk
