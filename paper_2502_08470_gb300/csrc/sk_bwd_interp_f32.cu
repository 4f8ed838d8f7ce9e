// Instantiations of the tape adjoint of the polynomial-interpolation scheme (float cell updates).
#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* bwd_tape_interp_ptr_f32(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 2, true>);
        case 3: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 3, true>);
        case 4: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 4, true>);
        case 5: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 5, true>);
        case 6: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 6, true>);
        case 7: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 7, true>);
        case 8: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 8, true>);
        case 9: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 9, true>);
        case 10: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 10, true>);
        case 11: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 11, true>);
        case 12: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 12, true>);
        default: return nullptr;
    }
}

}  // namespace sk
