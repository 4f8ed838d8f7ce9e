// Instantiations of the approximation-scheme forward wavefront that records the tape of output
// derivatives (float cell updates; the orders bwd_tape_kernel supports) and reads M from the buffer
// written by the tensor-core M kernel.
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

template <int N>
const void* tape_mx_kernel() {
    return reinterpret_cast<const void*>(&fwd_poly_kernel<float, N, N, false, 1, false, true, true>);
}

const void* fwd_approx_tape_mx_ptr_f32(int N) {
    switch (N) {
        case 2: return tape_mx_kernel<2>();
        case 3: return tape_mx_kernel<3>();
        case 4: return tape_mx_kernel<4>();
        case 5: return tape_mx_kernel<5>();
        case 6: return tape_mx_kernel<6>();
        case 7: return tape_mx_kernel<7>();
        case 8: return tape_mx_kernel<8>();
        case 9: return tape_mx_kernel<9>();
        case 10: return tape_mx_kernel<10>();
        case 12: return tape_mx_kernel<12>();
        default: return nullptr;
    }
}

}  // namespace sk
