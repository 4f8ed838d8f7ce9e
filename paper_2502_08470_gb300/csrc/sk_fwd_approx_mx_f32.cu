// Instantiations of the polynomial-approximation forward wavefront whose cells read M from the
// buffer written by the tensor-core M kernel (float cell updates, one warp per pair).
#include "sk_fwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

template <int N>
const void* mx_kernel() {
    return reinterpret_cast<const void*>(&fwd_poly_kernel<float, N, N, false, 1, false, false, true>);
}

const void* fwd_approx_mx_ptr_f32(int N) {
    switch (N) {
        case 2: return mx_kernel<2>();
        case 3: return mx_kernel<3>();
        case 4: return mx_kernel<4>();
        case 5: return mx_kernel<5>();
        case 6: return mx_kernel<6>();
        case 7: return mx_kernel<7>();
        case 8: return mx_kernel<8>();
        case 9: return mx_kernel<9>();
        case 10: return mx_kernel<10>();
        case 11: return mx_kernel<11>();
        case 12: return mx_kernel<12>();
        case 13: return mx_kernel<13>();
        case 14: return mx_kernel<14>();
        case 15: return mx_kernel<15>();
        case 16: return mx_kernel<16>();
        default: return nullptr;
    }
}

}  // namespace sk
