// Instantiations of the tape adjoint of the polynomial-interpolation scheme (double cell updates, orders 9..12 (units split so that they compile in parallel)).
#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* bwd_tape_interp_ptr_f64_1(int N) {
    switch (N) {
        case 9: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 9, true>);
        case 10: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 10, true>);
        case 11: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 11, true>);
        case 12: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 12, true>);
        default: return nullptr;
    }
}

const void* bwd_tape_interp_ptr_f64(int N) {
    if (const void* k = bwd_tape_interp_ptr_f64_0(N)) return k;
    return bwd_tape_interp_ptr_f64_1(N);
}

}  // namespace sk
