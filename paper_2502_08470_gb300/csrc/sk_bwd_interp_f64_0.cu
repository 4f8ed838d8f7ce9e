// Instantiations of the tape adjoint of the polynomial-interpolation scheme (double cell updates, orders 2..8 (units split so that they compile in parallel)).
#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* bwd_tape_interp_ptr_f64_0(int N) {
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 2, true>);
        case 3: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 3, true>);
        case 4: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 4, true>);
        case 5: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 5, true>);
        case 6: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 6, true>);
        case 7: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 7, true>);
        case 8: return reinterpret_cast<const void*>(&bwd_tape_kernel<double, 8, true>);
        default: return nullptr;
    }
}

}  // namespace sk
