// Instantiations of the approximation-scheme adjoint wavefronts (float cell updates): the
// checkpointing form, the tape-driven form and the dk/dM contraction.
#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"

namespace sk {

const void* bwd_approx_ptr_f32(int N, int dmax, int* stack_bytes) {
    if (dmax == 8) switch (N) {
        case 2: *stack_bytes = bwd_stack_bytes<float, 2, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 2, 4, 8>);
        case 3: *stack_bytes = bwd_stack_bytes<float, 3, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 3, 4, 8>);
        case 4: *stack_bytes = bwd_stack_bytes<float, 4, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 4, 4, 8>);
        case 5: *stack_bytes = bwd_stack_bytes<float, 5, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 5, 4, 8>);
        case 6: *stack_bytes = bwd_stack_bytes<float, 6, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 6, 4, 8>);
        case 7: *stack_bytes = bwd_stack_bytes<float, 7, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 7, 4, 8>);
        case 8: *stack_bytes = bwd_stack_bytes<float, 8, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 8, 4, 8>);
        case 9: *stack_bytes = bwd_stack_bytes<float, 9, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 9, 4, 8>);
        case 10: *stack_bytes = bwd_stack_bytes<float, 10, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 10, 4, 8>);
        case 12: *stack_bytes = bwd_stack_bytes<float, 12, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 12, 4, 8>);
        default: break;
    }
    if (dmax == 32) switch (N) {
        case 2: *stack_bytes = bwd_stack_bytes<float, 2, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 2, 4, 32>);
        case 3: *stack_bytes = bwd_stack_bytes<float, 3, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 3, 4, 32>);
        case 4: *stack_bytes = bwd_stack_bytes<float, 4, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 4, 4, 32>);
        case 5: *stack_bytes = bwd_stack_bytes<float, 5, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 5, 4, 32>);
        case 6: *stack_bytes = bwd_stack_bytes<float, 6, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 6, 4, 32>);
        case 7: *stack_bytes = bwd_stack_bytes<float, 7, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 7, 4, 32>);
        case 8: *stack_bytes = bwd_stack_bytes<float, 8, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 8, 4, 32>);
        case 9: *stack_bytes = bwd_stack_bytes<float, 9, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 9, 4, 32>);
        case 10: *stack_bytes = bwd_stack_bytes<float, 10, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 10, 4, 32>);
        case 12: *stack_bytes = bwd_stack_bytes<float, 12, 4>(); return reinterpret_cast<const void*>(&bwd_approx_kernel<float, 12, 4, 32>);
        default: break;
    }
    return nullptr;
}

const void* bwd_tape_ptr_f32(int N, bool interp) {
    if (interp) return bwd_tape_interp_ptr_f32(N);
    switch (N) {
        case 2: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 2, false>);
        case 3: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 3, false>);
        case 4: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 4, false>);
        case 5: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 5, false>);
        case 6: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 6, false>);
        case 7: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 7, false>);
        case 8: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 8, false>);
        case 9: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 9, false>);
        case 10: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 10, false>);
        case 12: return reinterpret_cast<const void*>(&bwd_tape_kernel<float, 12, false>);
        default: return nullptr;
    }
}

const void* bwd_contract_ptr_f32(int C) {
    switch (C) {
        case 8: return reinterpret_cast<const void*>(&bwd_contract_kernel<float, 8>);
        case 16: return reinterpret_cast<const void*>(&bwd_contract_kernel<float, 16>);
        case 32: return reinterpret_cast<const void*>(&bwd_contract_kernel<float, 32>);
        default: return nullptr;
    }
}

int bwd_segment_f32() { return 4; }

}  // namespace sk
