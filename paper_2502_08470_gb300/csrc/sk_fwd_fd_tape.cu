// Instantiations of the finite-difference forward wavefront that records the tape of the FD adjoint
// (one warp per pair; dyadic orders 0..4, R = 2^lambda node rows per lane).
#include "sk_dispatch.h"
#include "sk_fwd_fd.cuh"

namespace sk {

namespace {
template <typename T, int ORDER>
const void* fd_tape_rows(int lam) {
    switch (lam) {
        case 0: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 1, 1, true>);
        case 1: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 2, 1, true>);
        case 2: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 4, 1, true>);
        case 3: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 8, 1, true>);
        case 4: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 16, 1, true>);
        default: return nullptr;
    }
}
}  // namespace

const void* fwd_fd_tape_ptr(int T, int order, int lam) {
    if (T == 1) return order == 3 ? fd_tape_rows<float, 3>(lam) : order == 2 ? fd_tape_rows<float, 2>(lam) : fd_tape_rows<float, 1>(lam);
    return order == 3 ? fd_tape_rows<double, 3>(lam) : order == 2 ? fd_tape_rows<double, 2>(lam) : fd_tape_rows<double, 1>(lam);
}

}  // namespace sk
