// Instantiations of the finite-difference adjoint from the forward tape (dyadic orders 0..4).
#include "sk_bwd_fd.cuh"
#include "sk_dispatch.h"

namespace sk {

namespace {
template <typename T, int ORDER>
const void* bwd_fd_rows(int lam) {
    switch (lam) {
        case 0: return reinterpret_cast<const void*>(&bwd_fd_tape_kernel<T, ORDER, 1>);
        case 1: return reinterpret_cast<const void*>(&bwd_fd_tape_kernel<T, ORDER, 2>);
        case 2: return reinterpret_cast<const void*>(&bwd_fd_tape_kernel<T, ORDER, 4>);
        case 3: return reinterpret_cast<const void*>(&bwd_fd_tape_kernel<T, ORDER, 8>);
        case 4: return reinterpret_cast<const void*>(&bwd_fd_tape_kernel<T, ORDER, 16>);
        default: return nullptr;
    }
}
}  // namespace

const void* bwd_fd_tape_ptr(int T, int order, int lam) {
    if (T == 1) return order == 3 ? bwd_fd_rows<float, 3>(lam) : order == 2 ? bwd_fd_rows<float, 2>(lam) : bwd_fd_rows<float, 1>(lam);
    return order == 3 ? bwd_fd_rows<double, 3>(lam) : order == 2 ? bwd_fd_rows<double, 2>(lam) : bwd_fd_rows<double, 1>(lam);
}

int fd_tape_row_elems(int T, int lam) { return T ? fd_tape_row<float>(1 << lam) : fd_tape_row<double>(1 << lam); }

int bwd_fd_ring_bytes(int T, int lam) {
    switch (lam) {
        case 0: return T ? fd_ring_warp_bytes<float, 1>() : fd_ring_warp_bytes<double, 1>();
        case 1: return T ? fd_ring_warp_bytes<float, 2>() : fd_ring_warp_bytes<double, 2>();
        case 2: return T ? fd_ring_warp_bytes<float, 4>() : fd_ring_warp_bytes<double, 4>();
        case 3: return T ? fd_ring_warp_bytes<float, 8>() : fd_ring_warp_bytes<double, 8>();
        case 4: return T ? fd_ring_warp_bytes<float, 16>() : fd_ring_warp_bytes<double, 16>();
        default: return 0;
    }
}

}  // namespace sk
