// Instantiations of the cooperative-block (strip pipeline) finite-difference forward wavefront.
#include "sk_dispatch.h"
#include "sk_fwd_fd.cuh"

namespace sk {

namespace {
template <typename T, int ORDER>
const void* fd_rows(int lam) {
    // rows per lane: R = min(2^lambda, 16) (a divisor of 2^lambda, so a lane's rows share a cell)
    switch (lam < 4 ? lam : 4) {
        case 0: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 1, kCoopWarps>);
        case 1: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 2, kCoopWarps>);
        case 2: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 4, kCoopWarps>);
        case 3: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 8, kCoopWarps>);
        default: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 16, kCoopWarps>);
    }
}
}  // namespace

const void* fwd_fd_coop_ptr(int T, int order, int lam) {
    if (T == 1) return order == 2 ? fd_rows<float, 2>(lam) : fd_rows<float, 1>(lam);
    return order == 2 ? fd_rows<double, 2>(lam) : fd_rows<double, 1>(lam);
}

}  // namespace sk
