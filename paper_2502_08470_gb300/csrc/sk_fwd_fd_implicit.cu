// Instantiations of the implicit finite-difference forward wavefront (Remark "higherfd"; ORDER 3
// of sweep_fd), one-warp and cooperative-block variants.
#include "sk_dispatch.h"
#include "sk_fwd_fd.cuh"

namespace sk {

namespace {
template <typename T, int CW>
const void* fd_rows(int lam) {
    // rows per lane: R = min(2^lambda, 16) (a divisor of 2^lambda, so a lane's rows share a cell)
    switch (lam < 4 ? lam : 4) {
        case 0: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, 3, 1, CW>);
        case 1: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, 3, 2, CW>);
        case 2: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, 3, 4, CW>);
        case 3: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, 3, 8, CW>);
        default: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, 3, 16, CW>);
    }
}
}  // namespace

const void* fwd_fd_implicit_ptr(int T, int lam, bool coop) {
    if (T == 1) return coop ? fd_rows<float, kCoopWarps>(lam) : fd_rows<float, 1>(lam);
    return coop ? fd_rows<double, kCoopWarps>(lam) : fd_rows<double, 1>(lam);
}

}  // namespace sk
