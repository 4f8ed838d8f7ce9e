// Instantiations of the finite-difference forward wavefront and the kernel lookup.
#include "sk_dispatch.h"
#include "sk_fwd_fd.cuh"

namespace sk {

namespace {
template <typename T, int ORDER>
const void* fd_rows(int lam) {
    // rows per lane: R = min(2^lambda, 16) (a divisor of 2^lambda, so a lane's rows share a cell)
    switch (lam < 4 ? lam : 4) {
        case 0: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 1, 1>);
        case 1: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 2, 1>);
        case 2: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 4, 1>);
        case 3: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 8, 1>);
        default: return reinterpret_cast<const void*>(&fwd_fd_kernel<T, ORDER, 16, 1>);
    }
}
}  // namespace

const void* fwd_interp_ptr_f32(int N) {
    if (const void* k = fwd_interp_ptr_f32_0(N)) return k; if (const void* k = fwd_interp_ptr_f32_1(N)) return k; if (const void* k = fwd_interp_ptr_f32_2(N)) return k; if (const void* k = fwd_interp_ptr_f32_3(N)) return k; if (const void* k = fwd_interp_ptr_f32_4(N)) return k;
    return nullptr;
}

const void* fwd_interp_coop_ptr_f32(int N) {
    if (const void* k = fwd_interp_coop_ptr_f32_0(N)) return k; if (const void* k = fwd_interp_coop_ptr_f32_1(N)) return k; if (const void* k = fwd_interp_coop_ptr_f32_2(N)) return k; if (const void* k = fwd_interp_coop_ptr_f32_3(N)) return k; if (const void* k = fwd_interp_coop_ptr_f32_4(N)) return k;
    return nullptr;
}

const void* fwd_interp_ptr_f64(int N) {
    if (const void* k = fwd_interp_ptr_f64_0(N)) return k; if (const void* k = fwd_interp_ptr_f64_1(N)) return k; if (const void* k = fwd_interp_ptr_f64_2(N)) return k; if (const void* k = fwd_interp_ptr_f64_3(N)) return k; if (const void* k = fwd_interp_ptr_f64_4(N)) return k;
    return nullptr;
}

const void* fwd_interp_coop_ptr_f64(int N) {
    if (const void* k = fwd_interp_coop_ptr_f64_0(N)) return k; if (const void* k = fwd_interp_coop_ptr_f64_1(N)) return k; if (const void* k = fwd_interp_coop_ptr_f64_2(N)) return k; if (const void* k = fwd_interp_coop_ptr_f64_3(N)) return k; if (const void* k = fwd_interp_coop_ptr_f64_4(N)) return k;
    return nullptr;
}

const void* fwd_interp_mt_ptr_f32(int N) {
    if (const void* k = fwd_interp_mt_ptr_f32_0(N)) return k; if (const void* k = fwd_interp_mt_ptr_f32_1(N)) return k; if (const void* k = fwd_interp_mt_ptr_f32_2(N)) return k; if (const void* k = fwd_interp_mt_ptr_f32_3(N)) return k; if (const void* k = fwd_interp_mt_ptr_f32_4(N)) return k;
    return nullptr;
}

const void* fwd_interp_coop_mt_ptr_f32(int N) {
    if (const void* k = fwd_interp_coop_mt_ptr_f32_0(N)) return k; if (const void* k = fwd_interp_coop_mt_ptr_f32_1(N)) return k; if (const void* k = fwd_interp_coop_mt_ptr_f32_2(N)) return k; if (const void* k = fwd_interp_coop_mt_ptr_f32_3(N)) return k; if (const void* k = fwd_interp_coop_mt_ptr_f32_4(N)) return k;
    return nullptr;
}

const void* fwd_poly_kernel_ptr(int T, bool interp, int N, bool coop, bool mt, bool tape, bool mx) {
    if (mx) {
        if (T != 1 || interp || coop) return nullptr;
        return tape ? fwd_approx_tape_mx_ptr_f32(N) : fwd_approx_mx_ptr_f32(N);
    }
    if (tape && !interp) {
        if (coop) return nullptr;
        if (T == 1) return mt ? fwd_approx_tape_ptr_f32_mt(N) : fwd_approx_tape_ptr_f32(N);
        return mt ? nullptr : fwd_approx_tape_ptr_f64(N);
    }
    if (mt) {
        if (T != 1) return nullptr;
        if (coop) return interp ? fwd_interp_coop_mt_ptr_f32(N) : fwd_approx_coop_mt_ptr_f32(N);
        return interp ? fwd_interp_mt_ptr_f32(N) : fwd_approx_mt_ptr_f32(N);
    }
    if (coop) {
        if (T == 1) return interp ? fwd_interp_coop_ptr_f32(N) : fwd_approx_coop_ptr_f32(N);
        return interp ? fwd_interp_coop_ptr_f64(N) : fwd_approx_coop_ptr_f64(N);
    }
    if (T == 1) return interp ? fwd_interp_ptr_f32(N) : fwd_approx_ptr_f32(N);
    return interp ? fwd_interp_ptr_f64(N) : fwd_approx_ptr_f64(N);
}

const void* fwd_fd_kernel_ptr(int T, int order, int lam, bool coop, bool tape) {
    if (lam < 0 || lam > kLamMax) return nullptr;
    if (tape) return coop ? nullptr : fwd_fd_tape_ptr(T, order, lam);
    if (order == 3) return fwd_fd_implicit_ptr(T, lam, coop);
    if (coop) return fwd_fd_coop_ptr(T, order, lam);
    if (T == 1) return order == 2 ? fd_rows<float, 2>(lam) : fd_rows<float, 1>(lam);
    return order == 2 ? fd_rows<double, 2>(lam) : fd_rows<double, 1>(lam);
}

}  // namespace sk
