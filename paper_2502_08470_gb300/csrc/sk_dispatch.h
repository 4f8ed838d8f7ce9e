// Kernel lookup across the instantiation units (one per scheme family and precision, so that
// they compile in parallel).
#pragma once

namespace sk {

// T: 0 = FP64 cell updates, 1 = FP32.  NULL when no kernel exists for the request.
const void* fwd_poly_kernel_ptr(int T, bool interp, int N);
const void* fwd_fd_kernel_ptr(int T, int order, int lam);

const void* fwd_approx_ptr_f32(int N);
const void* fwd_approx_ptr_f64(int N);
const void* fwd_interp_ptr_f32(int N);
const void* fwd_interp_ptr_f64(int N);

}  // namespace sk
