// Kernel lookup across the instantiation units (one per scheme family and precision, so that
// they compile in parallel).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace sk {

// T: 0 = FP64 cell updates, 1 = FP32; coop: the cooperative-block (strip pipeline) variant,
// launched with kCoopWarps warps per block; mt: the tiled-M variant (FP32 only).  NULL when no
// kernel exists for the request.
// tape: the one-warp-per-pair kernel that records the forward tape (for the approximation scheme
// a separate instantiation records the derivatives of each cell's outputs with respect to M; the
// interpolation kernels record their inputs whenever the launch carries a tape).
// mx: the FP32 approximation-scheme variant whose cells read M from the buffer the tensor-core M
// kernel writes (one warp per pair; with tape, recording the tape of output derivatives).
const void* fwd_poly_kernel_ptr(int T, bool interp, int N, bool coop, bool mt, bool tape = false, bool mx = false);
const void* fwd_approx_mx_ptr_f32(int N);
const void* fwd_approx_tape_mx_ptr_f32(int N);
const void* fwd_approx_tape_ptr_f32(int N);
const void* fwd_approx_tape_ptr_f32_mt(int N);
const void* fwd_approx_tape_ptr_f64(int N);
const void* fwd_fd_kernel_ptr(int T, int order, int lam, bool coop, bool tape = false);
// The FD forward that records the adjoint's tape, the FD adjoint from it (dyadic orders 0..4; NULL
// otherwise), and the elements of one lane's tape row.
const void* fwd_fd_tape_ptr(int T, int order, int lam);
const void* bwd_fd_tape_ptr(int T, int order, int lam);
int fd_tape_row_elems(int T, int lam);
// Shared memory of one warp of bwd_fd_tape_kernel (its ring of tape rows).
int bwd_fd_ring_bytes(int T, int lam);
const void* fwd_fd_coop_ptr(int T, int order, int lam);
const void* fwd_fd_implicit_ptr(int T, int lam, bool coop);  // order 3
const void* fwd_approx_ptr_f32(int N);
const void* fwd_interp_ptr_f32(int N);
const void* fwd_approx_coop_ptr_f32(int N);
const void* fwd_interp_coop_ptr_f32(int N);
const void* fwd_approx_ptr_f64(int N);
const void* fwd_interp_ptr_f64(int N);
const void* fwd_approx_coop_ptr_f64(int N);
const void* fwd_interp_coop_ptr_f64(int N);
const void* fwd_approx_mt_ptr_f32(int N);
const void* fwd_interp_mt_ptr_f32(int N);
const void* fwd_approx_coop_mt_ptr_f32(int N);
const void* fwd_interp_coop_mt_ptr_f32(int N);
// interpolation orders are split over several units (chunk k of each family)
const void* fwd_interp_ptr_f32_0(int N);
const void* fwd_interp_ptr_f32_1(int N);
const void* fwd_interp_ptr_f32_2(int N);
const void* fwd_interp_ptr_f32_3(int N);
const void* fwd_interp_ptr_f32_4(int N);
const void* fwd_interp_coop_ptr_f32_0(int N);
const void* fwd_interp_coop_ptr_f32_1(int N);
const void* fwd_interp_coop_ptr_f32_2(int N);
const void* fwd_interp_coop_ptr_f32_3(int N);
const void* fwd_interp_coop_ptr_f32_4(int N);
const void* fwd_interp_ptr_f64_0(int N);
const void* fwd_interp_ptr_f64_1(int N);
const void* fwd_interp_ptr_f64_2(int N);
const void* fwd_interp_ptr_f64_3(int N);
const void* fwd_interp_ptr_f64_4(int N);
const void* fwd_interp_coop_ptr_f64_0(int N);
const void* fwd_interp_coop_ptr_f64_1(int N);
const void* fwd_interp_coop_ptr_f64_2(int N);
const void* fwd_interp_coop_ptr_f64_3(int N);
const void* fwd_interp_coop_ptr_f64_4(int N);
const void* fwd_interp_mt_ptr_f32_0(int N);
const void* fwd_interp_mt_ptr_f32_1(int N);
const void* fwd_interp_mt_ptr_f32_2(int N);
const void* fwd_interp_mt_ptr_f32_3(int N);
const void* fwd_interp_mt_ptr_f32_4(int N);
const void* fwd_interp_coop_mt_ptr_f32_0(int N);
const void* fwd_interp_coop_mt_ptr_f32_1(int N);
const void* fwd_interp_coop_mt_ptr_f32_2(int N);
const void* fwd_interp_coop_mt_ptr_f32_3(int N);
const void* fwd_interp_coop_mt_ptr_f32_4(int N);
}  // namespace sk

namespace sk {
// Adjoint of the approximation scheme: dmax = 8 or 32 (register accumulators for d <= dmax);
// writes the per-warp shared-memory stack size.  NULL when no kernel exists.
const void* bwd_approx_ptr_f32(int N, int dmax, int* stack_bytes);
const void* bwd_approx_ptr_f64(int N, int dmax, int* stack_bytes);
int bwd_segment_f32();  // steps of the checkpointing adjoint's strip tape held in its shared-memory ring
int bwd_segment_f64();
}  // namespace sk

namespace sk {
// Tape-driven adjoint of the polynomial schemes (NULL when no kernel exists for order N) and
// the contraction of its dk/dM buffer into increment gradients.
const void* bwd_tape_ptr_f32(int N, bool interp);
const void* bwd_tape_ptr_f64(int N, bool interp);
const void* bwd_tape_interp_ptr_f32(int N);
const void* bwd_tape_interp_ptr_f64(int N);
const void* bwd_tape_interp_ptr_f64_0(int N);
const void* bwd_tape_interp_ptr_f64_1(int N);
// C: coordinates per contraction pass (8, 16 or 32)
const void* bwd_contract_ptr_f32(int C);
const void* bwd_contract_ptr_f64(int C);
}  // namespace sk

namespace sk {
struct PathSet;
struct BwdParams;
// Tensor-core contraction of the tape adjoint's dk/dM tiles (FP32 compute; N = 16 or 32 operand
// coordinates): operand tiles of a path set (nblk 128-row blocks per path, tc_operand_bytes
// bytes), and the contraction itself on `sms` CTAs (nrb_max: row blocks of the longest X path).
size_t tc_operand_bytes(int N, int64_t paths, int nblk);
cudaError_t launch_tc_operands(int N, const PathSet& S, int inc_mode, int lam, int dpad, int nblk, void* out,
                               cudaStream_t st);
cudaError_t launch_tc_contraction(int N, const BwdParams& B, int nrb_max, int sms, cudaStream_t st);

struct Launch;
// Tensor-core M of the forward (FP32 approximation scheme, 4 < d <= 32; KP = 16 or 32 padded
// coordinates): operand tiles of a path set (nblk 128-row blocks per path, m_operand_bytes bytes),
// and the M of work items 0 .. L.npairs - 1 of a launch into mx (mx_stride bytes per item, the
// layout of Launch::mx) on `sms` CTAs.
size_t m_operand_bytes(int KP, int64_t paths, int nblk);
cudaError_t launch_m_operands(int KP, const PathSet& S, int inc_mode, int lam, int dpad, int nblk, void* out,
                              cudaStream_t st);
cudaError_t launch_m_tc(int KP, const Launch& L, const void* xt, const void* yt, int xt_nblk, int yt_nblk, float* mx,
                        int64_t mx_stride, int sms, cudaStream_t st);
}  // namespace sk

namespace sk {
// Message returned by sigkernel_last_error() on this host thread (for entry points in other units).
void set_last_error(const char* msg);
}  // namespace sk

namespace sk {
// Two-sample permutation test on MMD^2 from the pooled Gram K [n][n] (the K_AB block filled, the
// K_BA block written here): scratch of mmd_perm_scratch_bytes(n, nperm) bytes (256-byte aligned),
// out [2 + nperm] as in sigkernel_mmd2_test.  Stream-ordered; returns the launch status.
size_t mmd_perm_scratch_bytes(int64_t n, int64_t nperm);
cudaError_t launch_mmd_perm(double* K, int64_t n, int64_t na, const uint8_t* labels, int64_t nperm, int unbiased,
                            void* scratch, double* out, cudaStream_t st);
}  // namespace sk
