/*
 * sigkernel.h -- C ABI of the GB300 (sm_103a) signature-kernel library.
 *
 * The library evaluates k(x, y) = <S(x), S(y)> for piecewise-linear paths by solving the Goursat
 * problem d^2k/(ds dt) = <x'(s), y'(t)> k, k(0, .) = k(., 0) = 1 (Theorem "sigpdetheorem",
 * Section 1) cell by cell over the grid of increment pairs, with the schemes of Cass, Piatti &
 * Pei, "Numerical Schemes for Signature Kernels":
 *
 *   SK_FD1          first-order explicit finite differences on the dyadic grid P_lambda
 *                   (Definition "dyadic scheme", Section 2)
 *   SK_FD2          second-order explicit finite differences (eq. (secondexplicitscheme),
 *                   Remark "higherfd", Section 2)
 *   SK_POLY_APPROX  polynomial approximation scheme of order N (Definition
 *                   "def:polyapproxscheme" and the explicit update after it, Section 3.2)
 *   SK_POLY_INTERP  polynomial interpolation scheme of order N (Definition
 *                   "def:polyinterpscheme", Section 3.3)
 *   SK_FD_IMPLICIT  implicit finite differences (Remark "higherfd", Section 2): each sub-cell
 *                   solves k11 = k10 + k01 - k00 + (m/4)(k00 + k10 + k01 + k11) for k11, the
 *                   two-dimensional trapezoid rule on the four corners (the Remark prints the
 *                   factor as 1/2; 1/4 is the trapezoid weight and the only one that converges).
 *                   A sub-cell with m = <dx, dy> = 4 has no solution: the call then reports
 *                   SK_ERR_NONFINITE
 *
 * Every scheme accepts a dyadic order lambda >= 0: each cell is split into 2^lambda x 2^lambda
 * sub-cells by linear interpolation of the paths (Definition "dyadic scheme"); for the polynomial
 * schemes this is the hybrid method of Section 3.2.
 *
 * Conventions shared by every entry point
 *   * Paths.  A set of paths is an sk_paths: the points of all paths concatenated row-major
 *     ([total_rows][d], element type given by `dtype`), and int64 row offsets off[0..count]
 *     (path a is rows off[a] .. off[a+1]-1).  Both arrays live in DEVICE memory and are owned by
 *     the caller; the library never frees or retains them past the call's stream work.  With
 *     SK_FLAG_INCREMENTS the rows hold increments dx_i = x_{i+1} - x_i instead of points.  A path
 *     with a single point (or no increment) has the trivial signature and k = 1.  `max_len` is a
 *     host-side upper bound on the rows of any one path and `rows_total` the host-side row count
 *     off[count]; a path longer than max_len, with no row at all, or with rows outside
 *     [0, rows_total) sets the device error word (SK_ERR_BAD_LENGTH) and its outputs are NaN.
 *     (max_len << lambda) may not exceed 131072.
 *   * Only the increment inner products M_ij = <dx_i, dy_j> enter any scheme (the explicit
 *     update of Section 3.2 depends on C_ij (s_{i+1}-s_i)(t_{j+1}-t_j) only), so no time
 *     partition is passed.
 *   * Outputs are FP64, device memory, caller-owned.
 *   * Alignment.  Device pointers must be aligned to their elements: path rows to the input
 *     element (8, 4 or 2 bytes), offsets, pair lists, outputs and gradients to 8 bytes, and tapes
 *     to 256 bytes.  A misaligned pointer is refused with SK_ERR_INVALID_ARG before anything is
 *     launched.  Sizes of device buffers cannot be checked: each must hold what its entry point
 *     states.
 *   * Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream) and
 *     make no host-device synchronisation.  Argument errors are reported by the return code
 *     before anything is launched; errors that need device data (bad lengths, an exhausted
 *     bounded wait, non-finite results) go to a device error word read by
 *     sigkernel_device_status().
 *   * Workspace.  `workspace` is a device buffer of at least sigkernel_workspace_size() bytes,
 *     caller-owned, 256-byte aligned; calls sharing a workspace must not overlap on the GPU.  If
 *     `workspace` is NULL the call allocates and frees its own with cudaMallocAsync /
 *     cudaFreeAsync on `stream`.
 *   * Return codes are the SK_* values below; sigkernel_last_error() gives a message for the
 *     last failing call on the calling host thread.
 */
#ifndef SIGKERNEL_H_
#define SIGKERNEL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
    SK_OK = 0,
    SK_ERR_INVALID_ARG = -1,   /* null pointer, bad count, degree, lambda, d, dtype ... */
    SK_ERR_UNSUPPORTED = -2,   /* a valid request this build has no kernel for */
    SK_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the CUDA error) */
    SK_ERR_WORKSPACE = -4,     /* workspace smaller than sigkernel_workspace_size() */
    SK_ERR_DEVICE_TIMEOUT = -5,/* a bounded device-side wait ran out (device error word) */
    SK_ERR_NONFINITE = -6,     /* a result was NaN or infinite (device error word) */
    SK_ERR_BAD_LENGTH = -7,    /* a path had no rows or more than max_len rows (device word) */
    SK_ERR_BAD_LABELS = -8     /* a relabelling of sigkernel_mmd2_test did not mark exactly
                                  A->count paths (device word) */
};

/* Schemes. */
enum { SK_FD1 = 0, SK_FD2 = 1, SK_POLY_APPROX = 2, SK_POLY_INTERP = 3, SK_FD_IMPLICIT = 4 };

/* Element type of the input rows. */
enum { SK_F64 = 0, SK_F32 = 1, SK_BF16 = 2 };

/* Arithmetic of the cell updates.
 *   SK_COMPUTE_F64  every cell update in FP64 (the plain wavefront).
 *   SK_COMPUTE_F32  cell updates in FP32 with a per-antidiagonal power-of-two exponent carried
 *                   per pair (values are rescaled by 2^-64 / 2^64 when the antidiagonal's
 *                   magnitude leaves [2^-64, 2^64]); increments FP32 (BF16 inputs are widened),
 *                   M accumulated in FP32; the coefficient map of a cell with |M| > 1 is built
 *                   in FP64; endpoints and reductions in FP64. */
enum { SK_COMPUTE_F64 = 0, SK_COMPUTE_F32 = 1 };

/* Option flags. */
enum {
    SK_FLAG_SYMMETRIC = 1,    /* sigkernel_gram: Y is X; only a <= b is computed and mirrored */
    SK_FLAG_INCREMENTS = 2,   /* rows hold increments, not points */
    SK_FLAG_UNBIASED = 4,     /* sigkernel_mmd2: U-statistic (diagonals of K_AA, K_BB left out) */
    SK_FLAG_NO_SORT = 8,      /* process pairs in the given order (no cell-count ordering) */
    SK_FLAG_TIME_KERNEL = 16, /* record CUDA events around the wavefront kernel(s) of this call on
                                 `stream`; read the duration with sigkernel_last_kernel_ms() */
    SK_FLAG_STRIP_PIPELINE = 32,    /* forward: sweep every pair of 2 or more strips (32 grid rows
                                       each) with a block of warps, one strip per warp in a
                                       pipeline, instead of one warp per pair */
    SK_FLAG_NO_STRIP_PIPELINE = 64, /* forward: always one warp per pair.  With neither flag the
                                       library pipelines every pair of 2 or more strips when some
                                       pair has 32 or more strips and the batch is too small to
                                       fill the GPU with one warp per pair.  Neither applies to the
                                       tape forward or to the adjoints (one warp per pair).  With
                                       so few pairs that each pair's 16-warp ring can span 8 or
                                       more blocks, the pipelined polynomial forward spreads each
                                       ring over co-resident blocks (a cooperative launch; the
                                       results are the same bit for bit) */
    SK_FLAG_NO_TILED_M = 128,       /* forward, polynomial schemes in FP32, where the tensor cores
                                       do not compute M (see SK_FLAG_NO_TC): form each cell's M
                                       from its two increment rows.  By default, with d > 8, each
                                       warp first computes a strip's M_ij for all columns at once
                                       (the same values bit for bit) */
    SK_FLAG_CHECKPOINT = 256,       /* sigkernel_backward, approximation scheme: run the
                                       checkpointing adjoint (no tape; its workspace grows with the
                                       paths, not with the pair count) instead of the default
                                       adjoint from chunked forward tapes */
    SK_FLAG_NO_TC = 512             /* FP32: keep the tensor cores out.  By default (1) the
                                       approximation scheme's forward with one warp per pair
                                       (plain or recording a tape; not the strip pipeline) with
                                       4 < d <= 32 takes each cell's M_ij = <dx_i, dy_j> /
                                       4^lambda from a tcgen05 GEMM of the increments, run per
                                       chunk of pairs before the chunk's sweep (flag set: tiled
                                       or per-cell M on the FMA pipe, see SK_FLAG_NO_TILED_M),
                                       and (2) with 8 < d <= 32 an adjoint from a tape contracts
                                       dk/dM with the increments on the tensor cores when the
                                       refined grid of the longest pair fits its tensor memory
                                       ((ceil(rows / 128) + ceil(cols / 128)) x (16 or 32) <=
                                       256; flag set: on the FMA pipe).  The M kernel splits each
                                       FP32 increment into three BF16 parts and keeps six of the
                                       nine part products (at most about 2^-23 relative per
                                       product); the contraction splits dk/dM and the increments
                                       into two parts and keeps three products (at most about
                                       3 x 2^-16); both
                                       accumulate in FP32 */
};

typedef struct {
    int32_t scheme;           /* SK_FD1, SK_FD2, SK_POLY_APPROX, SK_POLY_INTERP, SK_FD_IMPLICIT */
    int32_t degree;           /* N: 2 <= N <= 16 (approximation), 2 <= N <= 12 (interpolation);
                                 ignored by FD (Definitions of Sections 3.2 and 3.3 take N >= 2) */
    int32_t dyadic;           /* lambda: 0 <= lambda <= 8 */
    int32_t compute;          /* SK_COMPUTE_F64 or SK_COMPUTE_F32 */
    int32_t interp_extra;     /* J for SK_POLY_INTERP: series terms kept beyond N before the
                                 interpolation projection; 0 = the build's value for the compute
                                 mode (6 for FP32, 10 for FP64); any other value must equal it */
    int32_t flags;            /* SK_FLAG_* */
    int32_t warps_per_block;  /* forward launch shape: 1, 2 or 4 warps per block for one warp per
                                 pair; 0 = the shape sigkernel_autotune chose for this shape of
                                 call, else the default (4) */
    int32_t reserved;         /* must be 0 */
} sk_options;

typedef struct {
    const void* rows;         /* device: [rows_total][d] elements of the call's dtype */
    const int64_t* offsets;   /* device: [count + 1], off[0] = 0, non-decreasing */
    int64_t count;            /* number of paths (>= 0) */
    int64_t max_len;          /* host: upper bound on off[a+1] - off[a] */
    int64_t rows_total;       /* host: off[count], the number of rows in `rows` */
} sk_paths;

/* Which call a workspace is sized for. */
enum { SK_OP_PAIRS = 0, SK_OP_GRAM = 1, SK_OP_BACKWARD = 2, SK_OP_MMD2 = 3, SK_OP_BACKWARD_TAPE = 4,
       SK_OP_MMD2_TEST = 5 };

/*
 * sigkernel_workspace_size -- writes to *bytes the device workspace the call `op` needs for
 * these shapes and options and returns SK_OK, or returns the SK_ERR_* code the call itself would
 * return for these arguments (then *bytes = 0).  `npairs` is the pair count for SK_OP_PAIRS /
 * SK_OP_BACKWARD / SK_OP_BACKWARD_TAPE with a pair list (pass -1 for a Gram); for SK_OP_MMD2 it
 * is 0 for the value alone and nonzero for the value with gradients (X = A, Y = B); for
 * SK_OP_MMD2_TEST it is the number of relabellings (X = A, Y = B); ignored otherwise.  Queries properties of the current device (SM count, occupancy); no memory traffic.
 */
int sigkernel_workspace_size(int32_t op, const sk_paths* X, const sk_paths* Y, int32_t d,
                             int64_t npairs, const sk_options* opt, size_t* bytes);

/*
 * sigkernel_pairs -- out[k] = k_hat(X_{pair_a[k]}, Y_{pair_b[k]}) for k < npairs.
 * The scheme output k_hat is the endpoint of the chosen scheme: for the polynomial schemes the
 * average of the top-edge and right-edge evaluations at the last cell (Definitions
 * "def:polyapproxscheme" and "def:polyinterpscheme"), for FD the last node of P_lambda.
 *   X, Y      path sets (device rows/offsets, see above); Y may equal X
 *   d         coordinates per row, 1 <= d <= 64
 *   dtype     SK_F64, SK_F32 or SK_BF16 (element type of X->rows and Y->rows)
 *   pair_a/b  device int64 [npairs]; indices into X and Y
 *   out       device double [npairs]
 * All pairs run in one persistent launch; pairs are taken from a work queue ordered by cell
 * count (largest first) unless SK_FLAG_NO_SORT.
 */
int sigkernel_pairs(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                    const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                    const sk_options* opt, double* out, void* workspace, size_t workspace_bytes,
                    void* stream);

/*
 * sigkernel_gram -- G[a][b] = k_hat(X_a, Y_b), G row-major [X->count][Y->count] device doubles.
 * With SK_FLAG_SYMMETRIC, Y must describe the same paths as X; only a <= b is solved and the
 * result mirrored (every scheme is symmetric under exchanging x and y: the cell map is invariant
 * under (p, s) <-> (q, t) and the endpoint averages both edges).  Other arguments as for
 * sigkernel_pairs.
 */
int sigkernel_gram(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                   const sk_options* opt, double* G, void* workspace, size_t workspace_bytes,
                   void* stream);

/*
 * sigkernel_backward -- reverse-mode derivative of the discrete scheme (the paper defines no
 * gradient; this is the exact adjoint of the scheme's own arithmetic, run as a reverse
 * wavefront).
 *   Pair-list mode (pair_a != NULL): grad_out[k] = dL/dk_hat(X_{pair_a[k]}, Y_{pair_b[k]}).
 *   Gram mode (pair_a == NULL): grad_out is [X->count][Y->count] row-major, dL/dG[a][b].
 *   grad_X  device double, same row layout as X->rows ([off[count]][d]): dL/d(row), added to
 *           the existing contents (the caller zeroes it first for a plain gradient); NULL skips.
 *   grad_Y  likewise for Y.  When Y is X (same rows pointer) both accumulate into the same
 *           buffer correctly if grad_X == grad_Y.
 * Every scheme records forward tapes in chunks of pairs (at most 64 GiB each, in the workspace)
 * and runs the tape adjoint after each chunk (sigkernel_forward_tape and sigkernel_backward_tape
 * below, one chunk at a time), so the call re-runs the forward sweep once.  When the paths are so
 * long that a chunk cannot fill the GPU, SK_POLY_APPROX runs the checkpointing adjoint instead
 * (the strip hand-offs as checkpoints, one strip's tape re-recorded from them at a time;
 * d <= 32) and the other schemes, which have none, return SK_ERR_UNSUPPORTED.
 * SK_FLAG_CHECKPOINT asks for the
 * checkpointing adjoint of SK_POLY_APPROX outright.  Orders with an adjoint: 2..10 and 12
 * (approximation), 2..12 (interpolation); the FD schemes for dyadic orders 0..4.
 * Accumulation uses device atomics, so the last bits of the gradient can vary between runs.
 */
int sigkernel_backward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                       const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                       const sk_options* opt, const double* grad_out, double* grad_X,
                       double* grad_Y, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Forward tape (approximation orders 2..10 and 12, interpolation orders 2..12, the FD schemes at
 * dyadic orders 0..4).  sigkernel_forward_tape computes the same results as sigkernel_pairs /
 * sigkernel_gram (Gram mode when pair_a is NULL; `out` is then [X->count][Y->count] and
 * SK_FLAG_SYMMETRIC applies) and also records, in the caller's `tape`, what the adjoint needs of
 * every cell and the exponent of each k_hat.  For SK_POLY_INTERP that is the cell's inputs (the
 * two incoming edge coefficient vectors, their exponent and the cell's M: 2N+4 elements padded to
 * 16 bytes); for SK_POLY_APPROX it is the derivatives of the cell's two outgoing edge vectors
 * with respect to M (orders 1..N of each), their exponent and M: 2N+2 elements; for the FD
 * schemes, per refined column, a lane's 2^lambda node differences, the two bottom nodes, the
 * sub-cell m and the exponent (2^lambda + 4 elements padded to 16 bytes).  sigkernel_backward_tape then
 * runs the adjoint from the tape without recomputing the forward sweep; it writes every cell's
 * dL/dM into its workspace and contracts that with the increments in a second kernel.  Both
 * calls must use the same X, Y, pair list, options and path contents.
 *   tape        device buffer, 256-byte aligned, caller-owned, >= sigkernel_tape_size() bytes;
 *               the size grows as npairs x (max_len << lambda)^2 x (2N+2) elements (approximation):
 *               about 61 GB for 16,384 pairs of 257-point paths at N = 6 in FP32.
 *   sigkernel_tape_size: `npairs` = -1 for a Gram; writes the bytes and returns SK_OK or SK_ERR_*.
 * The backward's workspace is sized with SK_OP_BACKWARD_TAPE; it holds one element per cell (4 B
 * in FP32, 8 B in FP64; about 4.4 GB for the Gram above).  Other arguments and the gradient
 * semantics are those of sigkernel_backward; any d <= 64 is supported.
 */
int sigkernel_tape_size(const sk_paths* X, const sk_paths* Y, int32_t d, int64_t npairs,
                        const sk_options* opt, size_t* bytes);
int sigkernel_forward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                           const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                           const sk_options* opt, double* out, void* tape, size_t tape_bytes,
                           void* workspace, size_t workspace_bytes, void* stream);
int sigkernel_backward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                            const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                            const sk_options* opt, const void* tape, size_t tape_bytes,
                            const double* grad_out, double* grad_X, double* grad_Y,
                            void* workspace, size_t workspace_bytes, void* stream);

/*
 * sigkernel_autotune -- choose the launch shape of a forward call (sigkernel_pairs when pair_a is
 * non-NULL, else sigkernel_gram; same arguments) by timing the candidates on these inputs:
 * one warp per pair in blocks of 1, 2 or 4 warps (each with and without the tiled M where it
 * applies), and the strip pipeline (blocks of 16 warps sharing each pair of two or more strips)
 * when some pair spans two strips.  Each candidate runs
 * once to warm up, then `trials` (1..1000) timed times on `stream`; `out` is overwritten with the
 * results.  The call allocates its own workspace (stream-ordered) and returns after the runs have
 * finished on the device.
 *   best     written with *opt except warps_per_block and the strip-pipeline and tiled-M flags,
 *            which name the winner explicitly (pass it to later calls to reuse the choice).
 *   best_ms  the winner's fastest call in milliseconds (NULL to skip).
 * The winner is also remembered in this process for calls of the same shape (scheme, degree,
 * lambda, compute mode, d, call kind, path counts, max_len, pair count, device) whose
 * warps_per_block is 0 and that set no strip-pipeline flag.  Workspace sizes follow the chosen
 * shape, so query sigkernel_workspace_size after tuning.  sigkernel_autotune_clear forgets every
 * remembered choice.  The paper has no counterpart: this is a facility of the library.
 */
int sigkernel_autotune(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                       const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                       const sk_options* opt, double* out, int32_t trials, sk_options* best,
                       float* best_ms, void* stream);
void sigkernel_autotune_clear(void);

/*
 * sigkernel_mmd2 -- squared maximum mean discrepancy between the path sets A and B with the
 * signature kernel (the paper's library offers MMD, Sections 1 and 4, without a formula):
 *   biased:   mean(K_AA) + mean(K_BB) - 2 mean(K_AB)
 *   unbiased (SK_FLAG_UNBIASED): K_AA and K_BB means over their off-diagonal entries.
 *   out       device double [4]: MMD^2, mean K_AA, mean K_BB, mean K_AB (as used above)
 *   grad_A/B  device double with A's / B's row layout, or NULL: d MMD^2 / d rows, OVERWRITTEN.
 * K_AA and K_BB are solved as symmetric Grams; the reduction runs in FP64 on the device.
 * Gradients (every scheme with an adjoint, see sigkernel_backward) run the adjoint from forward
 * tapes: each Gram block is solved in chunks of pairs whose tape is at most 64 GiB, the chunk's
 * forward recording the tape and the tape adjoint following at once with the block's constant
 * weights.  A block whose paths are so long that a chunk cannot fill the GPU uses the
 * checkpointing adjoint of sigkernel_backward instead (d <= 32; approximation scheme only, else
 * SK_ERR_UNSUPPORTED).
 * The workspace (SK_OP_MMD2 with npairs != 0) includes the tape.
 */
int sigkernel_mmd2(const sk_paths* A, const sk_paths* B, int32_t d, int32_t dtype,
                   const sk_options* opt, double* out, double* grad_A, double* grad_B,
                   void* workspace, size_t workspace_bytes, void* stream);

/*
 * sigkernel_mmd2_test -- two-sample permutation test on MMD^2 (the paper names statistical
 * hypothesis testing among the library's uses, Sections 1 and 4, without defining it; this is the
 * standard permutation test).  The pooled sample Z = (A_0..A_{na-1}, B_0..B_{nb-1}) is solved once
 * as one symmetric Gram K (blocks K_AA, K_BB symmetric and K_AB full, as in sigkernel_mmd2, then
 * K_BA = K_AB^T); each relabelling's statistic is then the MMD^2 (biased, or with SK_FLAG_UNBIASED
 * the U-statistic) of the two subsets it marks, read from K in FP64 on the device.
 *   labels   device uint8 [nperm][na + nb]: row p marks with a nonzero byte the pooled paths that
 *            relabelling p assigns to the first sample.  A row that does not mark exactly na paths
 *            gets a NaN statistic and sets SK_ERR_BAD_LABELS in the device error word.  The caller
 *            draws the relabellings (uniformly random permutations of the split, usually).
 *   nperm    0 <= nperm <= 2^24; na + nb <= 65536; na, nb >= 1 (>= 2 for the U-statistic)
 *   out      device double [2 + nperm]: out[0] = MMD^2 of the given split (A, B); out[1] = p-value
 *            (1 + #{p : out[2 + p] >= out[0]}) / (1 + nperm), NaN when any statistic is NaN;
 *            out[2 + p] = MMD^2 under relabelling p.
 * Workspace: SK_OP_MMD2_TEST with npairs = nperm; it holds K ((na + nb)^2 doubles).  A statistic
 * depends only on K and its own relabelling (bitwise, for a given na + nb).
 */
int sigkernel_mmd2_test(const sk_paths* A, const sk_paths* B, int32_t d, int32_t dtype,
                        const sk_options* opt, const uint8_t* labels, int64_t nperm, double* out,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * sigkernel_pairs_noalloc -- sigkernel_pairs for callers that cannot allocate device memory
 * (an allocator that forbids new device allocations, a host application that owns all device
 * memory, a loop that must not risk an allocation).  The paper has no counterpart.  Same
 * arguments and result as sigkernel_pairs, without a workspace: the scratch is a fixed 64 MiB
 * array in device global memory that every GPU loading the library holds until the process exits
 * (sigkernel_noalloc_capacity() gives its size).  A call needing more scratch than that returns
 * SK_ERR_WORKSPACE with both sizes in sigkernel_noalloc_last_error().  All calls on a device share
 * the array and leave their contents in it; each call clears the parts that must start at zero,
 * and calls that overlap on the GPU race.  The first call on a device looks up the array's
 * address with that device current: make it before any stream capture on that device.  The call
 * runs no cudaMalloc, cudaMallocAsync, cudaFree or other allocating routine.
 */
int sigkernel_pairs_noalloc(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                            const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                            const sk_options* opt, double* out, void* stream);
size_t sigkernel_noalloc_capacity(void);
const char* sigkernel_noalloc_last_error(void);

/*
 * sigkernel_fma_peak -- measures the multiply-add throughput of the current GPU and writes it to
 * *tflops in TFLOP/s (2 FLOP per FMA).  The paper has no counterpart: this is a measurement
 * utility whose result is the denominator of the roofline fractions of the ALU-bound wavefront
 * kernels.  Every thread of 4 blocks per SM (384 threads each) runs independent chains
 * v <- v * m + c; the kernel is launched once to warm up and then `reps` (1..100) times on
 * `stream`, each timed with CUDA events, and the fastest launch counts.
 *   compute  SK_COMPUTE_F32 or SK_COMPUTE_F64 (the FMA type)
 *   packed   nonzero (FP32 only): the chains run through the two-wide FP32 instruction (two FMAs
 *            per instruction)
 * Synchronous: returns after the last launch has finished.  A few milliseconds per launch.  It
 * changes no clock or other setting of the GPU: the figure is at whatever clock the GPU runs.
 */
int sigkernel_fma_peak(int32_t compute, int32_t packed, int32_t reps, double* tflops, void* stream);

/*
 * sigkernel_device_status -- synchronises `stream`, reads and clears the device error word of
 * the current device, and returns SK_OK or the first recorded SK_ERR_* code.
 */
int sigkernel_device_status(void* stream);

/*
 * sigkernel_last_kernel_ms -- device time in milliseconds between the two CUDA events recorded
 * around the wavefront kernel(s) of the last call made with SK_FLAG_TIME_KERNEL on this host
 * thread (waits for the second event).  Returns -1 if no such call was made.
 */
float sigkernel_last_kernel_ms(void);

/*
 * sigkernel_set_wait_limit -- how many times a strip-pipeline hand-off wait polls its progress word
 * (each poll followed by a ~64 ns sleep) before it gives up: the warp then records
 * SK_ERR_DEVICE_TIMEOUT in the device error word, finishes its sweep without waiting (that pair's
 * result is then wrong) and the kernel returns normally.  0 restores the default, 2^20 polls.
 * Process-wide; calls launched after it use the new limit.  The paper has no counterpart: this
 * is a robustness facility (a caller that wants a stalled pipeline reported sooner, and the test
 * of the timeout path).
 */
void sigkernel_set_wait_limit(uint32_t polls);

/* Message describing the last non-SK_OK return on this host thread ("" if none). */
const char* sigkernel_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int sigkernel_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIGKERNEL_H_ */
