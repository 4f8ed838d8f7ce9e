// Host side of the C ABI (include/sigkernel.h): argument checks, workspace layout, constant
// tables, the increment and scheduling kernels, and dispatch to the wavefront kernels.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "sk_bwd_poly.cuh"
#include "sk_common.cuh"
#include "sk_dispatch.h"

namespace sk {

__device__ int g_sk_error = 0;

namespace {

thread_local std::string t_last_error;
std::atomic<uint32_t> g_wait_limit{0};  // sigkernel_set_wait_limit (0 = the kernels' default)
thread_local cudaEvent_t t_ev0 = nullptr, t_ev1 = nullptr;
thread_local bool t_timed = false;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

// Launch shapes chosen by sigkernel_autotune, per shape of call (used when a call leaves
// warps_per_block at 0 and sets no strip-pipeline flag).
struct TuneKey {
    int dev, scheme, degree, dyadic, compute, dpad, mode;
    int64_t xmax, ymax, xcount, ycount, npairs;
    bool operator<(const TuneKey& o) const {
        const int64_t a[] = {dev, scheme, degree, dyadic, compute, dpad, mode, xmax, ymax, xcount, ycount, npairs};
        const int64_t b[] = {o.dev, o.scheme, o.degree, o.dyadic, o.compute, o.dpad, o.mode, o.xmax, o.ymax, o.xcount,
                             o.ycount, o.npairs};
        for (int i = 0; i < 12; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
struct TuneChoice {
    int wpb;   // warps per block of the one-warp-per-pair kernel
    int pipe;  // 1: strip pipeline, -1: none
    int mt;    // 1: tiled M where eligible, -1: per-cell M
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

TuneKey tune_key(int dev, const sk_paths* X, const sk_paths* Y, const sk_options* o, int dpad, int mode,
                 int64_t npairs) {
    return TuneKey{dev, o->scheme, o->degree, o->dyadic, o->compute, dpad, mode,
                   X->max_len, Y->max_len, X->count, Y->count, npairs};
}

#define SK_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(SK_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// A workspace that a call allocated for itself (the caller passed none).  It is freed in stream
// order on every return path, so a call that fails after the allocation does not leak it.
struct OwnedWorkspace {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    OwnedWorkspace() = default;
    OwnedWorkspace(const OwnedWorkspace&) = delete;
    OwnedWorkspace& operator=(const OwnedWorkspace&) = delete;
    ~OwnedWorkspace() {
        if (p) cudaFreeAsync(p, st);
    }
    cudaError_t release() {  // the success path's free, with its status
        void* q = p;
        p = nullptr;
        return q ? cudaFreeAsync(q, st) : cudaSuccess;
    }
};

// ------------------------------------------------------------------------------------------
// Increments dx_i = x_{i+1} - x_i (or the caller's increments) in the compute type, rows
// zero-padded to `dpad` elements.  One block per path (grid-stride over paths).
// ------------------------------------------------------------------------------------------
template <typename Tin> __device__ __forceinline__ double load_elem(const Tin* p) { return static_cast<double>(*p); }
template <> __device__ __forceinline__ double load_elem<__nv_bfloat16>(const __nv_bfloat16* p) {
    return static_cast<double>(__bfloat162float(*p));
}

template <typename Tin, typename T>
__global__ void increments_kernel(const Tin* __restrict__ rows, const int64_t* __restrict__ off, int64_t count,
                                  int64_t rows_total, int64_t max_len, int d, int dpad, int inc_mode,
                                  T* __restrict__ out) {
    for (int64_t a = blockIdx.x; a < count; a += gridDim.x) {
        const int64_t r0 = off[a], r1 = off[a + 1], n = r1 - r0;
        if (r0 < 0 || r1 > rows_total || n < (inc_mode ? 0 : 1) || n > max_len) continue;
        const int64_t len = inc_mode ? n : n - 1;
        for (int64_t idx = threadIdx.x; idx < len * dpad; idx += blockDim.x) {
            const int64_t i = idx / dpad;
            const int c = static_cast<int>(idx - i * dpad);
            double v = 0.0;
            if (c < d) {
                const Tin* p = rows + (r0 + i) * d + c;
                v = inc_mode ? load_elem(p) : load_elem(p + d) - load_elem(p);
            }
            out[(r0 + i) * dpad + c] = static_cast<T>(v);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Work queue ordered by cell count (largest first): a counting sort on floor(log2(cells)).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int cell_bucket(const Launch& L, int64_t item) {
    PairDesc P = decode_pair(L, item);
    if (P.lx <= 0 || P.ly <= 0) return 0;
    unsigned long long cells = static_cast<unsigned long long>(P.lx) * static_cast<unsigned long long>(P.ly);
    return 64 - __clzll(cells);  // 1..64
}

__global__ void sched_hist_kernel(Launch L, unsigned int* hist) {
    for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < L.npairs;
         it += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&hist[cell_bucket(L, it)], 1u);
}

__global__ void sched_scan_kernel(unsigned int* hist, unsigned int* cursor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned int acc = 0;
        for (int b = 64; b >= 0; --b) {
            cursor[b] = acc;
            acc += hist[b];
        }
    }
}

__global__ void sched_scatter_kernel(Launch L, unsigned int* cursor, int32_t* order) {
    for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < L.npairs;
         it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        unsigned int pos = atomicAdd(&cursor[cell_bucket(L, it)], 1u);
        order[pos] = static_cast<int32_t>(it);
    }
}

// ------------------------------------------------------------------------------------------
// Argument checks and workspace planning.
// ------------------------------------------------------------------------------------------
struct Plan {
    int T;               // 0 = FP64, 1 = FP32 compute
    int nvec, dpad;
    int64_t npairs;
    int mode;
    bool same_xy;        // Y's rows/offsets are X's
    const void* kern;    // wavefront kernel
    int threads;         // threads per block
    int blocks;          // persistent grid
    bool coop;           // cooperative-block kernel (strip pipeline for long pairs)
    int coop_min_strips; // strips from which a pair is swept by a whole block
    int grid_bpp;        // grid strip pipeline: blocks sharing each pair (0 = off)
    size_t off_gprog;    // its progress words [npairs][grid_bpp x kCoopWarps]
    bool mtile;          // tiled M (wide increments, polynomial schemes)
    int64_t mtile_cols;  // columns of one warp's M strip buffer
    int64_t mtile_off;   // byte offset of that buffer in a warp slot
    // tensor-core M (FP32 approximation scheme, 4 < d <= 32, one warp per pair): the forward is
    // swept in chunks of mx_chunk items, each preceded by the M kernel writing the chunk's M
    bool mx;
    int kp;              // padded coordinates of the M operand tiles (16 or 32)
    int xt_nblk, yt_nblk;// 128-row blocks per path of the operand tiles
    int64_t mx_stride;   // bytes of M per item
    int64_t mx_chunk;    // items per chunk (npairs when MX is off)
    size_t off_xt, off_yt, off_mx;
    int smem_x;          // dynamic shared memory of the tiled-M x rows per block
    int64_t slot_bytes;  // scratch per warp slot
    int64_t buf_cols;    // hand-off columns per warp slot
    // workspace layout (byte offsets)
    size_t off_incx, off_incy, off_queue, off_hist, off_order, off_scratch, total;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kGridMinBlocks = 8;  // fewest blocks a pair's ring may span in the grid strip pipeline
// Bytes of precomputed M a forward holds at once (the chunk of items whose M the tensor cores
// wrote before the chunk's sweep); a chunk is a whole number of the sweep's resident warps.
constexpr size_t kMxBudget = size_t(8) << 30;

int check_paths(const sk_paths* P, const char* name, int d) {
    if (!P) return fail(SK_ERR_INVALID_ARG, "%s is NULL", name);
    if (P->count < 0) return fail(SK_ERR_INVALID_ARG, "%s->count < 0", name);
    if (P->count > 0 && !P->offsets) return fail(SK_ERR_INVALID_ARG, "%s->offsets is NULL", name);
    if (P->rows_total < 0 || P->max_len < 0) return fail(SK_ERR_INVALID_ARG, "%s: negative sizes", name);
    if (P->rows_total > 0 && !P->rows) return fail(SK_ERR_INVALID_ARG, "%s->rows is NULL", name);
    if (P->count > (int64_t(1) << 30)) return fail(SK_ERR_UNSUPPORTED, "%s: more than 2^30 paths", name);
    (void)d;
    return SK_OK;
}

// The kernels read path rows as elements of the input type, and offsets, pair lists, outputs and
// gradients as 8-byte elements; a pointer misaligned for its elements would fault on the device,
// so the compute entry points refuse it before anything runs (NULL passes here: the callers check
// for NULL where a pointer is required).
int check_path_ptrs(const sk_paths* P, int32_t dtype, const char* name) {
    if (!P) return SK_OK;
    const size_t es = dtype == SK_F64 ? 8 : dtype == SK_F32 ? 4 : dtype == SK_BF16 ? 2 : 1;
    if (reinterpret_cast<uintptr_t>(P->rows) % es)
        return fail(SK_ERR_INVALID_ARG, "%s->rows is not %zu-byte aligned", name, es);
    if (reinterpret_cast<uintptr_t>(P->offsets) % 8) return fail(SK_ERR_INVALID_ARG, "%s->offsets is not 8-byte aligned", name);
    return SK_OK;
}

int check_call_ptrs(const sk_paths* X, const char* xn, const sk_paths* Y, const char* yn, int32_t dtype,
                    std::initializer_list<std::pair<const void*, const char*>> ptrs8) {
    int rc;
    if ((rc = check_path_ptrs(X, dtype, xn)) != SK_OK) return rc;
    if ((rc = check_path_ptrs(Y, dtype, yn)) != SK_OK) return rc;
    for (const auto& q : ptrs8)
        if (reinterpret_cast<uintptr_t>(q.first) % 8) return fail(SK_ERR_INVALID_ARG, "%s is not 8-byte aligned", q.second);
    return SK_OK;
}

int check_options(const sk_options* o, int32_t d, int32_t dtype) {
    if (!o) return fail(SK_ERR_INVALID_ARG, "options is NULL");
    if (o->reserved != 0) return fail(SK_ERR_INVALID_ARG, "options.reserved must be 0");
    if (o->scheme < SK_FD1 || o->scheme > SK_FD_IMPLICIT) return fail(SK_ERR_INVALID_ARG, "unknown scheme %d", o->scheme);
    if (o->compute != SK_COMPUTE_F64 && o->compute != SK_COMPUTE_F32)
        return fail(SK_ERR_INVALID_ARG, "unknown compute mode %d", o->compute);
    if (dtype != SK_F64 && dtype != SK_F32 && dtype != SK_BF16) return fail(SK_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    if (d < 1 || d > kDMax) return fail(SK_ERR_INVALID_ARG, "d = %d outside [1, %d]", d, kDMax);
    if (o->dyadic < 0 || o->dyadic > kLamMax) return fail(SK_ERR_INVALID_ARG, "dyadic order %d outside [0, %d]", o->dyadic, kLamMax);
    if (o->scheme == SK_POLY_APPROX && (o->degree < 2 || o->degree > kNMaxApprox))
        return fail(SK_ERR_INVALID_ARG, "approximation order %d outside [2, %d]", o->degree, kNMaxApprox);
    if (o->scheme == SK_POLY_INTERP && (o->degree < 2 || o->degree > kNMaxInterp))
        return fail(SK_ERR_INVALID_ARG, "interpolation order %d outside [2, %d]", o->degree, kNMaxInterp);
    if (o->scheme == SK_POLY_INTERP && o->interp_extra != 0) {
        int j = (o->compute == SK_COMPUTE_F32) ? kJF32 : kJF64;
        if (o->interp_extra != j)
            return fail(SK_ERR_UNSUPPORTED, "interp_extra %d: this build keeps J = %d for this compute mode",
                        o->interp_extra, j);
    }
    if (o->warps_per_block != 0 && o->warps_per_block != 1 && o->warps_per_block != 2 && o->warps_per_block != 4)
        return fail(SK_ERR_UNSUPPORTED, "warps_per_block %d (this build: 0, 1, 2 or 4)", o->warps_per_block);
    if (o->flags & ~(SK_FLAG_SYMMETRIC | SK_FLAG_INCREMENTS | SK_FLAG_UNBIASED | SK_FLAG_NO_SORT | SK_FLAG_TIME_KERNEL |
                     SK_FLAG_STRIP_PIPELINE | SK_FLAG_NO_STRIP_PIPELINE | SK_FLAG_NO_TILED_M | SK_FLAG_CHECKPOINT |
                     SK_FLAG_NO_TC))
        return fail(SK_ERR_INVALID_ARG, "unknown flag bits 0x%x", o->flags);
    if ((o->flags & SK_FLAG_STRIP_PIPELINE) && (o->flags & SK_FLAG_NO_STRIP_PIPELINE))
        return fail(SK_ERR_INVALID_ARG, "SK_FLAG_STRIP_PIPELINE and SK_FLAG_NO_STRIP_PIPELINE together");
    return SK_OK;
}

// allow_coop: the caller launches p.kern itself with p.threads (the plain forward); adjoint
// plans reuse this layout with their own one-warp-per-pair kernels and pass false.  tape: the
// forward records a tape (one warp per pair; its own kernels for the approximation scheme).
int plan_forward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                 int mode, int64_t npairs, Plan& p, bool allow_coop = false, bool tape = false) {
    int rc;
    if ((rc = check_options(o, d, dtype)) != SK_OK) return rc;
    if ((rc = check_paths(X, "X", d)) != SK_OK) return rc;
    if ((rc = check_paths(Y, "Y", d)) != SK_OK) return rc;
    const int lam = o->dyadic;
    // (max_len << lam) > kMaxRefined, written so that no shift can overflow for any max_len
    if (X->max_len > (kMaxRefined >> lam) || Y->max_len > (kMaxRefined >> lam))
        return fail(SK_ERR_UNSUPPORTED, "max_len << dyadic exceeds %d", kMaxRefined);
    if (mode == kGramUpper) {
        if (X->rows != Y->rows || X->offsets != Y->offsets || X->count != Y->count)
            return fail(SK_ERR_INVALID_ARG, "SK_FLAG_SYMMETRIC needs Y to describe the same paths as X");
    }
    p.T = (o->compute == SK_COMPUTE_F32) ? 1 : 0;
    const int vw = p.T ? 4 : 2;
    p.nvec = (d + vw - 1) / vw;
    p.dpad = p.nvec * vw;
    p.mode = mode;
    p.npairs = npairs;
    p.same_xy = (X->rows == Y->rows && X->offsets == Y->offsets && X->count == Y->count &&
                 X->rows_total == Y->rows_total);
    if (npairs > 0x7fffffffLL) return fail(SK_ERR_UNSUPPORTED, "more than 2^31-1 pairs in one call");

    const bool poly = o->scheme == SK_POLY_APPROX || o->scheme == SK_POLY_INTERP;
    int width = 1;  // values handed from strip to strip per refined column
    // Tiled M (FP32 polynomial schemes): with wide increments (padded d >= 12) a cell that forms M
    // from two increment rows is bound by those loads; each warp builds a strip's M at once
    // instead (produce_m_strip).
    const bool mt_eligible = poly && p.T == 1 && p.dpad >= 12;
    p.mtile = mt_eligible && !(o->flags & SK_FLAG_NO_TILED_M);
    auto kernel_for = [&](bool coop) -> const void* {
        return poly ? fwd_poly_kernel_ptr(p.T, o->scheme == SK_POLY_INTERP, o->degree, coop, p.mtile, tape)
                    : fwd_fd_kernel_ptr(p.T, o->scheme == SK_FD2 ? 2 : o->scheme == SK_FD_IMPLICIT ? 3 : 1, lam, coop, tape);
    };
    p.kern = kernel_for(false);
    if (poly) {
        const int hw = p.T ? 4 : 2;  // hand-off entries are padded to whole 16-byte vectors
        width = (o->degree + 1 + hw - 1) / hw * hw;
    }
    if (!p.kern) return fail(SK_ERR_UNSUPPORTED, "no kernel for scheme %d order %d compute %d", o->scheme, o->degree, o->compute);
    // Launch shape.  Explicit requests (warps_per_block, the strip-pipeline flags) win; otherwise a
    // shape that sigkernel_autotune measured for this shape of call; otherwise the defaults.
    int wpb_req = 0, pipe_req = 0;  // pipe_req: 1 strip pipeline, -1 none, 0 the default rule
    if (allow_coop) {
        wpb_req = o->warps_per_block;
        if (o->flags & SK_FLAG_STRIP_PIPELINE) pipe_req = 1;
        if (o->flags & SK_FLAG_NO_STRIP_PIPELINE) pipe_req = -1;
    }
    int dev = 0, sms = 0, per_sm = 0;
    SK_CUDA(cudaGetDevice(&dev));
    if (allow_coop && wpb_req == 0 && pipe_req == 0 && !(o->flags & SK_FLAG_NO_TILED_M)) {
        const TuneKey key = tune_key(dev, X, Y, o, p.dpad, mode, npairs);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            wpb_req = it->second.wpb;
            pipe_req = it->second.pipe;
            if (it->second.mt < 0 && p.mtile) {
                p.mtile = false;
                p.kern = kernel_for(false);
            }
        }
    }
    p.threads = (wpb_req ? wpb_req : kFwdWarps) * 32;
    p.coop = false;
    p.coop_min_strips = 0;
    p.grid_bpp = 0;
    const int esize = p.T ? 4 : 8;
    p.smem_x = 0;
    auto xsmem = [&](int threads) { return p.mtile ? (threads / 32) * 32 * p.dpad * esize : 0; };
    auto occupancy = [&](const void* k, int threads, int* per) -> int {
        const int sm = xsmem(threads);
        if (sm > 48 * 1024) SK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k, threads, sm));
        return SK_OK;
    };
    SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if ((rc = occupancy(p.kern, p.threads, &per_sm)) != SK_OK) return rc;
    if (per_sm < 1) per_sm = 1;
    // Strip pipeline: a pair of many strips swept by one warp is a serial chain of
    // nstrips x cols steps; when the batch cannot fill the GPU with one warp per pair, long pairs
    // are swept by blocks of kCoopWarps warps instead (one strip per warp, pipelined).
    if (allow_coop && pipe_req >= 0) {
        const int rows_per_lane = poly ? 1 : (lam < 4 ? (1 << lam) : 16);
        // rows of the longest X path: its increments (one fewer than its points in points mode)
        const int64_t max_rows = std::max<int64_t>(X->max_len - ((o->flags & SK_FLAG_INCREMENTS) ? 0 : 1), 1) << lam;
        const int64_t max_strips = ((max_rows / rows_per_lane) + 31) / 32;
        const bool forced = pipe_req > 0;
        const int64_t resident = static_cast<int64_t>(sms) * per_sm * (p.threads / 32);
        if (max_strips >= 2 && (forced || (max_strips >= 2 * kCoopWarps && npairs < 4 * resident))) {
            // Pipelined warps are all on the pipeline's critical path, so a strip's tiled-M build
            // delays the whole chain: per-cell M measured faster there (4096 pairs of 64..4096-point
            // paths, d = 16: 101 against 118 ms).
            const bool mt_one = p.mtile;
            p.mtile = false;
            const void* ck = kernel_for(true);
            int cper = 0;
            if (ck && (rc = occupancy(ck, kCoopWarps * 32, &cper)) != SK_OK) return rc;
            if (!(ck && cper >= 1)) p.mtile = mt_one;
            if (ck && cper >= 1) {
                p.kern = ck;
                p.coop = true;
                // once a batch is pipelined at all, every pair of two or more strips is (measured on
                // 4096 pairs of 64..4096-point paths: 101 ms against 197 ms with only pairs of
                // 2 kCoopWarps strips or more)
                p.coop_min_strips = 2;
                p.threads = kCoopWarps * 32;
                per_sm = cper;
                // Few long pairs: one block per pair would leave SMs idle, so each pair's ring of
                // warps spans several co-resident blocks (no more than its strips can use).  A
                // step costs several times more there (GPU-scope hand-off), so the ring must
                // spread over at least kGridMinBlocks blocks: 1 pair of 16385-point paths ran
                // 5.5x faster, 8 pairs of 4097 points 1.4x, but 32 pairs of 2049 points (4 blocks
                // each) 1.6x slower and 64 pairs of 1025 points (2 each) 2.8x slower.
                const int64_t rblocks = static_cast<int64_t>(sms) * cper;
                if (poly && npairs > 0 && max_strips >= kGridMinBlocks * kCoopWarps) {
                    const int64_t bpp = std::min<int64_t>(rblocks / npairs, (max_strips + kCoopWarps - 1) / kCoopWarps);
                    if (bpp >= kGridMinBlocks) p.grid_bpp = static_cast<int>(bpp);
                }
            }
        }
    }
    // Tensor-core M: in place of the per-cell or tiled M, the FP32 approximation scheme's
    // one-warp-per-pair sweep reads each cell's M from a buffer that a tcgen05 GEMM fills per chunk
    // of items (sk_m_tc.cu), for padded widths 8..32 (d from 5 to 32).  At d = 8 it took the
    // 128 x 128 Gram's plain forward from 10.62 to 9.02 ms (the M kernel included) and its tape
    // forward from 12.31 to 12.18 ms.  Off with SK_FLAG_NO_TC, for the interpolation scheme, for
    // the strip pipeline, and when even one wave of resident warps would need more than twice
    // kMxBudget.
    p.mx = false;
    p.kp = p.dpad <= 16 ? 16 : 32;
    p.xt_nblk = static_cast<int>(((X->max_len << lam) + 127) / 128);
    p.yt_nblk = static_cast<int>(((Y->max_len << lam) + 127) / 128);
    p.mx_stride = 0;
    p.mx_chunk = npairs;
    const bool mt_chosen = p.mtile;
    if (p.T == 1 && o->scheme == SK_POLY_APPROX && p.dpad >= 8 && p.dpad <= 32 && !p.coop &&
        !(o->flags & SK_FLAG_NO_TC)) {
        const void* km = fwd_poly_kernel_ptr(p.T, false, o->degree, false, false, tape, true);
        if (km) {
            const int64_t pts = (o->flags & SK_FLAG_INCREMENTS) ? 0 : 1;
            const int64_t rmax = std::max<int64_t>(X->max_len - pts, 1) << lam;
            const int64_t cmax = std::max<int64_t>(Y->max_len - pts, 1) << lam;
            const int64_t nsteps = ((rmax + 31) / 32 - 1) * std::max<int64_t>(cmax, 32) + 31 + cmax;
            // groups of four warp steps, 32 lanes x float4 each
            const int64_t stride = static_cast<int64_t>(align256(static_cast<size_t>((nsteps + 3) / 4) * 32 * 16));
            int mper = 0;
            p.mtile = false;  // no x-row staging for this kernel
            if ((rc = occupancy(km, p.threads, &mper)) != SK_OK) return rc;
            if (mper < 1) mper = 1;
            const int64_t resident = static_cast<int64_t>(sms) * mper * (p.threads / 32);
            int64_t chunk = npairs;
            if (static_cast<size_t>(npairs) * stride > kMxBudget) {
                chunk = static_cast<int64_t>(kMxBudget / static_cast<size_t>(stride));
                if (chunk >= resident) chunk -= chunk % resident;
                else if (static_cast<size_t>(resident) * stride <= 2 * kMxBudget) chunk = resident;
                else chunk = 0;
            }
            if (chunk > 0) {
                p.mx = true;
                p.kern = km;
                per_sm = mper;
                p.mx_stride = stride;
                p.mx_chunk = std::max<int64_t>(std::min(chunk, npairs), 1);
            } else {
                p.mtile = mt_chosen;
            }
        }
    }
    const int wpb = p.threads / 32;
    int64_t want = p.coop ? (p.grid_bpp > 0 ? npairs * p.grid_bpp : npairs) : (npairs + wpb - 1) / wpb;
    int64_t cap = static_cast<int64_t>(sms) * per_sm;
    p.blocks = static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
    p.buf_cols = (Y->max_len << lam) + 1;
    p.slot_bytes = static_cast<int64_t>(align256(static_cast<size_t>(p.buf_cols * width * esize + p.buf_cols * 4)));
    p.smem_x = xsmem(p.threads);
    p.mtile_cols = std::max<int64_t>(Y->max_len << lam, 1);
    p.mtile_off = p.slot_bytes;
    if (p.mtile) p.slot_bytes += static_cast<int64_t>(align256(static_cast<size_t>(2 * 32 * p.mtile_cols * esize)));

    size_t off = 0;
    p.off_incx = off;
    off += align256(static_cast<size_t>(X->rows_total) * p.dpad * esize);
    p.off_incy = p.same_xy ? p.off_incx : off;
    if (!p.same_xy) off += align256(static_cast<size_t>(Y->rows_total) * p.dpad * esize);
    p.off_queue = off;
    off += 256;
    p.off_hist = off;
    off += align256(2 * 65 * sizeof(unsigned int));
    p.off_order = off;
    off += align256(static_cast<size_t>(npairs) * sizeof(int32_t));
    p.off_scratch = off;
    off += static_cast<size_t>(p.blocks) * wpb * static_cast<size_t>(p.slot_bytes);
    p.off_gprog = off;
    if (p.grid_bpp > 0) off += align256(static_cast<size_t>(p.blocks) * wpb * sizeof(int));
    p.off_xt = p.off_yt = p.off_mx = off;
    if (p.mx) {
        p.off_xt = off;
        off += align256(m_operand_bytes(p.kp, X->count, p.xt_nblk));
        p.off_yt = p.same_xy ? p.off_xt : off;
        if (!p.same_xy) off += align256(m_operand_bytes(p.kp, Y->count, p.yt_nblk));
        p.off_mx = off;
        off += static_cast<size_t>(p.mx_chunk) * static_cast<size_t>(p.mx_stride);
    }
    p.total = off + 256;
    return SK_OK;
}

template <typename T>
int launch_increments(const sk_paths* S, int32_t d, int32_t dtype, int inc_mode, int dpad, void* out,
                      cudaStream_t st) {
    if (S->count == 0) return SK_OK;
    int blocks = static_cast<int>(S->count < 65535 ? S->count : 65535);
    T* o = static_cast<T*>(out);
    switch (dtype) {
        case SK_F64:
            increments_kernel<double, T><<<blocks, 128, 0, st>>>(static_cast<const double*>(S->rows), S->offsets,
                                                                 S->count, S->rows_total, S->max_len, d, dpad, inc_mode, o);
            break;
        case SK_F32:
            increments_kernel<float, T><<<blocks, 128, 0, st>>>(static_cast<const float*>(S->rows), S->offsets,
                                                                S->count, S->rows_total, S->max_len, d, dpad, inc_mode, o);
            break;
        default:
            increments_kernel<__nv_bfloat16, T><<<blocks, 128, 0, st>>>(
                static_cast<const __nv_bfloat16*>(S->rows), S->offsets, S->count, S->rows_total, S->max_len, d, dpad,
                inc_mode, o);
            break;
    }
    SK_CUDA(cudaGetLastError());
    return SK_OK;
}

// Tape of the forward pass (polynomial schemes): [npairs] int exponents of k_hat, then one
// fixed-stride block per work item of nsteps_max x 32 lanes x tape_row<T>(N, interp) elements.
struct TapePlan {
    size_t ek_bytes, stride, total;
    int64_t nsteps;  // warp steps of the longest item
    int64_t nsteps_c;  // FD: steps of the coarse-grid schedule of the dk/dM buffer
};

bool is_fd(const sk_options* o) {
    return o->scheme == SK_FD1 || o->scheme == SK_FD2 || o->scheme == SK_FD_IMPLICIT;
}
int fd_order(const sk_options* o) { return o->scheme == SK_FD2 ? 2 : o->scheme == SK_FD_IMPLICIT ? 3 : 1; }

int plan_tape(const sk_paths* X, const sk_paths* Y, const sk_options* o, int T, int64_t npairs, TapePlan& t) {
    const int lam = o->dyadic;
    // grid rows and columns of the longest paths: their increments (one fewer than their points)
    const int64_t pts = (o->flags & SK_FLAG_INCREMENTS) ? 0 : 1;
    const int64_t lx = std::max<int64_t>(X->max_len - pts, 1), ly = std::max<int64_t>(Y->max_len - pts, 1);
    int64_t rows = lx << lam;
    const int64_t cols = ly << lam;
    int row;
    if (is_fd(o)) {
        // FD: each lane sweeps 2^lambda node rows (one coarse row) over the refined columns
        if (lam > 4) return fail(SK_ERR_UNSUPPORTED, "the FD adjoint supports dyadic orders 0..4");
        rows = lx;
        row = fd_tape_row_elems(T, lam);
    } else {
        const bool interp = o->scheme == SK_POLY_INTERP;
        row = T ? tape_row<float>(o->degree, interp) : tape_row<double>(o->degree, interp);
    }
    const int64_t nsteps = ((rows + 31) / 32 - 1) * std::max<int64_t>(cols, 32) + 31 + cols;
    t.nsteps_c = ((lx + 31) / 32 - 1) * std::max<int64_t>(ly, 32) + 31 + ly;
    const int esize = T ? 4 : 8;
    t.nsteps = nsteps;
    t.ek_bytes = align256(static_cast<size_t>(npairs) * sizeof(int));
    t.stride = align256(static_cast<size_t>(nsteps) * 32 * row * esize);
    t.total = t.ek_bytes + static_cast<size_t>(npairs) * t.stride;
    return SK_OK;
}

int run_forward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o, int mode,
                const int64_t* pa, const int64_t* pb, int64_t npairs, double* out, int64_t ldo, void* ws,
                size_t ws_bytes, void* stream, void* tape = nullptr, size_t tape_bytes = 0, int64_t item_base = 0) {
    Plan p;
    int rc = plan_forward(X, Y, d, dtype, o, mode, npairs, p, tape == nullptr, tape != nullptr);
    if (rc != SK_OK) return rc;
    TapePlan tp{0, 0, 0, 0};
    if (tape) {
        if ((rc = plan_tape(X, Y, o, p.T, npairs, tp)) != SK_OK) return rc;
        if (tape_bytes < tp.total) return fail(SK_ERR_WORKSPACE, "tape %zu bytes < %zu required", tape_bytes, tp.total);
        if (reinterpret_cast<uintptr_t>(tape) % 256) return fail(SK_ERR_INVALID_ARG, "tape must be 256-byte aligned");
    }
    if (npairs == 0) return SK_OK;
    if (!out) return fail(SK_ERR_INVALID_ARG, "output pointer is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, p.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < p.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, p.total);
    }
    char* base = static_cast<char*>(ws);
    base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) / 256 * 256);
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    rc = p.T ? launch_increments<float>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st)
             : launch_increments<double>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st);
    if (rc == SK_OK && !p.same_xy)
        rc = p.T ? launch_increments<float>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st)
                 : launch_increments<double>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st);
    if (rc != SK_OK) return rc;

    Launch L;
    memset(&L, 0, sizeof(L));
    L.item_base = item_base;
    L.X = PathSet{base + p.off_incx, X->offsets, X->count, X->max_len, X->rows_total};
    L.Y = PathSet{base + p.off_incy, Y->offsets, Y->count, Y->max_len, Y->rows_total};
    L.nvec = p.nvec;
    L.dpad = p.dpad;
    L.inc_mode = inc_mode;
    L.lam = o->dyadic;
    L.mode = mode;
    L.npairs = npairs;
    L.pair_a = pa;
    L.pair_b = pb;
    L.queue = reinterpret_cast<unsigned int*>(base + p.off_queue);
    L.out = out;
    L.ldo = ldo;
    L.scratch = base + p.off_scratch;
    L.scratch_stride = p.slot_bytes;
    L.tau = 1.0f;
    L.order = nullptr;
    L.tape = tape ? static_cast<char*>(tape) + tp.ek_bytes : nullptr;
    L.tape_stride = static_cast<int64_t>(tp.stride);
    L.tape_ek = tape ? static_cast<int*>(tape) : nullptr;
    L.coop_min_strips = p.coop_min_strips;
    L.grid_bpp = p.grid_bpp;
    L.gprog = p.grid_bpp > 0 ? reinterpret_cast<int*>(base + p.off_gprog) : nullptr;
    if (p.grid_bpp > 0) SK_CUDA(cudaMemsetAsync(L.gprog, 0, static_cast<size_t>(p.blocks) * (p.threads / 32) * sizeof(int), st));
    L.mtile = p.mtile ? 1 : 0;
    L.mtile_cols = static_cast<int32_t>(p.mtile_cols);
    L.mtile_off = p.mtile_off;
    L.wait_limit = g_wait_limit.load(std::memory_order_relaxed);
    L.mx = nullptr;
    L.mx_stride = 0;
    int sms = 0;
    if (p.mx) {
        int dev = 0;
        SK_CUDA(cudaGetDevice(&dev));
        SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SK_CUDA(launch_m_operands(p.kp, L.X, inc_mode, L.lam, p.dpad, p.xt_nblk, base + p.off_xt, st));
        if (!p.same_xy) SK_CUDA(launch_m_operands(p.kp, L.Y, inc_mode, L.lam, p.dpad, p.yt_nblk, base + p.off_yt, st));
        L.mx = reinterpret_cast<const float*>(base + p.off_mx);
        L.mx_stride = p.mx_stride;
    }
    int64_t buf_cols = p.buf_cols;
    const int smem = p.smem_x;  // tiled-M x rows
    if (smem > 48 * 1024) SK_CUDA(cudaFuncSetAttribute(p.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const bool timed = (o->flags & SK_FLAG_TIME_KERNEL) != 0;
    if (timed) {
        if (!t_ev0) SK_CUDA(cudaEventCreate(&t_ev0));
        if (!t_ev1) SK_CUDA(cudaEventCreate(&t_ev1));
    }
    // Items in chunks of p.mx_chunk (one chunk unless M is precomputed): each chunk is a launch of
    // its own over items c0 .. c0 + n - 1 (pair lists, outputs and tape offset by c0; a Gram's
    // items by item_base), with its own queue and order.
    const int wpb = p.threads / 32;
    for (int64_t c0 = 0; c0 < npairs; c0 += p.mx_chunk) {
        const int64_t n = std::min(p.mx_chunk, npairs - c0);
        Launch C = L;
        C.npairs = n;
        if (c0 > 0) {
            if (mode == kPairsList) {
                C.pair_a = pa + c0;
                C.pair_b = pb + c0;
                C.out = out + c0;
            } else {
                C.item_base = item_base + c0;
            }
            if (tape) {
                C.tape = static_cast<char*>(L.tape) + c0 * L.tape_stride;
                C.tape_ek = L.tape_ek + c0;
            }
        }
        SK_CUDA(cudaMemsetAsync(base + p.off_queue, 0, 256 + align256(2 * 65 * sizeof(unsigned int)), st));
        if (!(o->flags & SK_FLAG_NO_SORT) && n > 1) {
            unsigned int* hist = reinterpret_cast<unsigned int*>(base + p.off_hist);
            int32_t* order = reinterpret_cast<int32_t*>(base + p.off_order);
            int sb = static_cast<int>((n + 255) / 256);
            if (sb > 4096) sb = 4096;
            sched_hist_kernel<<<sb, 256, 0, st>>>(C, hist);
            sched_scan_kernel<<<1, 32, 0, st>>>(hist, hist + 65);
            sched_scatter_kernel<<<sb, 256, 0, st>>>(C, hist + 65, order);
            SK_CUDA(cudaGetLastError());
            C.order = order;
        }
        if (timed && c0 == 0) SK_CUDA(cudaEventRecord(t_ev0, st));
        if (p.mx)
            SK_CUDA(launch_m_tc(p.kp, C, base + p.off_xt, base + p.off_yt, p.xt_nblk, p.yt_nblk,
                                reinterpret_cast<float*>(base + p.off_mx), p.mx_stride, sms, st));
        void* args[] = {&C, &buf_cols};
        if (p.grid_bpp > 0) {
            // the blocks of a pair wait on one another: launch them co-resident
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(p.blocks);
            cfg.blockDim = dim3(p.threads);
            cfg.dynamicSmemBytes = static_cast<size_t>(smem);
            cfg.stream = st;
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeCooperative;
            attr.val.cooperative = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            SK_CUDA(cudaLaunchKernelExC(&cfg, p.kern, args));
        } else {
            const int64_t want = p.coop ? n : (n + wpb - 1) / wpb;
            const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, p.blocks)));
            SK_CUDA(cudaLaunchKernel(p.kern, dim3(blocks), dim3(p.threads), args, smem, st));
        }
    }
    if (timed) {
        SK_CUDA(cudaEventRecord(t_ev1, st));
        t_timed = true;
    }
    SK_CUDA(owned.release());
    return SK_OK;
}

int64_t gram_items(const sk_paths* X, const sk_paths* Y, bool sym) {
    return sym ? X->count * (X->count + 1) / 2 : X->count * Y->count;
}

// ------------------------------------------------------------------------------------------
// Backward: d k / d increments (FP64, accumulated with atomics) -> d k / d rows.
// ------------------------------------------------------------------------------------------
__global__ void inc_to_row_grad_kernel(const double* __restrict__ ginc, const int64_t* __restrict__ off,
                                       int64_t count, int64_t rows_total, int64_t max_len, int d, int dpad,
                                       int inc_mode, double* __restrict__ grad) {
    for (int64_t a = blockIdx.x; a < count; a += gridDim.x) {
        const int64_t r0 = off[a], r1 = off[a + 1], n = r1 - r0;
        if (r0 < 0 || r1 > rows_total || n < (inc_mode ? 0 : 1) || n > max_len) continue;
        for (int64_t idx = threadIdx.x; idx < n * d; idx += blockDim.x) {
            const int64_t p = idx / d;
            const int c = static_cast<int>(idx - p * d);
            double v;
            if (inc_mode) {
                v = ginc[(r0 + p) * dpad + c];
            } else {  // x_p enters dx_{p-1} = x_p - x_{p-1} with +1 and dx_p = x_{p+1} - x_p with -1
                v = (p >= 1 ? ginc[(r0 + p - 1) * dpad + c] : 0.0) - (p + 1 < n ? ginc[(r0 + p) * dpad + c] : 0.0);
            }
            grad[(r0 + p) * d + c] += v;
        }
    }
}

struct BwdPlan {
    Plan f;                    // forward plan (increments, queue, order offsets)
    const void* kern;
    int K, dmax, stack_bytes, smem_bytes;
    int64_t cols_max, strips_max, strip_steps;
    int64_t off_fbuf, off_fexp, off_rbuf, off_rexp, off_ybar, slot_bytes;
    size_t off_gincx, off_gincy, off_scratch, total;
};

int plan_backward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o, int mode,
                  int64_t npairs, BwdPlan& b) {
    int rc = plan_forward(X, Y, d, dtype, o, mode, npairs, b.f);
    if (rc != SK_OK) return rc;
    if (o->scheme != SK_POLY_APPROX)
        return fail(SK_ERR_UNSUPPORTED, "sigkernel_backward supports the polynomial approximation scheme");
    const Plan& p = b.f;
    b.dmax = p.dpad <= 8 ? 8 : (p.dpad <= 32 ? 32 : 0);
    if (!b.dmax) return fail(SK_ERR_UNSUPPORTED, "sigkernel_backward supports d <= 32");
    b.kern = p.T ? bwd_approx_ptr_f32(o->degree, b.dmax, &b.stack_bytes)
                 : bwd_approx_ptr_f64(o->degree, b.dmax, &b.stack_bytes);
    if (!b.kern) return fail(SK_ERR_UNSUPPORTED, "no adjoint kernel for order %d", o->degree);
    b.K = p.T ? bwd_segment_f32() : bwd_segment_f64();
    b.smem_bytes = kFwdWarps * (b.stack_bytes + (p.T ? bwd_xacc_bytes<float>(p.dpad) : bwd_xacc_bytes<double>(p.dpad)));
    const int lam = o->dyadic, esize = p.T ? 4 : 8, N = o->degree;
    const int64_t rows_max = std::max<int64_t>(X->max_len << lam, 1);
    b.cols_max = std::max<int64_t>(Y->max_len << lam, 1);
    b.strips_max = (rows_max + 31) / 32;
    b.strip_steps = b.cols_max + 31;  // warp steps of one strip
    int64_t off = 0;                  // the strip tape: one tape step per warp step of a strip
    off += b.strip_steps * 32 * static_cast<int64_t>(p.T ? tape_row<float>(N, false) * 4 : tape_row<double>(N, false) * 8);
    off = static_cast<int64_t>(align256(off));
    b.off_fbuf = off;
    off += static_cast<int64_t>(align256(std::max<int64_t>(b.strips_max - 1, 1) * b.cols_max * (N + 1) * esize));
    b.off_fexp = off;
    off += static_cast<int64_t>(align256(std::max<int64_t>(b.strips_max - 1, 1) * b.cols_max * 4));
    b.off_rbuf = off;
    off += static_cast<int64_t>(align256(b.cols_max * (N + 1) * esize));
    b.off_rexp = off;
    off += static_cast<int64_t>(align256(b.cols_max * 4));
    b.off_ybar = off;  // the pair's dk/dy column sums in T, [coarse column][dpad]
    off += static_cast<int64_t>(align256(std::max<int64_t>(Y->max_len, 1) * p.dpad * esize));
    b.slot_bytes = off;
    int dev = 0, sms = 0, per_sm = 0;
    SK_CUDA(cudaGetDevice(&dev));
    SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SK_CUDA(cudaFuncSetAttribute(b.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, b.smem_bytes));
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b.kern, p.threads, b.smem_bytes));
    if (per_sm < 1) return fail(SK_ERR_UNSUPPORTED, "adjoint kernel does not fit an SM (%d bytes shared)", b.smem_bytes);
    const int64_t want = (npairs + kFwdWarps - 1) / kFwdWarps;
    const int64_t cap = static_cast<int64_t>(sms) * per_sm;
    b.f.blocks = static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
    // workspace: forward parts up to the scratch, then gradient accumulators, then the slots
    size_t o2 = p.off_scratch;
    b.off_gincx = o2;
    o2 += align256(static_cast<size_t>(X->rows_total) * p.dpad * sizeof(double));
    b.off_gincy = p.same_xy ? b.off_gincx : o2;
    if (!p.same_xy) o2 += align256(static_cast<size_t>(Y->rows_total) * p.dpad * sizeof(double));
    b.off_scratch = o2;
    o2 += static_cast<size_t>(b.f.blocks) * kFwdWarps * static_cast<size_t>(b.slot_bytes);
    b.total = o2 + 256;
    return SK_OK;
}

// Runs the adjoint for one call; gradients w.r.t. increments are ADDED to gincX / gincY (which
// may alias).  `base` is the aligned workspace laid out by plan_backward.
int launch_backward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o, int mode,
                    const int64_t* pa, const int64_t* pb, int64_t npairs, const double* gout, int64_t ldo,
                    const BwdPlan& b, char* base, double* gincX, double* gincY, cudaStream_t st) {
    const Plan& p = b.f;
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    int rc = p.T ? launch_increments<float>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st)
                 : launch_increments<double>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st);
    if (rc == SK_OK && !p.same_xy)
        rc = p.T ? launch_increments<float>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st)
                 : launch_increments<double>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st);
    if (rc != SK_OK) return rc;
    BwdParams B;
    memset(&B, 0, sizeof(B));
    Launch& L = B.L;
    L.X = PathSet{base + p.off_incx, X->offsets, X->count, X->max_len, X->rows_total};
    L.Y = PathSet{base + p.off_incy, Y->offsets, Y->count, Y->max_len, Y->rows_total};
    L.nvec = p.nvec;
    L.dpad = p.dpad;
    L.inc_mode = inc_mode;
    L.lam = o->dyadic;
    L.mode = mode;
    L.npairs = npairs;
    L.pair_a = pa;
    L.pair_b = pb;
    L.queue = reinterpret_cast<unsigned int*>(base + p.off_queue);
    L.out = nullptr;
    L.ldo = ldo;
    L.scratch = base + b.off_scratch;
    L.scratch_stride = b.slot_bytes;
    L.tau = 1.0f;
    L.order = nullptr;
    B.gout = gout;
    B.gincX = gincX;
    B.gincY = gincY;
    B.cols_max = b.cols_max;
    B.strips_max = b.strips_max;
    B.off_fbuf = b.off_fbuf;
    B.off_fexp = b.off_fexp;
    B.off_rbuf = b.off_rbuf;
    B.off_rexp = b.off_rexp;
    B.off_ybar = b.off_ybar;
    SK_CUDA(cudaMemsetAsync(base + p.off_queue, 0, 256 + align256(2 * 65 * sizeof(unsigned int)), st));
    if (!(o->flags & SK_FLAG_NO_SORT) && npairs > 1) {
        unsigned int* hist = reinterpret_cast<unsigned int*>(base + p.off_hist);
        int32_t* order = reinterpret_cast<int32_t*>(base + p.off_order);
        int sb = static_cast<int>(std::min<int64_t>((npairs + 255) / 256, 4096));
        sched_hist_kernel<<<sb, 256, 0, st>>>(L, hist);
        sched_scan_kernel<<<1, 32, 0, st>>>(hist, hist + 65);
        sched_scatter_kernel<<<sb, 256, 0, st>>>(L, hist + 65, order);
        SK_CUDA(cudaGetLastError());
        L.order = order;
    }
    void* args[] = {&B};
    const bool timed = (o->flags & SK_FLAG_TIME_KERNEL) != 0;
    if (timed) {
        if (!t_ev0) SK_CUDA(cudaEventCreate(&t_ev0));
        if (!t_ev1) SK_CUDA(cudaEventCreate(&t_ev1));
        SK_CUDA(cudaEventRecord(t_ev0, st));
    }
    SK_CUDA(cudaLaunchKernel(b.kern, dim3(p.blocks), dim3(p.threads), args, b.smem_bytes, st));
    if (timed) {
        SK_CUDA(cudaEventRecord(t_ev1, st));
        t_timed = true;
    }
    return SK_OK;
}

int convert_grad(const sk_paths* S, int32_t d, int dpad, int inc_mode, const double* ginc, double* grad,
                 cudaStream_t st) {
    if (!grad || S->count == 0) return SK_OK;
    int blocks = static_cast<int>(S->count < 65535 ? S->count : 65535);
    inc_to_row_grad_kernel<<<blocks, 128, 0, st>>>(ginc, S->offsets, S->count, S->rows_total, S->max_len, d, dpad,
                                                   inc_mode, grad);
    SK_CUDA(cudaGetLastError());
    return SK_OK;
}

int run_backward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                 const int64_t* pa, const int64_t* pb, int64_t npairs, const double* gout, double* gX, double* gY,
                 void* ws, size_t ws_bytes, void* stream) {
    const bool gram = (pa == nullptr);
    const bool sym = gram && (o->flags & SK_FLAG_SYMMETRIC);
    const int mode = gram ? (sym ? kGramUpper : kGramFull) : kPairsList;
    if (gram) npairs = gram_items(X, Y, sym);
    BwdPlan b;
    int rc = plan_backward(X, Y, d, dtype, o, mode, npairs, b);
    if (rc != SK_OK) return rc;
    if (b.f.same_xy && gY && gY != gX)
        return fail(SK_ERR_INVALID_ARG, "X and Y are the same paths: pass grad_Y = NULL or grad_Y = grad_X");
    if (npairs == 0) return SK_OK;
    if (!gout) return fail(SK_ERR_INVALID_ARG, "grad_out is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, b.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < b.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, b.total);
    }
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) / 256 * 256);
    double* gincX = reinterpret_cast<double*>(base + b.off_gincx);
    double* gincY = reinterpret_cast<double*>(base + b.off_gincy);
    SK_CUDA(cudaMemsetAsync(gincX, 0, static_cast<size_t>(X->rows_total) * b.f.dpad * sizeof(double), st));
    if (!b.f.same_xy)
        SK_CUDA(cudaMemsetAsync(gincY, 0, static_cast<size_t>(Y->rows_total) * b.f.dpad * sizeof(double), st));
    rc = launch_backward(X, Y, d, dtype, o, mode, pa, pb, npairs, gout, Y->count, b, base, gincX, gincY, st);
    if (rc != SK_OK) return rc;
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    if ((rc = convert_grad(X, d, b.f.dpad, inc_mode, gincX, gX, st)) != SK_OK) return rc;
    if (!b.f.same_xy && (rc = convert_grad(Y, d, b.f.dpad, inc_mode, gincY, gY, st)) != SK_OK) return rc;
    SK_CUDA(owned.release());
    return SK_OK;
}


// ------------------------------------------------------------------------------------------
// Backward from a forward tape.
// ------------------------------------------------------------------------------------------
struct TapeBwdPlan {
    Plan f;
    TapePlan t;
    const void* kern;
    const void* ckern;
    int smem_bytes, cblocks, csmem, cC;
    int64_t cols_max, off_rbuf, off_rexp, slot_bytes, mb_stride, acc_bytes;
    // tensor-core contraction: operand coordinates (16 or 32), 128-row blocks of the longest X and
    // Y paths, operand tiles in the workspace, CTAs
    bool tc;
    int tcN, nrb, ncb, tc_sms;
    size_t off_xt, off_yt;
    size_t off_gincx, off_gincy, off_scratch, off_mbuf, total;
};

int plan_backward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o, int mode,
                       int64_t npairs, TapeBwdPlan& b) {
    int rc = plan_forward(X, Y, d, dtype, o, mode, npairs, b.f);
    if (rc != SK_OK) return rc;
    const Plan& p = b.f;
    if ((rc = plan_tape(X, Y, o, p.T, npairs, b.t)) != SK_OK) return rc;
    const bool interp = o->scheme == SK_POLY_INTERP;
    const bool fd = is_fd(o);
    b.kern = fd ? bwd_fd_tape_ptr(p.T, fd_order(o), o->dyadic)
                : (p.T ? bwd_tape_ptr_f32(o->degree, interp) : bwd_tape_ptr_f64(o->degree, interp));
    if (!b.kern) return fail(SK_ERR_UNSUPPORTED, "no adjoint kernel for order %d", o->degree);
    // contraction: every coordinate of a padded increment row in one pass up to 32 (8, 16 or 32)
    b.cC = p.dpad <= 8 ? 8 : (p.dpad <= 16 ? 16 : 32);
    b.ckern = p.T ? bwd_contract_ptr_f32(b.cC) : bwd_contract_ptr_f64(b.cC);
    const int step_bytes = 32 * (p.T ? tape_row<float>(o->degree, interp) * 4 : tape_row<double>(o->degree, interp) * 8);
    b.smem_bytes = kFwdWarps * (fd ? bwd_fd_ring_bytes(p.T, o->dyadic) : bwd_tape_warp_bytes(step_bytes));
    const int esize = p.T ? 4 : 8, N = fd ? 0 : o->degree;  // FD hands one value per column down
    b.cols_max = std::max<int64_t>(Y->max_len << o->dyadic, 1);
    b.off_rbuf = 0;
    int64_t off = static_cast<int64_t>(align256(b.cols_max * (N + 1) * esize));
    b.off_rexp = off;
    off += static_cast<int64_t>(align256(b.cols_max * 4));
    b.slot_bytes = off;
    // dk/dM buffer: the tape's [step][lane] grid of one element per cell
    // (plus the rows past an item's last step that the contraction's tiles may read)
    b.mb_stride = static_cast<int64_t>(align256(static_cast<size_t>((fd ? b.t.nsteps_c : b.t.nsteps) + kContractSlack) *
                                                32 * esize));
    // Tensor-core contraction (FP32, 8 < d <= 32): dk/dM as BF16 hi/lo tiles of 128 x 128 cells
    // instead, when the longest pair's sums fit one half of the tensor memory.
    {
        const int64_t pts = (o->flags & SK_FLAG_INCREMENTS) ? 0 : 1;
        // the FD adjoint writes dk/dM on the coarse grid (the contraction then runs at lambda = 0)
        const int clam = fd ? 0 : o->dyadic;
        const int64_t rmax = std::max<int64_t>(X->max_len - pts, 1) << clam;
        const int64_t cmax = std::max<int64_t>(Y->max_len - pts, 1) << clam;
        b.tcN = p.dpad <= 16 ? 16 : 32;
        b.nrb = static_cast<int>((rmax + 127) / 128);
        b.ncb = static_cast<int>((cmax + 127) / 128);
        b.tc = p.T == 1 && !(o->flags & SK_FLAG_NO_TC) && p.dpad > 8 && p.dpad <= 32 &&
               static_cast<int64_t>(b.nrb + b.ncb) * b.tcN <= 256;
        if (b.tc) b.mb_stride = static_cast<int64_t>(b.nrb) * b.ncb * 65536;
    }
    // contraction: per-warp rings and staged rows, then the block's column accumulator
    int cwarp = 0, cwin = 0;
    if (p.T) {
        cwarp = b.cC == 8 ? contract_warp_bytes<float, 8>() : b.cC == 16 ? contract_warp_bytes<float, 16>()
                                                                : contract_warp_bytes<float, 32>();
        cwin = b.cC == 8 ? contract_window<float, 8>() : b.cC == 16 ? contract_window<float, 16>()
                                                            : contract_window<float, 32>();
    } else {
        cwarp = b.cC == 8 ? contract_warp_bytes<double, 8>() : b.cC == 16 ? contract_warp_bytes<double, 16>()
                                                                 : contract_warp_bytes<double, 32>();
        cwin = b.cC == 8 ? contract_window<double, 8>() : b.cC == 16 ? contract_window<double, 16>()
                                                             : contract_window<double, 32>();
    }
    // the accumulator holds a window of at most cwin columns (fewer when the paths are shorter)
    b.acc_bytes = static_cast<int64_t>(b.cC) * esize * std::min<int64_t>(cwin, b.cols_max);
    b.csmem = kContractWarps * cwarp + static_cast<int>(b.acc_bytes);
    int dev = 0, sms = 0, per_sm = 0, cper_sm = 0;
    SK_CUDA(cudaGetDevice(&dev));
    SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SK_CUDA(cudaFuncSetAttribute(b.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, b.smem_bytes));
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b.kern, p.threads, b.smem_bytes));
    if (per_sm < 1) return fail(SK_ERR_UNSUPPORTED, "adjoint kernel does not fit an SM");
    SK_CUDA(cudaFuncSetAttribute(b.ckern, cudaFuncAttributeMaxDynamicSharedMemorySize, b.csmem));
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cper_sm, b.ckern, kContractWarps * 32,
                                                          static_cast<size_t>(b.csmem)));
    if (cper_sm < 1) return fail(SK_ERR_UNSUPPORTED, "contraction kernel does not fit an SM");
    b.tc_sms = sms;
    b.cblocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(npairs, static_cast<int64_t>(sms) * cper_sm)));
    const int64_t want = (npairs + kFwdWarps - 1) / kFwdWarps;
    b.f.blocks = static_cast<int>(std::max<int64_t>(1, std::min(want, static_cast<int64_t>(sms) * per_sm)));
    size_t o2 = p.off_scratch;
    b.off_gincx = o2;
    o2 += align256(static_cast<size_t>(X->rows_total) * p.dpad * sizeof(double));
    b.off_gincy = p.same_xy ? b.off_gincx : o2;
    if (!p.same_xy) o2 += align256(static_cast<size_t>(Y->rows_total) * p.dpad * sizeof(double));
    b.off_scratch = o2;
    o2 += static_cast<size_t>(b.f.blocks) * kFwdWarps * static_cast<size_t>(b.slot_bytes);
    o2 = align256(o2);
    b.off_mbuf = o2;
    o2 += static_cast<size_t>(npairs) * static_cast<size_t>(b.mb_stride);
    o2 = align256(o2);
    b.off_xt = b.off_yt = o2;
    if (b.tc) {
        o2 += align256(tc_operand_bytes(b.tcN, X->count, b.nrb));
        b.off_yt = p.same_xy ? b.off_xt : o2;
        if (!p.same_xy) o2 += align256(tc_operand_bytes(b.tcN, Y->count, b.ncb));
    }
    b.total = o2 + 256;
    return SK_OK;
}

// Adjoint from a tape over work items item_base .. item_base + npairs - 1 (Gram modes) or the
// given pair list: increments, ordering, the tape adjoint and the contraction; gradients with
// respect to increments are ADDED to gincX / gincY (which may alias).  `base` is the aligned
// workspace laid out by plan_backward_tape for npairs items.
int launch_backward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                         int mode, const int64_t* pa, const int64_t* pb, int64_t npairs, int64_t item_base,
                         const void* tape, const double* gout, int64_t ldo, const TapeBwdPlan& b, char* base,
                         double* gincX, double* gincY, cudaStream_t st) {
    const Plan& p = b.f;
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    int rc = p.T ? launch_increments<float>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st)
             : launch_increments<double>(X, d, dtype, inc_mode, p.dpad, base + p.off_incx, st);
    if (rc == SK_OK && !p.same_xy)
        rc = p.T ? launch_increments<float>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st)
                 : launch_increments<double>(Y, d, dtype, inc_mode, p.dpad, base + p.off_incy, st);
    if (rc != SK_OK) return rc;
    BwdParams B;
    memset(&B, 0, sizeof(B));
    Launch& L = B.L;
    L.X = PathSet{base + p.off_incx, X->offsets, X->count, X->max_len, X->rows_total};
    L.Y = PathSet{base + p.off_incy, Y->offsets, Y->count, Y->max_len, Y->rows_total};
    L.nvec = p.nvec;
    L.dpad = p.dpad;
    L.inc_mode = inc_mode;
    L.lam = o->dyadic;
    L.mode = mode;
    L.npairs = npairs;
    L.item_base = item_base;
    L.pair_a = pa;
    L.pair_b = pb;
    L.queue = reinterpret_cast<unsigned int*>(base + p.off_queue);
    L.ldo = ldo;
    L.scratch = base + b.off_scratch;
    L.scratch_stride = b.slot_bytes;
    L.tau = 1.0f;
    TapePlan tp;  // the tape as the forward laid it out for these npairs items
    if ((rc = plan_tape(X, Y, o, p.T, npairs, tp)) != SK_OK) return rc;
    L.tape = const_cast<char*>(static_cast<const char*>(tape)) + tp.ek_bytes;
    L.tape_stride = static_cast<int64_t>(tp.stride);
    L.tape_ek = const_cast<int*>(static_cast<const int*>(tape));
    B.gout = gout;
    B.gincX = gincX;
    B.gincY = gincY;
    B.cols_max = b.cols_max;
    B.off_rbuf = b.off_rbuf;
    B.off_rexp = b.off_rexp;
    B.mbuf = base + b.off_mbuf;
    B.mb_stride = b.mb_stride;
    B.acc_bytes = b.acc_bytes;
    if (b.tc) {  // dk/dM tiles for the tensor cores, and the transposed split increments
        B.gtile = 1;
        B.gt_ncb = b.ncb;
        B.xt = base + b.off_xt;
        B.yt = base + b.off_yt;
        B.xt_nblk = b.nrb;
        B.yt_nblk = p.same_xy ? b.nrb : b.ncb;
        const int clam = is_fd(o) ? 0 : L.lam;
        SK_CUDA(launch_tc_operands(b.tcN, L.X, inc_mode, clam, p.dpad, b.nrb, base + b.off_xt, st));
        if (!p.same_xy) SK_CUDA(launch_tc_operands(b.tcN, L.Y, inc_mode, clam, p.dpad, b.ncb, base + b.off_yt, st));
    }
    SK_CUDA(cudaMemsetAsync(base + p.off_queue, 0, 256, st));
    if (!(o->flags & SK_FLAG_NO_SORT) && npairs > 1) {
        unsigned int* hist = reinterpret_cast<unsigned int*>(base + p.off_hist);
        int32_t* order = reinterpret_cast<int32_t*>(base + p.off_order);
        SK_CUDA(cudaMemsetAsync(hist, 0, align256(2 * 65 * sizeof(unsigned int)), st));
        int sb = static_cast<int>(std::min<int64_t>((npairs + 255) / 256, 4096));
        sched_hist_kernel<<<sb, 256, 0, st>>>(L, hist);
        sched_scan_kernel<<<1, 32, 0, st>>>(hist, hist + 65);
        sched_scatter_kernel<<<sb, 256, 0, st>>>(L, hist + 65, order);
        SK_CUDA(cudaGetLastError());
        L.order = order;
    }
    void* args[] = {&B};
    const bool timed = (o->flags & SK_FLAG_TIME_KERNEL) != 0;
    if (timed) {
        if (!t_ev0) SK_CUDA(cudaEventCreate(&t_ev0));
        if (!t_ev1) SK_CUDA(cudaEventCreate(&t_ev1));
        SK_CUDA(cudaEventRecord(t_ev0, st));
    }
    SK_CUDA(cudaLaunchKernel(b.kern, dim3(p.blocks), dim3(p.threads), args, b.smem_bytes, st));
    if (timed) {
        SK_CUDA(cudaEventRecord(t_ev1, st));
        t_timed = true;
    }
    if (is_fd(o)) B.L.lam = 0;  // the FD adjoint wrote dk/dM for the coarse cells
    if (b.tc) SK_CUDA(launch_tc_contraction(b.tcN, B, b.nrb, b.tc_sms, st));
    else SK_CUDA(cudaLaunchKernel(b.ckern, dim3(b.cblocks), dim3(kContractWarps * 32), args,
                                  static_cast<size_t>(b.csmem), st));
    return SK_OK;
}

int run_backward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                      const int64_t* pa, const int64_t* pb, int64_t npairs, const void* tape, size_t tape_bytes,
                      const double* gout, double* gX, double* gY, void* ws, size_t ws_bytes, void* stream) {
    const bool gram = (pa == nullptr);
    const bool sym = gram && (o->flags & SK_FLAG_SYMMETRIC);
    const int mode = gram ? (sym ? kGramUpper : kGramFull) : kPairsList;
    if (gram) npairs = gram_items(X, Y, sym);
    TapeBwdPlan b;
    int rc = plan_backward_tape(X, Y, d, dtype, o, mode, npairs, b);
    if (rc != SK_OK) return rc;
    if (b.f.same_xy && gY && gY != gX)
        return fail(SK_ERR_INVALID_ARG, "X and Y are the same paths: pass grad_Y = NULL or grad_Y = grad_X");
    if (!tape || tape_bytes < b.t.total) return fail(SK_ERR_WORKSPACE, "tape missing or smaller than %zu bytes", b.t.total);
    if (npairs == 0) return SK_OK;
    if (!gout) return fail(SK_ERR_INVALID_ARG, "grad_out is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, b.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < b.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, b.total);
    }
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) / 256 * 256);
    const Plan& p = b.f;
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    double* gincX = reinterpret_cast<double*>(base + b.off_gincx);
    double* gincY = reinterpret_cast<double*>(base + b.off_gincy);
    SK_CUDA(cudaMemsetAsync(gincX, 0, static_cast<size_t>(X->rows_total) * p.dpad * sizeof(double), st));
    if (!p.same_xy) SK_CUDA(cudaMemsetAsync(gincY, 0, static_cast<size_t>(Y->rows_total) * p.dpad * sizeof(double), st));
    if ((rc = launch_backward_tape(X, Y, d, dtype, o, mode, pa, pb, npairs, 0, tape, gout, Y->count, b, base, gincX,
                                   gincY, st)) != SK_OK)
        return rc;
    if ((rc = convert_grad(X, d, p.dpad, inc_mode, gincX, gX, st)) != SK_OK) return rc;
    if (!p.same_xy && (rc = convert_grad(Y, d, p.dpad, inc_mode, gincY, gY, st)) != SK_OK) return rc;
    SK_CUDA(owned.release());
    return SK_OK;
}

// ------------------------------------------------------------------------------------------
// MMD^2 from the three Gram blocks; weights of its backward.
// ------------------------------------------------------------------------------------------
__global__ void mmd2_reduce_kernel(const double* Kaa, int64_t na, const double* Kbb, int64_t nb, const double* Kab,
                                   int unbiased, double* out) {
    __shared__ double part[3][256];
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < na * na; i += blockDim.x)
        if (!unbiased || (i / na) != (i % na)) s[0] += Kaa[i];
    for (int64_t i = threadIdx.x; i < nb * nb; i += blockDim.x)
        if (!unbiased || (i / nb) != (i % nb)) s[1] += Kbb[i];
    for (int64_t i = threadIdx.x; i < na * nb; i += blockDim.x) s[2] += Kab[i];
    for (int q = 0; q < 3; ++q) part[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {  // fixed-order tree: deterministic
        if (static_cast<int>(threadIdx.x) < w)
            for (int q = 0; q < 3; ++q) part[q][threadIdx.x] += part[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double daa = unbiased ? static_cast<double>(na) * (na - 1) : static_cast<double>(na) * na;
        const double dbb = unbiased ? static_cast<double>(nb) * (nb - 1) : static_cast<double>(nb) * nb;
        const double maa = part[0][0] / daa, mbb = part[1][0] / dbb, mab = part[2][0] / (static_cast<double>(na) * nb);
        out[0] = maa + mbb - 2.0 * mab;
        out[1] = maa;
        out[2] = mbb;
        out[3] = mab;
    }
}

__global__ void fill_weights_kernel(double* W, int64_t n, int64_t m, double v, int zero_diag) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n * m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        W[i] = (zero_diag && (i / m) == (i % m)) ? 0.0 : v;
}

// MMD^2 planning, shared by sigkernel_mmd2 and sigkernel_workspace_size.  The three Gram blocks
// (K_AA and K_BB symmetric, K_AB full) run one after another in one workspace.  With gradients
// (polynomial schemes) each block runs in chunks of items: the forward records a tape of
// the chunk and the tape adjoint runs from it at once, with the block's constant upstream weights
// (MMD^2 is linear in the Gram entries).  A chunk's tape is at most kTapeChunkBudget bytes, and a
// chunk smaller than a block is a whole number of the adjoint's resident warps.  When the budget
// holds fewer items than half the adjoint's resident warps (very long paths), the block uses the
// checkpointing adjoint instead, which keeps only the strip hand-offs and one strip's tape per
// warp (approximation scheme only).  The same budget bounds the chunks of sigkernel_backward for
// the interpolation scheme.
// 64 GiB holds the tape of a 128 x 128 Gram of 257-point paths (61 GB at N = 6 in FP32) in one
// chunk: at 48 GiB it took two (10944 + 5440 pairs), and the second chunk's partial waves cost
// 2.3 ms of the 29.0 ms backward call.
constexpr size_t kTapeChunkBudget = size_t(64) << 30;

struct MmdPlan {
    bool grads;
    sk_options os, of;     // options of the symmetric blocks and of the cross block
    int64_t items[3];      // K_AA (upper), K_BB (upper), K_AB (full)
    int64_t chunk[3];      // items per chunk (gradients)
    bool tape[3];          // gradients from chunked tapes, else the checkpointing adjoint
    Plan f[3];
    TapeBwdPlan tb[3];
    BwdPlan cb[3];
    size_t gram_bytes, w_bytes, ginc_a, ginc_bytes, tape_bytes, sub, total;
};

int plan_mmd2(const sk_paths* A, const sk_paths* Bp, int32_t d, int32_t dtype, const sk_options* o, bool grads,
              MmdPlan& m) {
    if (!A || !Bp || !o) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (A->count < 1 || Bp->count < 1) return fail(SK_ERR_INVALID_ARG, "MMD^2 needs non-empty path sets");
    const bool unb = (o->flags & SK_FLAG_UNBIASED) != 0;
    if (unb && (A->count < 2 || Bp->count < 2)) return fail(SK_ERR_INVALID_ARG, "unbiased MMD^2 needs >= 2 paths per set");
    if (grads && is_fd(o) && o->dyadic > 4)
        return fail(SK_ERR_UNSUPPORTED, "MMD^2 gradients of the FD schemes support dyadic orders 0..4");
    m.grads = grads;
    m.os = *o;
    m.os.flags = (o->flags & (SK_FLAG_INCREMENTS | SK_FLAG_NO_SORT | SK_FLAG_TIME_KERNEL | SK_FLAG_STRIP_PIPELINE |
                              SK_FLAG_NO_STRIP_PIPELINE | SK_FLAG_NO_TILED_M | SK_FLAG_NO_TC)) | SK_FLAG_SYMMETRIC;
    m.of = m.os;
    m.of.flags &= ~SK_FLAG_SYMMETRIC;
    const sk_paths* xs[3] = {A, Bp, A};
    const sk_paths* ys[3] = {A, Bp, Bp};
    const int modes[3] = {kGramUpper, kGramUpper, kGramFull};
    m.items[0] = gram_items(A, A, true);
    m.items[1] = gram_items(Bp, Bp, true);
    m.items[2] = gram_items(A, Bp, false);
    int rc;
    m.sub = 0;
    m.tape_bytes = 0;
    for (int k = 0; k < 3; ++k) {
        const sk_options* ok = k < 2 ? &m.os : &m.of;
        if (!grads) {
            m.chunk[k] = m.items[k];
            if ((rc = plan_forward(xs[k], ys[k], d, dtype, ok, modes[k], m.items[k], m.f[k], true)) != SK_OK) return rc;
            m.sub = std::max(m.sub, m.f[k].total);
            continue;
        }
        Plan p1;
        if ((rc = plan_forward(xs[k], ys[k], d, dtype, ok, modes[k], 1, p1)) != SK_OK) return rc;
        TapePlan t1;
        if ((rc = plan_tape(xs[k], ys[k], ok, p1.T, 1, t1)) != SK_OK) return rc;
        TapeBwdPlan whole;
        if ((rc = plan_backward_tape(xs[k], ys[k], d, dtype, ok, modes[k], m.items[k], whole)) != SK_OK) return rc;
        const int64_t resident = std::max<int64_t>(1, static_cast<int64_t>(whole.f.blocks) * kFwdWarps);
        int64_t c = std::max<int64_t>(1, static_cast<int64_t>(kTapeChunkBudget / std::max<size_t>(t1.stride, 1)));
        if (c < m.items[k] && c > resident) c -= c % resident;
        m.chunk[k] = std::min(c, m.items[k]);
        m.tape[k] = m.chunk[k] == m.items[k] || 2 * m.chunk[k] >= resident;
        if (!m.tape[k]) {  // checkpointing adjoint over the whole block
            if (o->scheme != SK_POLY_APPROX)
                return fail(SK_ERR_UNSUPPORTED,
                            "MMD^2 gradients of this scheme need forward tapes, and these paths are too long for a "
                            "tape chunk to fill the GPU");
            m.chunk[k] = m.items[k];
            if ((rc = plan_forward(xs[k], ys[k], d, dtype, ok, modes[k], m.items[k], m.f[k], true)) != SK_OK) return rc;
            if ((rc = plan_backward(xs[k], ys[k], d, dtype, ok, modes[k], m.items[k], m.cb[k])) != SK_OK) return rc;
            m.sub = std::max(m.sub, std::max(m.f[k].total, m.cb[k].total));
            continue;
        }
        if ((rc = plan_forward(xs[k], ys[k], d, dtype, ok, modes[k], m.chunk[k], m.f[k], false, true)) != SK_OK)
            return rc;
        if ((rc = plan_backward_tape(xs[k], ys[k], d, dtype, ok, modes[k], m.chunk[k], m.tb[k])) != SK_OK) return rc;
        TapePlan tc;
        if ((rc = plan_tape(xs[k], ys[k], ok, p1.T, m.chunk[k], tc)) != SK_OK) return rc;
        m.tape_bytes = std::max(m.tape_bytes, tc.total);
        m.sub = std::max(m.sub, std::max(m.f[k].total, m.tb[k].total));
    }
    const int64_t na = A->count, nb = Bp->count;
    const int dpad = m.f[0].dpad;
    m.gram_bytes = align256((na * na + nb * nb + na * nb) * sizeof(double));
    m.w_bytes = grads ? m.gram_bytes : 0;
    m.ginc_a = grads ? align256(static_cast<size_t>(A->rows_total) * dpad * 8) : 0;
    m.ginc_bytes = grads ? m.ginc_a + align256(static_cast<size_t>(Bp->rows_total) * dpad * 8) : 0;
    m.total = m.gram_bytes + m.w_bytes + m.ginc_bytes + align256(m.tape_bytes) + m.sub + 512;
    return SK_OK;
}

int run_mmd2(const sk_paths* A, const sk_paths* Bp, int32_t d, int32_t dtype, const sk_options* o, double* out,
             double* gA, double* gB, void* ws, size_t ws_bytes, void* stream) {
    if (!out) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    const bool grads = gA || gB;
    MmdPlan m;
    int rc = plan_mmd2(A, Bp, d, dtype, o, grads, m);
    if (rc != SK_OK) return rc;
    const bool unb = (o->flags & SK_FLAG_UNBIASED) != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, m.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < m.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, m.total);
    }
    const int64_t na = A->count, nb = Bp->count;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) / 256 * 256);
    double* Kaa = reinterpret_cast<double*>(base);
    double* Kbb = Kaa + na * na;
    double* Kab = Kbb + nb * nb;
    double* Waa = reinterpret_cast<double*>(base + m.gram_bytes);
    double* Wbb = Waa + na * na;
    double* Wab = Wbb + nb * nb;
    double* gincA = reinterpret_cast<double*>(base + m.gram_bytes + m.w_bytes);
    double* gincB = reinterpret_cast<double*>(base + m.gram_bytes + m.w_bytes + m.ginc_a);
    char* tape = base + m.gram_bytes + m.w_bytes + m.ginc_bytes;
    char* sub_ws = tape + align256(m.tape_bytes);
    const sk_paths* xs[3] = {A, Bp, A};
    const sk_paths* ys[3] = {A, Bp, Bp};
    const int modes[3] = {kGramUpper, kGramUpper, kGramFull};
    double* Ks[3] = {Kaa, Kbb, Kab};
    const int64_t ldos[3] = {na, nb, nb};
    if (!grads) {
        for (int k = 0; k < 3; ++k)
            if ((rc = run_forward(xs[k], ys[k], d, dtype, k < 2 ? &m.os : &m.of, modes[k], nullptr, nullptr, m.items[k],
                                  Ks[k], ldos[k], sub_ws, m.sub, st)) != SK_OK)
                return rc;
    } else {
        const double waa = unb ? 1.0 / (static_cast<double>(na) * (na - 1)) : 1.0 / (static_cast<double>(na) * na);
        const double wbb = unb ? 1.0 / (static_cast<double>(nb) * (nb - 1)) : 1.0 / (static_cast<double>(nb) * nb);
        const double wab = -2.0 / (static_cast<double>(na) * nb);
        fill_weights_kernel<<<64, 256, 0, st>>>(Waa, na, na, waa, unb ? 1 : 0);
        fill_weights_kernel<<<64, 256, 0, st>>>(Wbb, nb, nb, wbb, unb ? 1 : 0);
        fill_weights_kernel<<<64, 256, 0, st>>>(Wab, na, nb, wab, 0);
        SK_CUDA(cudaGetLastError());
        SK_CUDA(cudaMemsetAsync(gincA, 0, m.ginc_bytes, st));
        const double* Ws[3] = {Waa, Wbb, Wab};
        double* gx[3] = {gincA, gincB, gincA};
        double* gy[3] = {gincA, gincB, gincB};
        char* sb = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(sub_ws) + 255) / 256 * 256);
        for (int k = 0; k < 3; ++k) {
            const sk_options* ok = k < 2 ? &m.os : &m.of;
            if (!m.tape[k]) {
                if ((rc = run_forward(xs[k], ys[k], d, dtype, ok, modes[k], nullptr, nullptr, m.items[k], Ks[k], ldos[k],
                                      sub_ws, m.sub, st)) != SK_OK)
                    return rc;
                if ((rc = launch_backward(xs[k], ys[k], d, dtype, ok, modes[k], nullptr, nullptr, m.items[k], Ws[k],
                                          ldos[k], m.cb[k], sb, gx[k], gy[k], st)) != SK_OK)
                    return rc;
                continue;
            }
            for (int64_t i0 = 0; i0 < m.items[k]; i0 += m.chunk[k]) {
                const int64_t n = std::min(m.chunk[k], m.items[k] - i0);
                if ((rc = run_forward(xs[k], ys[k], d, dtype, ok, modes[k], nullptr, nullptr, n, Ks[k], ldos[k], sub_ws,
                                      m.sub, st, tape, m.tape_bytes, i0)) != SK_OK)
                    return rc;
                if ((rc = launch_backward_tape(xs[k], ys[k], d, dtype, ok, modes[k], nullptr, nullptr, n, i0, tape, Ws[k],
                                               ldos[k], m.tb[k], sb, gx[k], gy[k], st)) != SK_OK)
                    return rc;
            }
        }
        const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
        const int dpad = m.f[0].dpad;
        if (gA) {
            SK_CUDA(cudaMemsetAsync(gA, 0, static_cast<size_t>(A->rows_total) * d * sizeof(double), st));
            if ((rc = convert_grad(A, d, dpad, inc_mode, gincA, gA, st)) != SK_OK) return rc;
        }
        if (gB) {
            SK_CUDA(cudaMemsetAsync(gB, 0, static_cast<size_t>(Bp->rows_total) * d * sizeof(double), st));
            if ((rc = convert_grad(Bp, d, dpad, inc_mode, gincB, gB, st)) != SK_OK) return rc;
        }
    }
    mmd2_reduce_kernel<<<1, 256, 0, st>>>(Kaa, na, Kbb, nb, Kab, unb ? 1 : 0, out);
    SK_CUDA(cudaGetLastError());
    SK_CUDA(owned.release());
    return SK_OK;
}

// sigkernel_backward of the polynomial schemes: the items are taken in chunks whose forward
// records a tape (at most kTapeChunkBudget bytes) and whose tape adjoint follows at once, as in
// sigkernel_mmd2.  When the paths are so long that a chunk holds fewer items than half the
// adjoint's resident warps, the plan says so (fits = false): the approximation scheme then runs the
// checkpointing adjoint, and the interpolation scheme, which has none, is refused
// (SK_ERR_UNSUPPORTED).
struct ChunkBwdPlan {
    bool fits;        // a chunk fills the GPU (else the chunked plan below is not made)
    int64_t items, chunk;
    Plan f;           // forward of one chunk, recording its tape
    TapeBwdPlan tb;   // tape adjoint of one chunk
    size_t ginc_a, ginc_bytes, tape_bytes, out_bytes, sub, total;
};

int plan_backward_chunked(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                          int mode, int64_t items, ChunkBwdPlan& c) {
    Plan p1;
    int rc;
    if ((rc = plan_forward(X, Y, d, dtype, o, mode, 1, p1)) != SK_OK) return rc;
    TapePlan t1;
    if ((rc = plan_tape(X, Y, o, p1.T, 1, t1)) != SK_OK) return rc;
    TapeBwdPlan whole;
    if ((rc = plan_backward_tape(X, Y, d, dtype, o, mode, std::max<int64_t>(items, 1), whole)) != SK_OK) return rc;
    const int64_t resident = std::max<int64_t>(1, static_cast<int64_t>(whole.f.blocks) * kFwdWarps);
    int64_t chunk = std::max<int64_t>(1, static_cast<int64_t>(kTapeChunkBudget / std::max<size_t>(t1.stride, 1)));
    if (chunk < items && chunk > resident) chunk -= chunk % resident;
    chunk = std::max<int64_t>(1, std::min(chunk, items));
    c.fits = !(chunk < items && 2 * chunk < resident);
    if (!c.fits) {
        if (o->scheme != SK_POLY_APPROX)
            return fail(SK_ERR_UNSUPPORTED, "sigkernel_backward of this scheme needs forward tapes, and these paths "
                                            "are too long for a tape chunk to fill the GPU");
        return SK_OK;
    }
    c.items = items;
    c.chunk = chunk;
    if ((rc = plan_forward(X, Y, d, dtype, o, mode, chunk, c.f, false, true)) != SK_OK) return rc;
    if ((rc = plan_backward_tape(X, Y, d, dtype, o, mode, chunk, c.tb)) != SK_OK) return rc;
    TapePlan tc;
    if ((rc = plan_tape(X, Y, o, p1.T, chunk, tc)) != SK_OK) return rc;
    c.tape_bytes = tc.total;
    const int64_t nout = mode == kPairsList ? chunk : X->count * Y->count;
    c.out_bytes = align256(static_cast<size_t>(std::max<int64_t>(nout, 1)) * sizeof(double));
    c.ginc_a = align256(static_cast<size_t>(X->rows_total) * p1.dpad * sizeof(double));
    c.ginc_bytes = c.ginc_a + (p1.same_xy ? 0 : align256(static_cast<size_t>(Y->rows_total) * p1.dpad * sizeof(double)));
    c.sub = std::max(c.f.total, c.tb.total);
    c.total = c.ginc_bytes + align256(c.tape_bytes) + c.out_bytes + c.sub + 512;
    return SK_OK;
}

// sigkernel_backward runs from chunked tapes for both polynomial schemes unless the caller asks for
// the checkpointing adjoint (approximation scheme only).
bool uses_tape_chunks(const sk_options* o) {
    if (o->scheme == SK_POLY_INTERP || is_fd(o)) return true;
    return o->scheme == SK_POLY_APPROX && !(o->flags & SK_FLAG_CHECKPOINT);
}

int run_backward_chunked(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* o,
                         const int64_t* pa, const int64_t* pb, int64_t npairs, const double* gout, double* gX,
                         double* gY, void* ws, size_t ws_bytes, void* stream) {
    const bool gram = (pa == nullptr);
    const bool sym = gram && (o->flags & SK_FLAG_SYMMETRIC);
    const int mode = gram ? (sym ? kGramUpper : kGramFull) : kPairsList;
    if (gram) npairs = gram_items(X, Y, sym);
    ChunkBwdPlan c;
    int rc = plan_backward_chunked(X, Y, d, dtype, o, mode, npairs, c);
    if (rc != SK_OK) return rc;
    if (!c.fits)  // approximation scheme, paths too long for tape chunks: checkpointing adjoint
        return run_backward(X, Y, d, dtype, o, pa, pb, npairs, gout, gX, gY, ws, ws_bytes, stream);
    if (c.f.same_xy && gY && gY != gX)
        return fail(SK_ERR_INVALID_ARG, "X and Y are the same paths: pass grad_Y = NULL or grad_Y = grad_X");
    if (npairs == 0) return SK_OK;
    if (!gout) return fail(SK_ERR_INVALID_ARG, "grad_out is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, c.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < c.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, c.total);
    }
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) / 256 * 256);
    double* gincX = reinterpret_cast<double*>(base);
    double* gincY = c.f.same_xy ? gincX : reinterpret_cast<double*>(base + c.ginc_a);
    char* tape = base + c.ginc_bytes;
    double* outbuf = reinterpret_cast<double*>(tape + align256(c.tape_bytes));
    char* sub_ws = reinterpret_cast<char*>(outbuf) + c.out_bytes;
    char* sb = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(sub_ws) + 255) / 256 * 256);
    SK_CUDA(cudaMemsetAsync(gincX, 0, c.ginc_bytes, st));
    const int64_t ldo = gram ? Y->count : 0;
    for (int64_t i0 = 0; i0 < npairs; i0 += c.chunk) {
        const int64_t n = std::min(c.chunk, npairs - i0);
        const int64_t* pai = gram ? nullptr : pa + i0;
        const int64_t* pbi = gram ? nullptr : pb + i0;
        const double* gi = gram ? gout : gout + i0;
        const int64_t base_item = gram ? i0 : 0;
        if ((rc = run_forward(X, Y, d, dtype, o, mode, pai, pbi, n, outbuf, ldo, sub_ws, c.sub, st, tape, c.tape_bytes,
                              base_item)) != SK_OK)
            return rc;
        if ((rc = launch_backward_tape(X, Y, d, dtype, o, mode, pai, pbi, n, base_item, tape, gi, ldo, c.tb, sb, gincX,
                                       gincY, st)) != SK_OK)
            return rc;
    }
    const int inc_mode = (o->flags & SK_FLAG_INCREMENTS) ? 1 : 0;
    if ((rc = convert_grad(X, d, c.f.dpad, inc_mode, gincX, gX, st)) != SK_OK) return rc;
    if (!c.f.same_xy && (rc = convert_grad(Y, d, c.f.dpad, inc_mode, gincY, gY, st)) != SK_OK) return rc;
    SK_CUDA(owned.release());
    return SK_OK;
}

// Permutation test on MMD^2: the pooled Gram K of Z = (A, B) from the three blocks of
// sigkernel_mmd2 written in place (K_AA and K_BB symmetric, K_AB full; K_BA mirrored by the test's
// own kernel), then the statistics of every relabelling (launch_mmd_perm).
constexpr int64_t kMaxPooled = 65536;
constexpr int64_t kMaxPerm = int64_t(1) << 24;

struct MmdTestPlan {
    MmdPlan m;
    size_t k_bytes, scratch, total;
};

int plan_mmd2_test(const sk_paths* A, const sk_paths* Bp, int32_t d, int32_t dtype, const sk_options* o, int64_t nperm,
                   MmdTestPlan& t) {
    if (nperm < 0 || nperm > kMaxPerm) return fail(SK_ERR_INVALID_ARG, "nperm %lld outside [0, 2^24]", (long long)nperm);
    int rc = plan_mmd2(A, Bp, d, dtype, o, false, t.m);
    if (rc != SK_OK) return rc;
    const int64_t n = A->count + Bp->count;
    if (n > kMaxPooled) return fail(SK_ERR_UNSUPPORTED, "%lld pooled paths (this build: <= %lld)", (long long)n,
                                    (long long)kMaxPooled);
    t.k_bytes = align256(static_cast<size_t>(n) * n * sizeof(double));
    t.scratch = mmd_perm_scratch_bytes(n, nperm);
    t.total = t.k_bytes + t.scratch + t.m.sub + 512;
    return SK_OK;
}

int run_mmd2_test(const sk_paths* A, const sk_paths* Bp, int32_t d, int32_t dtype, const sk_options* o,
                  const uint8_t* labels, int64_t nperm, double* out, void* ws, size_t ws_bytes, void* stream) {
    if (!out) return fail(SK_ERR_INVALID_ARG, "out is NULL");
    if (nperm > 0 && !labels) return fail(SK_ERR_INVALID_ARG, "labels is NULL");
    MmdTestPlan t;
    int rc = plan_mmd2_test(A, Bp, d, dtype, o, nperm, t);
    if (rc != SK_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OwnedWorkspace owned;
    if (!ws) {
        SK_CUDA(cudaMallocAsync(&ws, t.total, st));
        owned.p = ws;
        owned.st = st;
    } else if (ws_bytes < t.total) {
        return fail(SK_ERR_WORKSPACE, "workspace %zu bytes < %zu required", ws_bytes, t.total);
    }
    const int64_t na = A->count, n = A->count + Bp->count;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) / 256 * 256);
    double* K = reinterpret_cast<double*>(base);
    char* scratch = base + t.k_bytes;
    char* sub_ws = scratch + t.scratch;
    const sk_paths* xs[3] = {A, Bp, A};
    const sk_paths* ys[3] = {A, Bp, Bp};
    const int modes[3] = {kGramUpper, kGramUpper, kGramFull};
    double* Ks[3] = {K, K + na * n + na, K + na};
    for (int k = 0; k < 3; ++k)
        if ((rc = run_forward(xs[k], ys[k], d, dtype, k < 2 ? &t.m.os : &t.m.of, modes[k], nullptr, nullptr, t.m.items[k],
                              Ks[k], n, sub_ws, t.m.sub, st)) != SK_OK)
            return rc;
    SK_CUDA(launch_mmd_perm(K, n, na, labels, nperm, (o->flags & SK_FLAG_UNBIASED) ? 1 : 0, scratch, out, st));
    SK_CUDA(owned.release());
    return SK_OK;
}

}  // namespace

void set_last_error(const char* msg) { t_last_error = msg; }

}  // namespace sk

using namespace sk;

// An NVTX range over an entry point, for timelines of profilers that attach to the process (a
// no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

extern "C" {

int sigkernel_autotune(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const int64_t* pair_a,
                       const int64_t* pair_b, int64_t npairs, const sk_options* opt, double* out, int32_t trials,
                       sk_options* best, float* best_ms, void* stream) {
    NvtxRange nvtx_range("sigkernel_autotune");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{pair_a, "pair_a"}, {pair_b, "pair_b"}, {out, "out"}});
    if (prc != SK_OK) return prc;
    if (!opt || !X || !Y || !out || !best) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (trials < 1 || trials > 1000) return fail(SK_ERR_INVALID_ARG, "trials %d outside [1, 1000]", trials);
    if (pair_a && (!pair_b || npairs < 0)) return fail(SK_ERR_INVALID_ARG, "bad pair list");
    const bool gram = pair_a == nullptr;
    const bool sym = gram && (opt->flags & SK_FLAG_SYMMETRIC);
    const int mode = gram ? (sym ? kGramUpper : kGramFull) : kPairsList;
    const int64_t n = gram ? gram_items(X, Y, sym) : npairs;
    const int64_t ldo = gram ? Y->count : 0;
    const int strip = SK_FLAG_STRIP_PIPELINE | SK_FLAG_NO_STRIP_PIPELINE | SK_FLAG_TIME_KERNEL;
    struct Cand {
        int wpb, pipe, mt;
    };
    // one warp per pair with 1, 2, 4 warps per block, with and without tiled M; the pipeline
    Cand all[7] = {{1, -1, 1}, {2, -1, 1}, {4, -1, 1}, {1, -1, -1}, {2, -1, -1}, {4, -1, -1}, {0, 1, -1}};
    Cand cands[7];
    int ncand = 0;
    size_t ws_bytes = 0;
    int rc;
    auto cand_options = [&](const Cand& c) {
        sk_options co = *opt;
        co.flags = (opt->flags & ~(strip | SK_FLAG_NO_TILED_M)) |
                   (c.pipe > 0 ? SK_FLAG_STRIP_PIPELINE : SK_FLAG_NO_STRIP_PIPELINE) | (c.mt < 0 ? SK_FLAG_NO_TILED_M : 0);
        co.warps_per_block = c.wpb;
        return co;
    };
    for (int c = 0; c < 7; ++c) {
        sk_options co = cand_options(all[c]);
        Plan p;
        if ((rc = plan_forward(X, Y, d, dtype, &co, mode, n, p, true)) != SK_OK) return rc;
        if (all[c].pipe > 0 && !p.coop) continue;            // no pair spans two strips
        if (all[c].pipe < 0 && all[c].mt > 0 && !p.mtile) continue;  // tiled M not applicable
        cands[ncand++] = all[c];
        ws_bytes = std::max(ws_bytes, p.total);
    }
    if (n == 0) return fail(SK_ERR_INVALID_ARG, "nothing to tune: no pairs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SK_CUDA(cudaMallocAsync(&ws, ws_bytes, st));
    float best_t = -1.f;
    int best_c = 0;
    rc = SK_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(SK_ERR_CUDA, "cudaEventCreate failed");
    }
    for (int c = 0; c < ncand && rc == SK_OK; ++c) {
        const sk_options co = cand_options(cands[c]);
        float t_min = -1.f;
        for (int t = 0; t <= trials && rc == SK_OK; ++t) {  // t = 0 warms up
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = fail(SK_ERR_CUDA, "cudaEventRecord failed"); break; }
            rc = run_forward(X, Y, d, dtype, &co, mode, pair_a, pair_b, n, out, ldo, ws, ws_bytes, stream);
            if (rc != SK_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(SK_ERR_CUDA, "timing a candidate failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (t > 0 && (t_min < 0.f || ms < t_min)) t_min = ms;
        }
        if (rc == SK_OK && (best_t < 0.f || t_min < best_t)) {
            best_t = t_min;
            best_c = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(ws, st);
    if (rc != SK_OK) return rc;
    int dev = 0;
    SK_CUDA(cudaGetDevice(&dev));
    const int vw = opt->compute == SK_COMPUTE_F32 ? 4 : 2;
    const int dpad = (d + vw - 1) / vw * vw;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[tune_key(dev, X, Y, opt, dpad, mode, n)] =
            TuneChoice{cands[best_c].wpb ? cands[best_c].wpb : kFwdWarps, cands[best_c].pipe, cands[best_c].mt};
    }
    *best = cand_options(cands[best_c]);
    if (best_ms) *best_ms = best_t;
    return SK_OK;
}

void sigkernel_autotune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

int sigkernel_version(void) { return 200; }

void sigkernel_set_wait_limit(uint32_t polls) { g_wait_limit.store(polls, std::memory_order_relaxed); }

const char* sigkernel_last_error(void) { return t_last_error.c_str(); }

float sigkernel_last_kernel_ms(void) {
    if (!t_timed) return -1.0f;
    float ms = -1.0f;
    if (cudaEventSynchronize(t_ev1) != cudaSuccess) return -1.0f;
    if (cudaEventElapsedTime(&ms, t_ev0, t_ev1) != cudaSuccess) return -1.0f;
    return ms;
}

int sigkernel_workspace_size(int32_t op, const sk_paths* X, const sk_paths* Y, int32_t d, int64_t npairs,
                             const sk_options* opt, size_t* bytes) {
    t_last_error.clear();
    if (!bytes) return fail(SK_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = 0;
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    Plan p;
    int rc;
    const int dtype = SK_F64;  // sizes do not depend on the input element type
    switch (op) {
        case SK_OP_PAIRS:
            rc = plan_forward(X, Y, d, dtype, opt, kPairsList, npairs, p, true);
            break;
        case SK_OP_GRAM: {
            bool sym = (opt->flags & SK_FLAG_SYMMETRIC) != 0;
            rc = plan_forward(X, Y, d, dtype, opt, sym ? kGramUpper : kGramFull, gram_items(X, Y, sym), p, true);
            break;
        }
        case SK_OP_BACKWARD: {
            const bool gram = npairs < 0;
            const bool sym = gram && (opt->flags & SK_FLAG_SYMMETRIC);
            if (uses_tape_chunks(opt)) {
                ChunkBwdPlan c;
                rc = plan_backward_chunked(X, Y, d, dtype, opt, gram ? (sym ? kGramUpper : kGramFull) : kPairsList,
                                           gram ? gram_items(X, Y, sym) : npairs, c);
                if (rc != SK_OK || c.fits) {
                    if (rc == SK_OK) *bytes = c.total;
                    return rc;
                }
            }
            BwdPlan b;
            rc = plan_backward(X, Y, d, dtype, opt, gram ? (sym ? kGramUpper : kGramFull) : kPairsList,
                               gram ? gram_items(X, Y, sym) : npairs, b);
            if (rc == SK_OK) *bytes = b.total;
            return rc;
        }
        case SK_OP_BACKWARD_TAPE: {
            const bool gram = npairs < 0;
            const bool sym = gram && (opt->flags & SK_FLAG_SYMMETRIC);
            TapeBwdPlan b;
            rc = plan_backward_tape(X, Y, d, dtype, opt, gram ? (sym ? kGramUpper : kGramFull) : kPairsList,
                                    gram ? gram_items(X, Y, sym) : npairs, b);
            if (rc == SK_OK) *bytes = b.total;
            return rc;
        }
        case SK_OP_MMD2: {
            // sized by the same planning as sigkernel_mmd2 (X = A, Y = B); npairs = 1 asks for
            // the gradient's workspace, 0 for the value alone
            MmdPlan m;
            rc = plan_mmd2(X, Y, d, dtype, opt, npairs != 0, m);
            if (rc == SK_OK) *bytes = m.total;
            return rc;
        }
        case SK_OP_MMD2_TEST: {
            MmdTestPlan t;
            rc = plan_mmd2_test(X, Y, d, dtype, opt, npairs, t);
            if (rc == SK_OK) *bytes = t.total;
            return rc;
        }
        default:
            return fail(SK_ERR_UNSUPPORTED, "workspace for op %d", op);
    }
    if (rc == SK_OK) *bytes = p.total;
    return rc;
}

int sigkernel_pairs(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const int64_t* pair_a,
                    const int64_t* pair_b, int64_t npairs, const sk_options* opt, double* out, void* workspace,
                    size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_pairs");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{pair_a, "pair_a"}, {pair_b, "pair_b"}, {out, "out"}});
    if (prc != SK_OK) return prc;
    if (npairs < 0) return fail(SK_ERR_INVALID_ARG, "npairs < 0");
    if (npairs > 0 && (!pair_a || !pair_b)) return fail(SK_ERR_INVALID_ARG, "pair index arrays are NULL");
    return run_forward(X, Y, d, dtype, opt, kPairsList, pair_a, pair_b, npairs, out, 0, workspace, workspace_bytes,
                       stream);
}

int sigkernel_gram(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const sk_options* opt, double* G,
                   void* workspace, size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_gram");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{G, "G"}});
    if (prc != SK_OK) return prc;
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    bool sym = (opt->flags & SK_FLAG_SYMMETRIC) != 0;
    return run_forward(X, Y, d, dtype, opt, sym ? kGramUpper : kGramFull, nullptr, nullptr, gram_items(X, Y, sym), G,
                       Y->count, workspace, workspace_bytes, stream);
}

int sigkernel_backward(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const int64_t* pair_a,
                       const int64_t* pair_b, int64_t npairs, const sk_options* opt, const double* grad_out,
                       double* grad_X, double* grad_Y, void* workspace, size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_backward");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{pair_a, "pair_a"}, {pair_b, "pair_b"}, {grad_out, "grad_out"},
                                                      {grad_X, "grad_X"}, {grad_Y, "grad_Y"}});
    if (prc != SK_OK) return prc;
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (pair_a && (!pair_b || npairs < 0)) return fail(SK_ERR_INVALID_ARG, "bad pair list");
    if (uses_tape_chunks(opt))
        return run_backward_chunked(X, Y, d, dtype, opt, pair_a, pair_b, npairs, grad_out, grad_X, grad_Y, workspace,
                                    workspace_bytes, stream);
    return run_backward(X, Y, d, dtype, opt, pair_a, pair_b, npairs, grad_out, grad_X, grad_Y, workspace,
                        workspace_bytes, stream);
}

int sigkernel_tape_size(const sk_paths* X, const sk_paths* Y, int32_t d, int64_t npairs, const sk_options* opt,
                        size_t* bytes) {
    t_last_error.clear();
    if (!bytes) return fail(SK_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = 0;
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    const bool gram = npairs < 0;
    const bool sym = gram && (opt->flags & SK_FLAG_SYMMETRIC);
    Plan p;
    int rc = plan_forward(X, Y, d, SK_F64, opt, gram ? (sym ? kGramUpper : kGramFull) : kPairsList,
                          gram ? gram_items(X, Y, sym) : npairs, p);
    if (rc != SK_OK) return rc;
    TapePlan t;
    if ((rc = plan_tape(X, Y, opt, p.T, p.npairs, t)) != SK_OK) return rc;
    *bytes = t.total;
    return SK_OK;
}

int sigkernel_forward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const int64_t* pair_a,
                           const int64_t* pair_b, int64_t npairs, const sk_options* opt, double* out, void* tape,
                           size_t tape_bytes, void* workspace, size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_forward_tape");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{pair_a, "pair_a"}, {pair_b, "pair_b"}, {out, "out"}});
    if (prc != SK_OK) return prc;
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (!tape) return fail(SK_ERR_INVALID_ARG, "tape is NULL");
    if (reinterpret_cast<uintptr_t>(tape) % 256) return fail(SK_ERR_INVALID_ARG, "tape must be 256-byte aligned");
    if (pair_a == nullptr) {
        const bool sym = (opt->flags & SK_FLAG_SYMMETRIC) != 0;
        return run_forward(X, Y, d, dtype, opt, sym ? kGramUpper : kGramFull, nullptr, nullptr, gram_items(X, Y, sym),
                           out, Y->count, workspace, workspace_bytes, stream, tape, tape_bytes);
    }
    if (!pair_b || npairs < 0) return fail(SK_ERR_INVALID_ARG, "bad pair list");
    return run_forward(X, Y, d, dtype, opt, kPairsList, pair_a, pair_b, npairs, out, 0, workspace, workspace_bytes,
                       stream, tape, tape_bytes);
}

int sigkernel_backward_tape(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype, const int64_t* pair_a,
                            const int64_t* pair_b, int64_t npairs, const sk_options* opt, const void* tape,
                            size_t tape_bytes, const double* grad_out, double* grad_X, double* grad_Y, void* workspace,
                            size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_backward_tape");
    t_last_error.clear();
    int prc = check_call_ptrs(X, "X", Y, "Y", dtype, {{pair_a, "pair_a"}, {pair_b, "pair_b"}, {grad_out, "grad_out"},
                                                      {grad_X, "grad_X"}, {grad_Y, "grad_Y"}});
    if (prc != SK_OK) return prc;
    // the adjoint streams tape steps with bulk copies, which need 16-byte aligned sources; the
    // forward lays the tape out from a 256-byte aligned base
    if (reinterpret_cast<uintptr_t>(tape) % 256) return fail(SK_ERR_INVALID_ARG, "tape must be 256-byte aligned");
    if (!opt || !X || !Y) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (pair_a && (!pair_b || npairs < 0)) return fail(SK_ERR_INVALID_ARG, "bad pair list");
    return run_backward_tape(X, Y, d, dtype, opt, pair_a, pair_b, npairs, tape, tape_bytes, grad_out, grad_X, grad_Y,
                             workspace, workspace_bytes, stream);
}

int sigkernel_mmd2(const sk_paths* A, const sk_paths* B, int32_t d, int32_t dtype, const sk_options* opt, double* out,
                   double* grad_A, double* grad_B, void* workspace, size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("sigkernel_mmd2");
    t_last_error.clear();
    int prc = check_call_ptrs(A, "A", B, "B", dtype, {{out, "out"}, {grad_A, "grad_A"}, {grad_B, "grad_B"}});
    if (prc != SK_OK) return prc;
    return run_mmd2(A, B, d, dtype, opt, out, grad_A, grad_B, workspace, workspace_bytes, stream);
}

int sigkernel_mmd2_test(const sk_paths* A, const sk_paths* B, int32_t d, int32_t dtype, const sk_options* opt,
                        const uint8_t* labels, int64_t nperm, double* out, void* workspace, size_t workspace_bytes,
                        void* stream) {
    NvtxRange nvtx_range("sigkernel_mmd2_test");
    t_last_error.clear();
    int prc = check_call_ptrs(A, "A", B, "B", dtype, {{out, "out"}});
    if (prc != SK_OK) return prc;
    return run_mmd2_test(A, B, d, dtype, opt, labels, nperm, out, workspace, workspace_bytes, stream);
}

int sigkernel_device_status(void* stream) {
    t_last_error.clear();
    SK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int code = 0, zero = 0;
    SK_CUDA(cudaMemcpyFromSymbol(&code, g_sk_error, sizeof(int)));
    SK_CUDA(cudaMemcpyToSymbol(g_sk_error, &zero, sizeof(int)));
    if (code != 0) return fail(code, "device error word %d", code);
    return SK_OK;
}

}  // extern "C"
