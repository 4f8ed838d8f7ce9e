// Shared device-side definitions of the sm_103a signature-kernel library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sigkernel.h"
#include "sk_projection_table.h"

namespace sk {

constexpr int kNMaxApprox = 16;  // largest order N of the approximation scheme
constexpr int kNMaxInterp = 12;  // largest order N of the interpolation scheme
constexpr int kJMax = 12;        // largest number of series terms kept beyond N (interpolation)
constexpr int kNEMax = 24;       // largest series length - 1 held by a cell (N + J)
constexpr int kLamMax = 8;
constexpr int kDMax = 64;
constexpr int kJF32 = 6;         // interpolation: series terms beyond N kept in FP32
constexpr int kJF64 = 10;        // ... and in FP64
constexpr int kMaxRefined = 131072;  // bound on (rows per path) << lambda (keeps step counters in int32)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kFwdWarps = 4;     // warps per block of the persistent wavefront kernels

// Device error word: the first SK_ERR_* code recorded by any kernel of the library.
extern __device__ int g_sk_error;

__device__ __forceinline__ void record_error(int code) { atomicCAS(&g_sk_error, 0, code); }

// Coefficients that depend only on the (compile-time) indices of the unrolled cell loops are
// constexpr, so they fold into instruction immediates instead of being fetched from the constant
// bank every cell: 1/m, the Hankel coefficient n!/(n+k)!, and the interpolation projection
// kProj (sk_projection_table.h, generated by gen_projection_table.py).
__host__ __device__ constexpr double cx_inv(int m) { return 1.0 / static_cast<double>(m); }
__host__ __device__ constexpr double cx_hank(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r /= static_cast<double>(n + i);
    return r;
}
__host__ __device__ constexpr double cx_rfact(int n) { return cx_hank(0, n); }  // 1/n!

template <typename T> struct Tab;
template <> struct Tab<float> {
    static __device__ __forceinline__ float inv(int m) { return static_cast<float>(cx_inv(m)); }
    static __device__ __forceinline__ float hank(int n, int k) { return static_cast<float>(cx_hank(n, k)); }
    static __device__ __forceinline__ float proj(int N, int n, int jj) { return static_cast<float>(proj_coef(N, n, jj)); }
};
template <> struct Tab<double> {
    static __device__ __forceinline__ double inv(int m) { return cx_inv(m); }
    static __device__ __forceinline__ double hank(int n, int k) { return cx_hank(n, k); }
    static __device__ __forceinline__ double proj(int N, int n, int jj) { return proj_coef(N, n, jj); }
};

// Exact power of two 2^e from its IEEE-754 bits (|e| within the normal range of T).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) {
    return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
}

// Vector type used for increment rows (16-byte loads).
template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
    static __device__ __forceinline__ float dot(float4 a, float4 b, float acc) {
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        return fmaf(a.w, b.w, acc);
    }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
    static __device__ __forceinline__ double dot(double2 a, double2 b, double acc) {
        acc = fma(a.x, b.x, acc);
        return fma(a.y, b.y, acc);
    }
};

// <dx_i, dy_j> over `nvec` 16-byte chunks of zero-padded increment rows (read-only path).
template <typename T>
__device__ __forceinline__ T row_dot(const T* __restrict__ x, const T* __restrict__ y, int nvec) {
    using V = typename Vec<T>::type;
    const V* xv = reinterpret_cast<const V*>(x);
    const V* yv = reinterpret_cast<const V*>(y);
    T acc = T(0);
    for (int c = 0; c < nvec; ++c) acc = Vec<T>::dot(__ldg(xv + c), __ldg(yv + c), acc);
    return acc;
}

// ---------------------------------------------------------------------------------------------
// Pair description shared by the forward and backward kernels.
// ---------------------------------------------------------------------------------------------
enum PairMode : int { kPairsList = 0, kGramFull = 1, kGramUpper = 2 };

struct PathSet {
    const void* inc;         // increments, T[rows_total][dpad], zero padded; the increments of
                             // path a start at row off[a] (points mode leaves its last row unused)
    const int64_t* off;      // caller's row offsets [count + 1]
    int64_t count;
    int64_t max_len;         // caller's bound on rows per path
    int64_t rows_total;      // caller's row count
};

struct PairDesc {
    int64_t a, b;            // path indices
    int64_t xs, ys;          // first increment row of each path
    int64_t lx, ly;          // increments per path (>= 0), or -1 when the path is invalid
};

struct Launch {
    PathSet X, Y;
    int32_t nvec;            // 16-byte chunks per increment row
    int32_t dpad;            // padded row length in elements
    int32_t inc_mode;        // 1 when the caller's rows are increments
    int32_t lam;             // dyadic order
    int32_t mode;            // PairMode
    int64_t npairs;          // work items
    const int64_t* pair_a;
    const int64_t* pair_b;
    const int32_t* order;    // work-item order (NULL = natural)
    unsigned int* queue;     // work counter (zeroed before launch)
    double* out;             // pairs: [npairs]; gram: [X.count][Y.count]
    int64_t ldo;             // leading dimension of a Gram output
    void* scratch;           // per-warp-slot hand-off buffers
    int64_t scratch_stride;  // bytes per warp slot
    float tau;               // |M| above which an FP32 map is built in FP64
    // Optional tape of the forward pass (polynomial schemes): per work item, per warp step, per
    // lane, one row of tape_row<T>(N, interp) elements (see there), plus the exponent of k_hat
    // per item.  NULL when not recorded.
    void* tape;
    int64_t tape_stride;     // bytes per work item
    int* tape_ek;            // [npairs]
    // Cooperative strip pipeline (kernels launched with several warps per pair): a pair with at
    // least this many strips is swept by all warps of a block together; shorter pairs get one
    // warp each.
    int32_t coop_min_strips;
    // Tiled M (polynomial schemes, wide increments): when nonzero, each warp builds the M_ij of
    // a strip (32 rows x cols) in its scratch, at byte offset mtile_off of its slot, two strips
    // deep ([2][32][mtile_cols]), before lane 0 enters the strip; the cells then read M there
    // instead of forming the inner product from two increment rows each.
    int32_t mtile;
    int32_t mtile_cols;
    int64_t mtile_off;
    // Gram modes: work item k of this launch is item k + item_base of the whole Gram (a call can
    // sweep a sub-range of a Gram's items; its tape and queue are indexed by k).
    int64_t item_base;
    // Grid strip pipeline (few long pairs): when nonzero, grid_bpp blocks of the pipelined kernel
    // share each work item, all launched co-resident; block b takes slot b / grid_bpp of the queue
    // order and is part b % grid_bpp of that item's ring of grid_bpp x CW warps.  The ring's
    // progress words are gprog[slot][grid_bpp x CW] in global memory (zeroed before the launch).
    int32_t grid_bpp;
    int* gprog;
    // Polls a strip-pipeline hand-off wait makes before it gives up (0 = kSpinLimit).
    uint32_t wait_limit;
    // Precomputed M (FP32 approximation scheme, one warp per pair): per work item k of the launch,
    // at byte offset k * mx_stride, the cells' M_ij / 4^lambda in the warp's schedule, in groups of
    // four warp steps: lane r's M of steps 4G .. 4G + 3 is the float4 at index 32 G + r.  NULL when
    // the cells form M themselves.
    const float* mx;
    int64_t mx_stride;
};

// Width, in elements of T, of one lane's tape row.
//   Interpolation scheme: the cell's inputs a[0..N], b[0..N], the exponent (element 2N+2) and the
//   cell's M (element 2N+3), padded to 16 bytes.
//   Approximation scheme: the derivatives of the cell's outputs with respect to M,
//   d a'_n / dM (n = 1..N, elements 0..N-1) and d b'_n / dM (elements N..2N-1), the exponent
//   (element 2N) and M (element 2N+1): 2N+2 elements, a whole number of 8-byte halves.  The
//   adjoint needs a and b only through these derivatives (dk/dM = sum_n abar'_n da'_n/dM +
//   bbar'_n db'_n/dM), so each lane's row is two elements shorter and the adjoint forms dk/dM
//   in 2N multiply-adds instead of about 3N^2.
template <typename T>
__host__ __device__ constexpr int tape_row(int N, bool interp) {
    return interp ? ((2 * (N + 1) + 2) * static_cast<int>(sizeof(T)) + 15) / 16 * 16 / static_cast<int>(sizeof(T))
                  : 2 * N + 2;
}

__device__ __forceinline__ int64_t upper_row(int64_t p, int64_t n) {
    // Row a of the upper triangle (a <= b) holding linear index p (row a has n - a entries).
    double nn = static_cast<double>(n);
    double disc = (2.0 * nn + 1.0) * (2.0 * nn + 1.0) - 8.0 * static_cast<double>(p);
    int64_t a = static_cast<int64_t>(floor(((2.0 * nn + 1.0) - sqrt(disc)) * 0.5));
    if (a < 0) a = 0;
    if (a > n - 1) a = n - 1;
    // exact correction: start(a) = a*n - a*(a-1)/2
    while (a > 0 && a * n - a * (a - 1) / 2 > p) --a;
    while (a + 1 < n && (a + 1) * n - (a + 1) * a / 2 <= p) ++a;
    return a;
}

__device__ __forceinline__ void path_span(const PathSet& S, int64_t a, int inc_mode, int64_t& start,
                                          int64_t& len) {
    int64_t r0 = S.off[a], r1 = S.off[a + 1];
    int64_t rows = r1 - r0;
    if (r0 < 0 || r1 > S.rows_total || rows < (inc_mode ? 0 : 1) || rows > S.max_len) {
        start = 0;
        len = -1;
        return;
    }
    start = r0;
    len = inc_mode ? rows : rows - 1;
}

__device__ __forceinline__ PairDesc decode_pair(const Launch& L, int64_t item) {
    PairDesc P;
    if (L.mode == kPairsList) {
        P.a = L.pair_a[item];
        P.b = L.pair_b[item];
    } else if (L.mode == kGramFull) {
        const int64_t gi = item + L.item_base;
        P.a = gi / L.Y.count;
        P.b = gi - P.a * L.Y.count;
    } else {
        const int64_t gi = item + L.item_base;
        int64_t n = L.X.count;
        P.a = upper_row(gi, n);
        P.b = P.a + (gi - (P.a * n - P.a * (P.a - 1) / 2));
    }
    bool okx = P.a >= 0 && P.a < L.X.count, oky = P.b >= 0 && P.b < L.Y.count;
    if (!okx || !oky) {
        P.lx = P.ly = -1;
        P.xs = P.ys = 0;
        return P;
    }
    path_span(L.X, P.a, L.inc_mode, P.xs, P.lx);
    path_span(L.Y, P.b, L.inc_mode, P.ys, P.ly);
    return P;
}

__device__ __forceinline__ void write_result(const Launch& L, int64_t item, const PairDesc& P, double v) {
    if (L.mode == kPairsList) {
        L.out[item] = v;
    } else {
        L.out[P.a * L.ldo + P.b] = v;
        if (L.mode == kGramUpper) L.out[P.b * L.ldo + P.a] = v;
    }
}

// Pop the next work item for a whole block (call from one thread).
__device__ __forceinline__ int64_t pop_item(const Launch& L) {
    const unsigned int k = atomicAdd(L.queue, 1u);
    if (static_cast<int64_t>(k) >= L.npairs) return -1;
    return L.order ? static_cast<int64_t>(L.order[k]) : static_cast<int64_t>(k);
}

// Strip pipeline of a cooperative block: the warp that runs strip g publishes, after writing
// the hand-off entry of column j, the monotonic count g * cols + j + 1 in its shared-memory
// word; the warp that runs strip g + 1 waits for that count before reading the entry.  Release
// and acquire at CTA scope order the hand-off's global-memory stores and loads around it.
constexpr uint32_t kSpinLimit = 1u << 20;  // default polls (with a short sleep) before a wait gives up

__device__ __forceinline__ uint32_t wait_polls(const Launch& L) { return L.wait_limit ? L.wait_limit : kSpinLimit; }

__device__ __forceinline__ void publish_progress(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))),
                 "r"(v)
                 : "memory");
}

__device__ __forceinline__ int acquire_progress(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];"
                 : "=r"(v)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
                 : "memory");
    return v;
}

// Bounded wait for *p >= need (at most `polls` polls); false (and the device error word set) when
// it runs out.
__device__ __forceinline__ bool wait_progress(const int* p, int need, uint32_t polls) {
    for (uint32_t it = 0; it < polls; ++it) {
        if (acquire_progress(p) >= need) return true;
        __nanosleep(64);
    }
    record_error(SK_ERR_DEVICE_TIMEOUT);
    return false;
}

// The same progress words in global memory, ordered at GPU scope, for a ring that spans blocks
// (grid strip pipeline).  The release orders the hand-off entries stored before it; the acquire
// orders the entry loads after it.
__device__ __forceinline__ void publish_progress_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait for *p >= need; *seen gets the value observed (the caller may then read every
// entry up to it without another acquire).  False (and the device error word set) when it runs out.
__device__ __forceinline__ bool wait_progress_gpu(const int* p, int need, int* seen, uint32_t polls) {
    for (uint32_t it = 0; it < polls; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= need) {
            *seen = v;
            return true;
        }
        __nanosleep(64);
    }
    record_error(SK_ERR_DEVICE_TIMEOUT);
    return false;
}

// Columns a ring spanning blocks publishes at once: a GPU-scope release every step stalls the
// publishing lane (and so its warp) far longer than the step itself.
constexpr int kGridPublish = 8;

// Pop the next work item for a warp (lane 0 takes it, all lanes receive it).
__device__ __forceinline__ int64_t next_item(const Launch& L) {
    unsigned int k = 0;
    if ((threadIdx.x & 31) == 0) k = atomicAdd(L.queue, 1u);
    k = __shfl_sync(kFull, k, 0);
    if (static_cast<int64_t>(k) >= L.npairs) return -1;
    return L.order ? static_cast<int64_t>(L.order[k]) : static_cast<int64_t>(k);
}

}  // namespace sk
