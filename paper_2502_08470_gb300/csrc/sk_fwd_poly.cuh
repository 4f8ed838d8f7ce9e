// Forward wavefront of the polynomial schemes (approximation, Section 3.2; interpolation,
// Section 3.3) for sm_103a.
//
// Coordinates.  In a cell with bottom-left corner (s_i, t_j) let u = (s - s_i)/ds and
// v = (t - t_j)/dt.  The bottom edge k(s, t_j) = sum_n p_n (s - s_i)^n is held as the factorial-
// scaled coefficients a_n = n! p_n ds^n (so k(s, t_j) = sum_n a_n u^n / n!), the left edge as
// b_n = n! q_n dt^n.  Substituting into the update of Proposition "approxsolution" (eqs.
// (powerseries1), (powerseries2)) with C ds dt = M = <dx_i, dy_j> gives
//     a'_n = sum_{k<=n} a_k e_{n-k}  +  e_n sum_{k>=1} b_k n!/(n+k)!,      e_m = M^m / m!
//     b'_n = sum_{k<=n} b_k e_{n-k}  +  e_n sum_{k>=1} a_k n!/(n+k)!
// so a cell depends on M only (no time partition), its Toeplitz part is a convolution with the
// truncated exponential e(M), and its coupling part is a constant Hankel matrix n!/(n+k)!.
//   * Approximation (Def. "def:polyapproxscheme"): n = 0..N, i.e. pi_N after Lambda.
//   * Interpolation (Def. "def:polyinterpscheme"): Phi^N of Proposition "propinterp" applied to
//     degree-N edges is the same series untruncated; its factorial-scaled coefficients are
//     computed for n = 0..N+J and Omega^N (interpolation at the N+1 Chebyshev extrema) is the
//     constant projection a' = c_{0..N} + P c_{N+1..N+J}.  The right edge uses a_0 = g_0 in
//     its 0F1(1; z) term, as eq. (interpformula) is printed.
// Endpoint: k_hat = 1/2 sum_n (a_n + b_n)/n! at the last cell (u = v = 1).
//
// Parallel layout.  One warp owns one pair.  Lane r owns grid rows r, r+32, r+64, ... (a
// "strip" of 32 rows at a time).  Cell (32 s + r, j) is updated at warp step s*P + j + r with
// P = max(cols, 32): the a-vector stays in the lane, the b-vector moves one lane up per step
// through __shfl_up_sync, and lane 31's right edges are handed to lane 0 of the next strip
// through a per-warp buffer (written P - 31 >= 1 steps before they are read).  Each warp step
// is one antidiagonal of the strip's cells (Fig. "gridparallel"); consecutive strips overlap so
// no lane idles between them.
//
// FP32 range.  Each lane carries a power-of-two exponent for its (a, b) pair; the two inputs of a
// cell are brought to the larger exponent, and after the update the pair is rescaled by 2^-64
// or 2^64 whenever |a'_0|, |b'_0| leave [2^-64, 2^64].  Exact in binary arithmetic, so results
// change only by rounding.
#pragma once

#include <type_traits>

#include "sk_common.cuh"
#include "sk_tma.cuh"

namespace sk {

template <typename T, int NE>
__device__ __forceinline__ void build_exp_series(T M, float tau, T (&e)[NE + 1]) {
    e[0] = T(1);
    if constexpr (std::is_same<T, float>::value) {
        if (fabsf(M) > tau) {
            // Large |M|: build the map coefficients M^m/m! in FP64 and round once.
            double md = static_cast<double>(M), v = 1.0;
#pragma unroll
            for (int m = 1; m <= NE; ++m) {
                v *= md * cx_inv(m);
                e[m] = static_cast<float>(v);
            }
            return;
        }
    }
    (void)tau;
#pragma unroll
    for (int m = 1; m <= NE; ++m) e[m] = e[m - 1] * (M * Tab<T>::inv(m));
}

// Broadcast of one FP32 value into both halves of a packed pair.
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// One cell: inputs a (bottom), b (left), outputs the factorial-scaled series of the top (ct)
// and right (cr) edges, n = 0..NE:
//     ct_n = sum_{k<=n} a_k e_{n-k} + e_n sum_{k>=1} b_k n!/(n+k)!     (cr_n likewise with a, b
// exchanged; the interpolation scheme's corner term k = 0 is a_0 on both edges).  Since e_0 = 1,
// the k = 0 term joins the coupling, ct_n = e_n (a_0 + H_n(b)) + sum_{1<=k<=n} a_k e_{n-k}, and the
// k = n term is a_n itself: every sum starts from a value it already has, so the cell is all
// fused multiply-adds (28 fewer instructions per cell at N = 6 than starting each sum with a
// product).
template <typename T, int N, int NE, bool INTERP>
__device__ __forceinline__ void cell_series(const T (&a)[N + 1], const T (&b)[N + 1], const T (&e)[NE + 1],
                                            T (&ct)[NE + 1], T (&cr)[NE + 1]) {
#pragma unroll
    for (int n = 0; n <= NE; ++n) {
        // corner term plus the coupling through the opposite edge: c_0 + sum_{k>=1} (.)_k n!/(n+k)!
        T ta = a[0], tb = INTERP ? a[0] : b[0];
#pragma unroll
        for (int k = 1; k <= N; ++k) {
            ta = fma(b[k], Tab<T>::hank(n, k), ta);
            tb = fma(a[k], Tab<T>::hank(n, k), tb);
        }
        if (n == 0) {
            ct[0] = ta;
            cr[0] = tb;
            continue;
        }
        // Toeplitz part without its k = 0 term: sum_{1<=k<=min(n,N)} (.)_k e_{n-k}
        T vt, vr;
        if (n <= N) {
            vt = a[n];
            vr = b[n];
        } else {
            vt = a[N] * e[n - N];
            vr = b[N] * e[n - N];
        }
#pragma unroll
        for (int k = (n <= N ? n : N) - 1; k >= 1; --k) {
            vt = fma(a[k], e[n - k], vt);
            vr = fma(b[k], e[n - k], vr);
        }
        ct[n] = fma(e[n], ta, vt);
        cr[n] = fma(e[n], tb, vr);
    }
}

// The approximation cell (NE = N) as cell_series, bit for bit, plus the derivatives of its outputs
// with respect to M, which are all the adjoint needs of the cell's inputs.  With e_m = M^m/m!
// (d e_m / dM = e_{m-1}) and the Toeplitz sums T_n = sum_{k<=n} a_k e_{n-k}:
//     d a'_n / dM = T_{n-1} + e_{n-1} ha_n,   d b'_n / dM = S_{n-1} + e_{n-1} hb_n   (n = 1..N)
// where S_n is the Toeplitz sum of b; da[n-1] and db[n-1] receive them.  As in cell_series the
// k = 0 term joins the coupling: d a'_{n+1} / dM = e_n (a_0 + ha_{n+1}) + sum_{1<=k<=n} a_k e_{n-k}.
template <typename T, int N>
__device__ __forceinline__ void cell_series_dm(const T (&a)[N + 1], const T (&b)[N + 1], const T (&e)[N + 1],
                                               T (&ct)[N + 1], T (&cr)[N + 1], T (&da)[N], T (&db)[N]) {
    T ta[N + 1], tb[N + 1];  // a_0 + ha_n, b_0 + hb_n
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        ta[n] = a[0];
        tb[n] = b[0];
#pragma unroll
        for (int k = 1; k <= N; ++k) {
            ta[n] = fma(b[k], Tab<T>::hank(n, k), ta[n]);
            tb[n] = fma(a[k], Tab<T>::hank(n, k), tb[n]);
        }
    }
    ct[0] = ta[0];
    cr[0] = tb[0];
    da[0] = ta[1];
    db[0] = tb[1];
#pragma unroll
    for (int n = 1; n <= N; ++n) {
        T vt = a[n], vr = b[n];
#pragma unroll
        for (int k = n - 1; k >= 1; --k) {
            vt = fma(a[k], e[n - k], vt);
            vr = fma(b[k], e[n - k], vr);
        }
        ct[n] = fma(e[n], ta[n], vt);
        cr[n] = fma(e[n], tb[n], vr);
        if (n < N) {
            da[n] = fma(e[n], ta[n + 1], vt);
            db[n] = fma(e[n], tb[n + 1], vr);
        }
    }
}

// Both edges through the interpolation projection.  (Pairing the two edges through the two-wide
// FP32 instructions, as the adjoint does, measured slower here: building the pairs from the
// separately held edges cost more instructions than it saved.)
template <typename T, int N, int NE, bool INTERP>
__device__ __forceinline__ void project_both(const T (&ct)[NE + 1], const T (&cr)[NE + 1], T (&a)[N + 1],
                                             T (&bo)[N + 1]) {
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        T vt = ct[n], vr = cr[n];
        if constexpr (INTERP) {
#pragma unroll
            for (int j = N + 1; j <= NE; ++j) {
                vt = fma(Tab<T>::proj(N, n, j - N - 1), ct[j], vt);
                vr = fma(Tab<T>::proj(N, n, j - N - 1), cr[j], vr);
            }
        }
        a[n] = vt;
        bo[n] = vr;
    }
}

template <typename T, int N, int NE, bool INTERP>
__device__ __forceinline__ void project(const T (&c)[NE + 1], T (&out)[N + 1]) {
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        T v = c[n];
        if constexpr (INTERP) {
#pragma unroll
            for (int j = N + 1; j <= NE; ++j) v = fma(Tab<T>::proj(N, n, j - N - 1), c[j], v);
        }
        out[n] = v;
    }
}

template <typename T, int NE>
__device__ __forceinline__ double series_at_one(const T (&c)[NE + 1]) {
    double acc = 0.0;
#pragma unroll
    for (int n = NE; n >= 0; --n) acc = fma(static_cast<double>(c[n]), cx_rfact(n), acc);
    return acc;
}

template <typename T>
__device__ __forceinline__ T pow2t(int e) {
    if constexpr (std::is_same<T, float>::value) return pow2f(e);
    else return pow2d(e);
}

// Bytes of one warp step of the tape (32 lanes x one row).
template <typename T, int N, bool INTERP>
__host__ __device__ constexpr int fwd_tape_step_bytes() {
    return 32 * tape_row<T>(N, INTERP) * static_cast<int>(sizeof(T));
}

// A lane's exponent stored in a tape element of type T (its bit pattern, read back with
// exponent_from).
template <typename T>
__device__ __forceinline__ T exponent_as(int e) {
    if constexpr (std::is_same<T, float>::value) return __int_as_float(e);
    else return __longlong_as_double(static_cast<long long>(e));
}
template <typename T>
__device__ __forceinline__ int exponent_from(T v) {
    if constexpr (std::is_same<T, float>::value) return __float_as_int(v);
    else return static_cast<int>(__double_as_longlong(v));
}

// Element q of an approximation tape row: d a'_{q+1}/dM (q < N), d b'_{q-N+1}/dM (q < 2N), the
// exponent (q = 2N), M (q = 2N+1).
template <typename T, int N>
__device__ __forceinline__ T dm_row_elem(int q, const T (&da)[N], const T (&db)[N], int ea, T M) {
    return q < N ? da[q] : (q < 2 * N ? db[q - N] : (q == 2 * N ? exponent_as<T>(ea) : M));
}

// One lane's row of an approximation-scheme tape step at `item_tape` (the item's tape): the row's
// whole 16-byte vectors laid out [vector][lane] (each vector store of the warp fills 512
// contiguous bytes), then, when the row has an 8-byte remainder (FP32 with N even), that half
// laid out [lane] (256 contiguous bytes).  Streaming (evict-first) stores: the adjoint reads the
// tape only after the whole forward.
template <typename T, int N>
__device__ __forceinline__ void store_dm_row(char* item_tape, int step, int lane, const T (&da)[N], const T (&db)[N],
                                             int ea, T M) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int TR = tape_row<T>(N, false);
    constexpr int NV = TR / W;
    char* base = item_tape + static_cast<int64_t>(step) * fwd_tape_step_bytes<T, N, false>();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        V t;
        T* tp = reinterpret_cast<T*>(&t);
#pragma unroll
        for (int q2 = 0; q2 < W; ++q2) tp[q2] = dm_row_elem<T, N>(v * W + q2, da, db, ea, M);
        __stcs(reinterpret_cast<V*>(base) + v * 32 + lane, t);
    }
    if constexpr (TR % W != 0) {
        static_assert(std::is_same<T, float>::value && TR % W == 2, "8-byte remainder of an FP32 row");
        const float2 t = make_float2(dm_row_elem<T, N>(NV * W, da, db, ea, M), dm_row_elem<T, N>(NV * W + 1, da, db, ea, M));
        __stcs(reinterpret_cast<float2*>(base + NV * 32 * 16) + lane, t);
    }
}

// Resident blocks per SM requested from the register allocator: the live state of a lane is
// about 3 (N+1) edge values, 3 (NE+1) series values and ~24 addresses / counters (plus, with
// tiled M, the producer's 16 accumulators, one 16-byte chunk and its buffer addresses).
template <typename T, int N, int NE, bool MT = false>
constexpr int fwd_poly_min_blocks() {
    constexpr int words = (3 * (N + 1) + 3 * (NE + 1) + 24 + (MT ? 28 : 0)) * (sizeof(T) == 8 ? 2 : 1);
    constexpr int b = 65536 / (kFwdWarps * 32 * words);
    return b < 1 ? 1 : (b > 8 ? 8 : b);
}

// Tiled M for strip g: M[r][c] = <dx_{row}, dy_c> / 4^lambda for the strip's 32 rows and every
// column, written to dst ([32][mcols], rows past the last grid row left unwritten).  Lane q owns
// columns q, q + 32, ... and keeps that increment row in registers a 16-byte chunk at a time; the
// strip's x rows sit in shared memory (xs, [32][dpad]) and are read as broadcasts, so 32 cells
// share each operand load instead of each cell gathering two rows.  The inner products run in
// row_dot's order, so M is bit for bit the value row_dot gives.
template <typename T>
__device__ __forceinline__ void produce_m_strip(const T* __restrict__ xbase, const T* __restrict__ ybase, int dpad,
                                                int lam, int rows, int cols, int g, T sub, T* xs, T* dst, int mcols) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int RH = 16;  // rows per pass (accumulators per lane)
    const int lane = threadIdx.x & 31;
    __syncwarp();  // earlier readers of xs are done
    {
        const T* xr = xbase + static_cast<int64_t>(min((g << 5) + lane, rows - 1) >> lam) * dpad;
        for (int k = 0; k < dpad; k += W)
            *reinterpret_cast<V*>(xs + lane * dpad + k) = __ldg(reinterpret_cast<const V*>(xr + k));
    }
    __syncwarp();
    for (int c0 = 0; c0 < cols; c0 += 32) {
        const int c = c0 + lane;
        const V* yv = reinterpret_cast<const V*>(ybase + static_cast<int64_t>(min(c, cols - 1) >> lam) * dpad);
#pragma unroll 1
        for (int rh = 0; rh < 32; rh += RH) {
            T acc[RH];
#pragma unroll
            for (int r = 0; r < RH; ++r) acc[r] = T(0);
            for (int k = 0; k < dpad / W; ++k) {
                const V y = __ldg(yv + k);
#pragma unroll
                for (int r = 0; r < RH; ++r)
                    acc[r] = Vec<T>::dot(*reinterpret_cast<const V*>(xs + (rh + r) * dpad + k * W), y, acc[r]);
            }
            if (c < cols) {
#pragma unroll
                for (int r = 0; r < RH; ++r)
                    if ((g << 5) + rh + r < rows) dst[static_cast<int64_t>(rh + r) * mcols + c] = acc[r] * sub;
            }
        }
    }
    __syncwarp();  // the strip's M is visible to every lane
}

// Warps of a block that sweep one long pair together (strip pipeline); see sweep_poly.  Sixteen
// measured faster than eight both on few long pairs (64 pairs of 1025-point paths: 4.6 against
// 5.8 ms) and on uneven batches (4096 pairs of 64..4096-point paths: 101 against 121 ms).
constexpr int kCoopWarps = 16;

template <typename T, int N, int NE, bool MT = false>
constexpr int fwd_poly_coop_min_blocks() {
    // Two 16-warp blocks per SM (64 registers) measured faster for the approximation scheme up to
    // order 6 in FP32, despite a few spilled registers: 4096 pairs of 64..4096-point paths ran in
    // 83.7 ms against 101.4 ms.  The interpolation scheme's longer series spill more, and it ran
    // slower that way (64 pairs of 1025-point oscillatory paths: 5.47 against 4.76 ms), so it
    // keeps one block.
    if constexpr (std::is_same<T, float>::value && NE == N && N <= 6 && !MT) return 2;
    constexpr int b = fwd_poly_min_blocks<T, N, NE, MT>() * kFwdWarps / kCoopWarps;
    return b < 1 ? 1 : b;
}

// Sweep of one pair by one warp (CW = 1), or by warp w of a ring of `ring` warps that share it:
// warp w runs strips w, w + ring, w + 2 ring, ... in the same overlapped schedule a single warp
// uses for all of them (local strip sigma starts at local step sigma * P).  Lane 31 of strip g
// writes its right edges into this warp's hand-off buffer (own_buf); lane 0 of strip g + 1 reads
// them from the buffer of the warp that ran strip g (prev_buf, the warp's own buffer when
// CW = 1).  In a ring the hand-off is ordered by the progress words prog[]; a buffer entry of
// strip g is overwritten by strip g + ring only after strip g + 1 has consumed it, because strip
// g + ring depends on strip g + 1 through the chain of strips in between.
//
// The ring is the CW warps of one block (ring = CW, progress words in shared memory, CTA-scope
// ordering), or, with GS, blocks x CW warps spread over co-resident blocks (progress words in
// global memory, GPU-scope ordering, published every kGridPublish columns).
template <typename T, int N, int NE, bool INTERP, int CW, bool MT, bool GS = false, bool DMT = false, bool MX = false>
__device__ __forceinline__ void sweep_poly(const Launch& L, int64_t item, const PairDesc& P, int w, char* own_buf,
                                           const char* prev_buf, int* prog, int64_t buf_cols, T* xstage,
                                           int ring = CW) {
    constexpr bool kRescale = std::is_same<T, float>::value;
    static_assert(!MX || (CW == 1 && !MT && std::is_same<T, float>::value), "precomputed M: FP32, one warp per pair");
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int NB = (N + 1 + W - 1) / W * W;  // hand-off entry width, padded to whole vectors
    const int lane = threadIdx.x & 31;
    V* hbuf = reinterpret_cast<V*>(own_buf);                                                // [buf_cols][NB / W]
    int* ebuf = reinterpret_cast<int*>(own_buf + buf_cols * NB * static_cast<int64_t>(sizeof(T)));
    const V* hprev = reinterpret_cast<const V*>(prev_buf);
    const int* eprev = reinterpret_cast<const int*>(prev_buf + buf_cols * NB * static_cast<int64_t>(sizeof(T)));
    const int dpad = L.dpad;
    const T* __restrict__ incX = static_cast<const T*>(L.X.inc);
    const T* __restrict__ incY = static_cast<const T*>(L.Y.inc);

    const int lam = L.lam;
    const int rows = static_cast<int>(P.lx << lam);
    const int cols = static_cast<int>(P.ly << lam);
    // Period of a warp's strips.  Alone, a warp starts its next strip as soon as lane 0 is free
    // (P = max(cols, 32)).  In a cooperative block that overlap can deadlock: a warp whose lane 0
    // waits on the ring of other warps also holds back its lanes still publishing the previous
    // strip, which those warps need.  A warp therefore starts strip k + 1 only after finishing
    // strip k (P = cols + 31), unless the rows are longer than the ring's lag (cols > 31 CW),
    // where the overlapped schedule keeps every wait pointed at finished work.  A model of this
    // schedule (tests/test_pipeline_schedule.py) checks the rule and the deadlock it avoids.
    // A ring spanning blocks publishes its progress every kGridPublish columns, which lengthens
    // the lag the overlapped schedule must exceed (the schedule model checks this rule too).
    constexpr int kLag = GS ? 31 + kGridPublish : 31;
    const int period = CW == 1 ? (cols > 32 ? cols : 32) : (cols > kLag * ring ? cols : cols + 31);
    const int nstrips = (rows + 31) >> 5;
    const int last_lane = (rows - 1) - ((nstrips - 1) << 5);
    // this warp's strips: w, w + ring, ...; the one holding the last row ends at lane last_lane
    const int nloc = w < nstrips ? (nstrips - 1 - w) / ring + 1 : 0;
    if (nloc == 0) return;
    const bool has_last = (nstrips - 1) % ring == w;
    const int nsteps = (nloc - 1) * period + (has_last ? last_lane : 31) + cols;
    const T sub = pow2t<T>(-2 * lam);  // M of a sub-cell of P_lambda is M_ij / 4^lambda
    const T* xbase = incX + P.xs * dpad;
    const T* ybase = incY + P.ys * dpad;

    T a[N + 1], bo[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) { a[n] = T(0); bo[n] = T(0); }
    int ea = 0, eo = 0;
    int jj = -lane, sl = 0;                 // column and local strip of this lane
    int g = w, row = (w << 5) + lane;       // global strip and grid row
    bool stuck = false;                     // a hand-off wait ran out (CW > 1 only)
    int seen = 0;                           // progress of the warp before, as last observed (GS)
    const T* xrow = xbase + static_cast<int64_t>(min(row, rows - 1) >> lam) * dpad;
    // tiled M (MT): this warp's [2][32][mcols] strip buffers; lane 0's column and local strip
    const int mcols = MT ? L.mtile_cols : 0;
    T* mbuf = MT ? reinterpret_cast<T*>(own_buf + L.mtile_off) : nullptr;
    int jj0 = 0, sl0 = 0;
    // precomputed M (MX): this item's groups of four warp steps (lane r's M of steps 4G .. 4G + 3 in
    // the float4 32 G + r).  Group G + 1 is loaded on entering group G, four to seven steps ahead of
    // its use: the groups come from HBM, and a step's cell arithmetic alone does not cover the load
    // latency (measured: the sweep of 256 x 256 / 2 pairs of 513-point paths took 112 ms reading M
    // at its step and 77 ms reading ahead).
    const float4* mxi = MX ? reinterpret_cast<const float4*>(reinterpret_cast<const char*>(L.mx) + item * L.mx_stride)
                           : nullptr;
    float4 mcur = make_float4(0.f, 0.f, 0.f, 0.f), mnxt = mcur;
    if constexpr (MX) mnxt = __ldcs(mxi + lane);  // group 0

    for (int step = 0; step < nsteps; ++step) {
        if constexpr (MT) {
            if (jj0 == 0 && sl0 < nloc)  // lane 0 enters local strip sl0: build its M first
                produce_m_strip<T>(xbase, ybase, dpad, lam, rows, cols, w + sl0 * ring, sub, xstage,
                                   mbuf + (sl0 & 1) * 32 * static_cast<int64_t>(mcols), mcols);
            if (++jj0 == period) {
                jj0 = 0;
                ++sl0;
            }
        }
        T b[N + 1];
#pragma unroll
        for (int n = 0; n <= N; ++n) b[n] = __shfl_up_sync(kFull, bo[n], 1);
        int eb = kRescale ? __shfl_up_sync(kFull, eo, 1) : 0;
        const bool active = static_cast<unsigned>(jj) < static_cast<unsigned>(cols) && row < rows && sl < nloc;
        if (active && lane == 0) {
            if (g == 0) {  // q^{0,j} = e_0 (left boundary k(0, .) = 1)
#pragma unroll
                for (int n = 0; n <= N; ++n) b[n] = (n == 0) ? T(1) : T(0);
                eb = 0;
            } else {
                if constexpr (CW > 1) {
                    const int* pp = prog + (w + ring - 1) % ring;
                    if constexpr (GS) {
                        const int need = (g - 1) * cols + jj + 1;
                        if (!stuck && seen < need && !wait_progress_gpu(pp, need, &seen, wait_polls(L))) stuck = true;
                    } else {
                        if (!stuck && !wait_progress(pp, (g - 1) * cols + jj + 1, wait_polls(L))) stuck = true;
                    }
                }
                const V* src = hprev + static_cast<int64_t>(jj) * (NB / W);
#pragma unroll
                for (int v = 0; v < NB / W; ++v) {
                    const V t = src[v];
                    const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
                    for (int q = 0; q < W; ++q)
                        if (v * W + q <= N) b[v * W + q] = tp[q];
                }
                if (kRescale) eb = eprev[jj];
            }
        }
        if (active && jj == 0) {  // p^{i,0} = e_0 (bottom boundary k(., 0) = 1)
#pragma unroll
            for (int n = 0; n <= N; ++n) a[n] = (n == 0) ? T(1) : T(0);
            ea = 0;
        }
        if (kRescale && active && ea != eb) {  // bring both inputs to the larger exponent
            if (ea > eb) {
                const T f = (eb - ea < -126) ? T(0) : pow2t<T>(eb - ea);
#pragma unroll
                for (int n = 0; n <= N; ++n) b[n] *= f;
            } else {
                const T f = (ea - eb < -126) ? T(0) : pow2t<T>(ea - eb);
#pragma unroll
                for (int n = 0; n <= N; ++n) a[n] *= f;
                ea = eb;
            }
        }
        // Every lane runs the cell (inactive lanes on a clamped, in-bounds column); only
        // the results of active lanes are ever consumed.
        const int jc = min(max(jj, 0), cols - 1);
        T M;
        if constexpr (MT) M = active ? mbuf[((sl & 1) * 32 + lane) * static_cast<int64_t>(mcols) + jc] : T(0);
        else if constexpr (MX) {
            if ((step & 3) == 0) {  // entering group step / 4: its M was read a group ago
                mcur = mnxt;
                const int gn = (step >> 2) + 1;
                if (4 * gn < nsteps) mnxt = __ldcs(mxi + static_cast<int64_t>(gn) * 32 + lane);
            }
            M = active ? mcur.x : T(0);
            mcur = make_float4(mcur.y, mcur.z, mcur.w, 0.f);
        }
        else M = row_dot<T>(xrow, ybase + static_cast<int64_t>(jc >> lam) * dpad, L.nvec) * sub;
        if constexpr (CW == 1 && INTERP) {
            if (L.tape != nullptr) {
                // Interpolation scheme: record the cell's inputs (a, b, exponent, M) for the
                // adjoint.  A step of the tape is laid out [vector][lane] (16-byte vectors), so
                // each of the lane's vector stores fills 512 contiguous bytes with the warp's other
                // lanes.  The stores are streaming (evict-first): the adjoint reads the tape only
                // after the whole forward (12.4 ms for the 128x128 Gram's forward, against 13.3 ms
                // with plain or L2-only stores).
                constexpr int TR = tape_row<T>(N, true);
                constexpr int kStepBytes = 32 * TR * static_cast<int>(sizeof(T));
                V* dst = reinterpret_cast<V*>(static_cast<char*>(L.tape) + item * L.tape_stride +
                                              static_cast<int64_t>(step) * kStepBytes);
#pragma unroll
                for (int v = 0; v < TR / W; ++v) {
                    V t;
                    T* tp = reinterpret_cast<T*>(&t);
#pragma unroll
                    for (int q2 = 0; q2 < W; ++q2) {
                        const int q = v * W + q2;
                        tp[q2] = q <= N ? a[q] : (q <= 2 * N + 1 ? b[q - N - 1] : T(0));
                        if (q == 2 * N + 2) tp[q2] = exponent_as<T>(ea);
                        if (q == 2 * N + 3) tp[q2] = M;
                    }
                    __stcs(dst + v * 32 + lane, t);
                }
            }
        }
        T e[NE + 1];
        build_exp_series<T, NE>(M, L.tau, e);
        T ct[NE + 1], cr[NE + 1];
        if constexpr (DMT) {
            // Approximation scheme with a tape: the cell also gives the derivatives of its outputs
            // with respect to M, recorded (with the inputs' exponent and M) in place of the inputs.
            T da[N], db[N];
            cell_series_dm<T, N>(a, b, e, ct, cr, da, db);
            store_dm_row<T, N>(static_cast<char*>(L.tape) + item * L.tape_stride, step, lane, da, db, ea, M);
        } else {
            cell_series<T, N, NE, INTERP>(a, b, e, ct, cr);
        }
        if constexpr (INTERP) {
            if (active && row == rows - 1 && jj == cols - 1) {
                const double v0 = 0.5 * (series_at_one<T, NE>(ct) + series_at_one<T, NE>(cr));
                const double v = kRescale ? ldexp(v0, ea) : v0;
                if (!isfinite(v)) record_error(SK_ERR_NONFINITE);
                write_result(L, item, P, v);
                if (L.tape_ek != nullptr) {
                    int e2 = 0;
                    if (v0 != 0.0) frexp(v0, &e2);
                    L.tape_ek[item] = (kRescale ? ea : 0) + e2;
                }
            }
        }
        project_both<T, N, NE, INTERP>(ct, cr, a, bo);
        if (kRescale && (step & 3) == 0 && active) {
            const float mag = fmaxf(fabsf(static_cast<float>(a[0])), fabsf(static_cast<float>(bo[0])));
            if (mag > 0x1p64f) {
#pragma unroll
                for (int n = 0; n <= N; ++n) { a[n] *= pow2t<T>(-64); bo[n] *= pow2t<T>(-64); }
                ea += 64;
            } else if (mag < 0x1p-64f) {
                float full = 0.f;
#pragma unroll
                for (int n = 0; n <= N; ++n)
                    full = fmaxf(full, fmaxf(fabsf(static_cast<float>(a[n])), fabsf(static_cast<float>(bo[n]))));
                if (full < 0x1p-64f && full > 0.f) {
#pragma unroll
                    for (int n = 0; n <= N; ++n) { a[n] *= pow2t<T>(64); bo[n] *= pow2t<T>(64); }
                    ea -= 64;
                }
            }
        }
        eo = ea;
        if (active && lane == 31 && g + 1 < nstrips) {  // hand the right edge to the next strip
            V* dst = hbuf + static_cast<int64_t>(jj) * (NB / W);
#pragma unroll
            for (int v = 0; v < NB / W; ++v) {
                V t;
                T* tp = reinterpret_cast<T*>(&t);
#pragma unroll
                for (int q = 0; q < W; ++q) tp[q] = (v * W + q <= N) ? bo[v * W + q] : T(0);
                dst[v] = t;
            }
            if (kRescale) ebuf[jj] = eo;
            if constexpr (CW > 1) {
                if constexpr (GS) {
                    if ((jj + 1) % kGridPublish == 0 || jj == cols - 1) publish_progress_gpu(prog + w, g * cols + jj + 1);
                } else {
                    publish_progress(prog + w, g * cols + jj + 1);
                }
            }
        }
        __syncwarp();
        if (++jj == period) {
            jj = 0;
            ++sl;
            g += ring;
            row += 32 * ring;
            xrow = xbase + static_cast<int64_t>(min(row, rows - 1) >> lam) * dpad;
        }
    }
    if constexpr (!INTERP) {
        // The last cell was the final step of lane `last_lane` in the warp holding the last
        // strip; for the approximation scheme its outputs are still in (a, bo):
        // k_hat = 1/2 sum_n (a_n + b_n) / n!.
        if (has_last && lane == last_lane) {
            const double v0 = 0.5 * (series_at_one<T, N>(a) + series_at_one<T, N>(bo));
            const double v = kRescale ? ldexp(v0, ea) : v0;
            if (!isfinite(v)) record_error(SK_ERR_NONFINITE);
            write_result(L, item, P, v);
            if (L.tape_ek != nullptr) {
                int e2 = 0;
                if (v0 != 0.0) frexp(v0, &e2);
                L.tape_ek[item] = (kRescale ? ea : 0) + e2;
            }
        }
    }
}

// Result of a pair that has no cells (or bad lengths); false when the pair needs a sweep.
__device__ __forceinline__ bool trivial_pair(const Launch& L, int64_t item, const PairDesc& P) {
    if (P.lx < 0 || P.ly < 0) {
        if ((threadIdx.x & 31) == 0) {
            record_error(SK_ERR_BAD_LENGTH);
            if (P.a >= 0 && P.a < L.X.count && P.b >= 0 && P.b < L.Y.count)
                write_result(L, item, P, __longlong_as_double(0x7ff8000000000000LL));
        }
        return true;
    }
    if (P.lx == 0 || P.ly == 0) {
        if ((threadIdx.x & 31) == 0) write_result(L, item, P, 1.0);
        return true;
    }
    return false;
}

// Forward wavefront, persistent.  MT: tiled M (produce_m_strip) instead of per-cell inner
// products.  CW = 1: blocks of kFwdWarps independent warps, one pair per warp.  CW > 1: blocks of
// CW warps; the block takes pairs of at least L.coop_min_strips strips together (strip pipeline,
// sweep_poly<..., CW>), and at the first shorter pair (the queue is ordered by cell count, longest
// first) its warps fall back to one pair each.  DMT (approximation scheme, CW = 1): record the
// tape of output derivatives with respect to M (L.tape must be set); the interpolation kernels
// record their tape of cell inputs whenever L.tape is set.  MX (FP32 approximation scheme,
// CW = 1): the cells read M from the buffer L.mx that the tensor-core M kernel wrote.
template <typename T, int N, int NE, bool INTERP, int CW, bool MT, bool DMT = false, bool MX = false>
__global__ void __launch_bounds__((CW > 1 ? CW : kFwdWarps) * 32,
                                  (CW > 1 ? fwd_poly_coop_min_blocks<T, N, NE, MT>() : fwd_poly_min_blocks<T, N, NE, MT>()))
    fwd_poly_kernel(Launch L, int64_t buf_cols) {
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    char* block_base = static_cast<char*>(L.scratch) + static_cast<int64_t>(blockIdx.x) * nw * L.scratch_stride;
    char* own = block_base + wib * L.scratch_stride;
    // dynamic shared memory: the x rows of the tiled-M producer ([32][dpad] per warp, with L.mtile)
    extern __shared__ __align__(128) unsigned char fwd_smem[];
    T* xstage = reinterpret_cast<T*>(fwd_smem) + wib * 32 * L.dpad;

    if constexpr (CW > 1) {
        if (L.grid_bpp > 0) {  // grid strip pipeline: this block is part k of its slot's ring
            const int bpp = L.grid_bpp;
            const int64_t slot = blockIdx.x / bpp;
            const int k = static_cast<int>(blockIdx.x - slot * bpp);
            if (slot >= L.npairs) return;
            const int64_t item = L.order ? static_cast<int64_t>(L.order[slot]) : slot;
            const PairDesc P = decode_pair(L, item);
            if (trivial_pair(L, item, P)) return;
            const int ring = bpp * CW;
            const int wr = k * CW + wib;                 // this warp's place in the ring
            const int pw = (wr + ring - 1) % ring;       // the warp before it
            const char* prev = static_cast<char*>(L.scratch) +
                               ((slot * bpp + pw / CW) * nw + pw % CW) * L.scratch_stride;
            sweep_poly<T, N, NE, INTERP, CW, MT, true>(L, item, P, wr, own, prev, L.gprog + slot * ring, buf_cols,
                                                       xstage, ring);
            return;
        }
        __shared__ long long s_item;
        __shared__ int s_prog[CW];
        for (;;) {
            if (threadIdx.x == 0) s_item = pop_item(L);
            __syncthreads();
            const int64_t item = s_item;
            if (threadIdx.x < CW) s_prog[threadIdx.x] = 0;
            __syncthreads();  // every warp has read s_item and sees the cleared progress words
            if (item < 0) return;
            const PairDesc P = decode_pair(L, item);
            const int nstrips = P.lx > 0 ? static_cast<int>(((P.lx << L.lam) + 31) >> 5) : 0;
            if (nstrips < L.coop_min_strips) {  // short pairs from here on: one warp each
                if (wib == 0 && !trivial_pair(L, item, P))
                    sweep_poly<T, N, NE, INTERP, 1, MT>(L, item, P, 0, own, own, nullptr, buf_cols, xstage);
                break;
            }
            if (!trivial_pair(L, item, P))
                sweep_poly<T, N, NE, INTERP, CW, MT>(L, item, P, wib, own, block_base + ((wib + CW - 1) % CW) * L.scratch_stride,
                                                 s_prog, buf_cols, xstage);
        }
    }
    for (;;) {
        const int64_t item = next_item(L);
        if (item < 0) break;
        const PairDesc P = decode_pair(L, item);
        if (trivial_pair(L, item, P)) continue;
        sweep_poly<T, N, NE, INTERP, 1, MT, false, DMT, MX>(L, item, P, 0, own, own, nullptr, buf_cols, xstage);
    }
}

}  // namespace sk
