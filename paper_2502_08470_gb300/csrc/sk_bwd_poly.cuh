// Reverse-mode derivative (adjoint wavefront) of the polynomial approximation scheme for
// sm_103a.  The paper defines no gradient; this is the exact adjoint of the scheme's own
// arithmetic (Definition "def:polyapproxscheme" in the factorial-scaled form of sk_fwd_poly.cuh).
//
// Adjoint of one cell.  With e_m = M^m/m!, H_nk = n!/(n+k)!, ha_n = sum_{k>=1} b_k H_nk,
// hb_n = sum_{k>=1} a_k H_nk and the forward map a'_n = sum_{k<=n} a_k e_{n-k} + e_n ha_n,
// b'_n = sum_{k<=n} b_k e_{n-k} + e_n hb_n, the adjoints (abar' of a', bbar' of b') give
//     abar_k = sum_{n>=k} abar'_n e_{n-k} + [k>=1] sum_n (bbar'_n e_n) H_nk
//     bbar_k = sum_{n>=k} bbar'_n e_{n-k} + [k>=1] sum_n (abar'_n e_n) H_nk
//     ebar_m = sum_{n>=m} (abar'_n a_{n-m} + bbar'_n b_{n-m}) + abar'_m ha_m + bbar'_m hb_m
//     Mbar   = sum_{m>=1} ebar_m e_{m-1}                       (d e_m / dM = e_{m-1})
// The endpoint 1/2 sum_n (a_n + b_n)/n! seeds abar' = bbar' = 1/(2 n!) at the last cell.  A sub-cell
// of P_lambda has M = M_ij / 4^lambda, so dk/dM_ij sums the sub-cell Mbar / 4^lambda, and
// d k / d dx_i = sum_j (dk/dM_ij) dy_j, d k / d dy_j = sum_i (dk/dM_ij) dx_i.
//
// Schedule of the checkpointing adjoint (one warp per pair, same lane/strip layout as the forward
// kernel; memory per warp slot: the pair's strip hand-offs and one strip's tape):
//   F  forward replay of the whole pair; every strip's hand-off column (the checkpoints) goes to
//      per-warp scratch and the exponent of k_hat is kept.
//   for each 32-row strip, from the top one down:
//   R1 re-run the strip's forward from its hand-off column, recording each cell's output
//      derivatives with respect to M, exponent and M (the forward tape's rows) in a per-warp
//      strip tape;
//   R2 walk the strip's steps backward from that tape (each lane copies its rows into a
//      shared-memory ring K steps ahead) applying the adjoint.  The right-edge adjoint moves one
//      lane down per step (__shfl_down_sync) together with the column partial sums of dk/dy
//      (lane 0 adds them into a per-warp row of the pair's columns, added to the y gradient once
//      per pair), lane 0 hands the adjoint to lane 31 of the strip below through a per-warp
//      buffer, and each lane keeps dk/dx of its row in shared memory.
// FP32 keeps power-of-two exponents per lane for the forward values (as in the forward kernel)
// and, separately, for the adjoints; dk/dM is accumulated relative to 2^E(k) of the pair.
#pragma once

#include <type_traits>

#include "sk_fwd_poly.cuh"
#include "sk_tma.cuh"
#include "sk_umma.cuh"

namespace sk {

constexpr int kZeroExp = -(1 << 20);  // exponent tag of an all-zero adjoint

struct BwdParams {
    Launch L;                 // pairs, increments, queue, order, per-warp scratch
    const double* gout;       // upstream gradient (pairs: [npairs]; Gram: [X.count][Y.count])
    double* gincX;            // d L / d increments of X, [X.rows_total][dpad]
    double* gincY;            // same for Y (may alias gincX)
    int64_t cols_max;         // refined columns a hand-off buffer holds
    int64_t strips_max;       // strips of the longest x path
    int64_t off_fbuf, off_fexp, off_rbuf, off_rexp, off_ybar;  // byte offsets inside a warp slot
    void* mbuf;               // tape adjoint: per-item dk/dM, [step][lane] of T (or tiles, gtile)
    int64_t mb_stride;        // bytes per item of mbuf
    int64_t acc_bytes;        // contraction: shared-memory column accumulator bytes per block
    // Tensor-core contraction (FP32): the adjoint writes dk/dM as BF16 hi/lo tiles (gtile_index)
    // of gt_ncb column blocks per row block, and the contraction reads them with bulk copies.
    int32_t gtile;
    int32_t gt_ncb;
    const void* xt;           // transposed, split increments of X / Y (tc_operand_offset), or NULL
    const void* yt;
    int32_t xt_nblk, yt_nblk; // 128-row blocks per path in xt / yt
};

// dk/dM tiles for the tensor-core contraction.  An item's buffer holds 128 x 128 blocks of the
// refined cell grid (row block i / 128, column block j / 128; gt_ncb column blocks per row block),
// 64 KB each: the BF16 high parts of the 128 x 128 values, then their BF16 low parts
// (value - high, rounded).  Within a plane, the values sit in 8 x 8 "core matrices" of 128
// contiguous bytes, core matrix ((i % 128) / 8, (j % 128) / 8) at index ((i % 128) / 8) * 16 +
// (j % 128) / 8, element (i % 8, j % 8) at (i % 8) * 8 + (j % 8).  That is the layout the tensor
// core reads without swizzling, both as a row-major (K = j) operand and as its transpose (K = i).
__device__ __forceinline__ int64_t gtile_index(int i, int j, int ncb) {
    const int64_t blk = static_cast<int64_t>(i >> 7) * ncb + (j >> 7);
    const int ii = i & 127, jj = j & 127;
    return blk * 32768 + ((ii >> 3) * 16 + (jj >> 3)) * 64 + (ii & 7) * 8 + (jj & 7);
}
constexpr int kGtilePlane = 16384;  // BF16 elements of one plane of a block

// Zero both planes of the cells of an item's padded tile grid that lie outside its rows x cols
// (the tensor-core contraction sums over whole 128-cell blocks).  One warp.
__device__ __forceinline__ void gtile_zero_padding(void* item_tiles, int rows, int cols, int ncb) {
    const int lane = threadIdx.x & 31;
    __nv_bfloat16* gt = static_cast<__nv_bfloat16*>(item_tiles);
    const int rpad = (rows + 127) & ~127, cpad = (cols + 127) & ~127;
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    for (int i = rows; i < rpad; ++i)
        for (int j = lane; j < cpad; j += 32) {
            const int64_t q = gtile_index(i, j, ncb);
            gt[q] = z;
            gt[q + kGtilePlane] = z;
        }
    for (int i = 0; i < rows; ++i)
        for (int j = cols + lane; j < cpad; j += 32) {
            const int64_t q = gtile_index(i, j, ncb);
            gt[q] = z;
            gt[q + kGtilePlane] = z;
        }
}

template <typename T>
__device__ __forceinline__ T pow2c(int e) {  // 2^e, or 0 below the normal range
    if constexpr (std::is_same<T, float>::value) return e < -126 ? 0.f : pow2f(e > 127 ? 127 : e);
    else return e < -1022 ? 0.0 : pow2d(e > 1023 ? 1023 : e);
}

template <typename T, int N>
__device__ __forceinline__ void set_unit(T (&v)[N + 1]) {
#pragma unroll
    for (int n = 0; n <= N; ++n) v[n] = (n == 0) ? T(1) : T(0);
}

// Bring (a, ea) and (b, eb) to the larger exponent (FP32 only).
template <typename T, int N>
__device__ __forceinline__ void align_inputs(T (&a)[N + 1], int& ea, T (&b)[N + 1], int eb) {
    if (ea == eb) return;
    if (ea > eb) {
        const T f = pow2c<T>(eb - ea);
#pragma unroll
        for (int n = 0; n <= N; ++n) b[n] *= f;
    } else {
        const T f = pow2c<T>(ea - eb);
#pragma unroll
        for (int n = 0; n <= N; ++n) a[n] *= f;
        ea = eb;
    }
}

// The replays' renormalisation of a cell's outputs (a, bo) by 2^-+64 into exponent ea (FP32).
template <typename T, int N>
__device__ __forceinline__ void rescale_edges(T (&a)[N + 1], T (&bo)[N + 1], int& ea) {
    if constexpr (std::is_same<T, float>::value) {
        const float mag = fmaxf(fabsf(a[0]), fabsf(bo[0]));
        if (mag > 0x1p64f) {
#pragma unroll
            for (int n = 0; n <= N; ++n) { a[n] *= 0x1p-64f; bo[n] *= 0x1p-64f; }
            ea += 64;
        } else if (mag < 0x1p-64f) {
            float full = 0.f;
#pragma unroll
            for (int n = 0; n <= N; ++n) full = fmaxf(full, fmaxf(fabsf(a[n]), fabsf(bo[n])));
            if (full < 0x1p-64f && full > 0.f) {
#pragma unroll
                for (int n = 0; n <= N; ++n) { a[n] *= 0x1p64f; bo[n] *= 0x1p64f; }
                ea -= 64;
            }
        }
    }
}

// One forward cell of the approximation scheme with the replays' renormalisation:
// (a, b) -> (a, bo) in place, exponent ea.
template <typename T, int N>
__device__ __forceinline__ void fwd_cell(T (&a)[N + 1], const T (&b)[N + 1], T M, float tau, T (&bo)[N + 1],
                                         int& ea) {
    T e[N + 1], ct[N + 1], cr[N + 1];
    build_exp_series<T, N>(M, tau, e);
    cell_series<T, N, N, false>(a, b, e, ct, cr);
#pragma unroll
    for (int n = 0; n <= N; ++n) { a[n] = ct[n]; bo[n] = cr[n]; }
    rescale_edges<T, N>(a, bo, ea);
}

// Scale a cell's forward inputs to magnitude ~1 by an exact power of two (FP32), folding the shift
// into their exponent, so that products with adjoints (kept within 2^+-64) cannot overflow.
template <typename T, int N>
__device__ __forceinline__ void unit_scale(T (&fa)[N + 1], T (&fb)[N + 1], int& ef) {
    if constexpr (std::is_same<T, float>::value) {
        const float m = fmaxf(fabsf(fa[0]), fabsf(fb[0]));
        if (m > 0x1p16f || (m < 0x1p-16f && m > 0.f)) {
            int sh = 0;
            frexpf(m, &sh);
            const float f = pow2c<float>(-sh);
#pragma unroll
            for (int n = 0; n <= N; ++n) { fa[n] *= f; fb[n] *= f; }
            ef += sh;
        }
    }
}

// Edge adjoints of one approximation cell: given abar' (ga) and bbar' (gb), the adjoints of the
// inputs a (ra) and b (rb); they depend on the cell only through e.
// unit_scale for a tape row of output derivatives: all 2N entries scaled by one power of two to
// magnitude ~1 (largest entry), the shift folded into their exponent.
template <typename T, int N>
__device__ __forceinline__ void unit_scale_dm(T (&da)[N], T (&db)[N], int& ef) {
    if constexpr (std::is_same<T, float>::value) {
        float m = 0.f;
#pragma unroll
        for (int n = 0; n < N; ++n) m = fmaxf(m, fmaxf(fabsf(da[n]), fabsf(db[n])));
        if (m > 0x1p16f || (m < 0x1p-16f && m > 0.f)) {
            int sh = 0;
            frexpf(m, &sh);
            const float f = pow2c<float>(-sh);
#pragma unroll
            for (int n = 0; n < N; ++n) { da[n] *= f; db[n] *= f; }
            ef += sh;
        }
    }
}

template <typename T, int N>
__device__ __forceinline__ void cell_adjoint_edges(const T (&e)[N + 1], const T (&ga)[N + 1], const T (&gb)[N + 1],
                                                   T (&ra)[N + 1], T (&rb)[N + 1]) {
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the a- and b-side adjoints run the same products on different data, so they go as
        // packed pairs through the two-wide FP32 instructions.
        // e_0 = 1: the n = 0 weights and the n = k Toeplitz terms need no product, so every sum
        // starts from its n = k term.
        float2 w[N + 1];  // (gb_n e_n, ga_n e_n): weights of the Hankel couplings
        w[0] = make_float2(gb[0], ga[0]);
#pragma unroll
        for (int n = 1; n <= N; ++n) w[n] = __fmul2_rn(make_float2(gb[n], ga[n]), dup2(e[n]));
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            float2 v = make_float2(ga[k], gb[k]);  // (ra_k, rb_k), from the n = k Toeplitz term
            if (k >= 1) {
#pragma unroll
                for (int n = 0; n <= N; ++n) v = __ffma2_rn(w[n], dup2(Tab<float>::hank(n, k)), v);
            }
#pragma unroll
            for (int n = k + 1; n <= N; ++n) v = __ffma2_rn(make_float2(ga[n], gb[n]), dup2(e[n - k]), v);
            ra[k] = v.x;
            rb[k] = v.y;
        }
        return;
    }
    T al[N + 1], be[N + 1];
    al[0] = ga[0];
    be[0] = gb[0];
#pragma unroll
    for (int n = 1; n <= N; ++n) { al[n] = ga[n] * e[n]; be[n] = gb[n] * e[n]; }
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        T va = ga[k], vb = gb[k];  // the n = k Toeplitz term (e_0 = 1)
        if (k >= 1) {
#pragma unroll
            for (int n = 0; n <= N; ++n) {
                va = fma(be[n], Tab<T>::hank(n, k), va);
                vb = fma(al[n], Tab<T>::hank(n, k), vb);
            }
        }
#pragma unroll
        for (int n = k + 1; n <= N; ++n) {
            va = fma(ga[n], e[n - k], va);
            vb = fma(gb[n], e[n - k], vb);
        }
        ra[k] = va;
        rb[k] = vb;
    }
}

// Adjoint of one approximation cell from its inputs (checkpointing adjoint, which replays them).
template <typename T, int N>
__device__ __forceinline__ void cell_adjoint(const T (&a)[N + 1], const T (&b)[N + 1], const T (&e)[N + 1],
                                             const T (&ga)[N + 1], const T (&gb)[N + 1], T (&ra)[N + 1],
                                             T (&rb)[N + 1], T& mbar) {
    cell_adjoint_edges<T, N>(e, ga, gb, ra, rb);
    if constexpr (std::is_same<T, float>::value) {
        // the dk/dM sum over n split into its a- and b-side halves (packed), added once per m
        float mb = 0.f;
#pragma unroll
        for (int m = 1; m <= N; ++m) {
            float2 h = __fmul2_rn(make_float2(b[1], a[1]), dup2(Tab<float>::hank(m, 1)));  // (ha, hb)
#pragma unroll
            for (int k = 2; k <= N; ++k) h = __ffma2_rn(make_float2(b[k], a[k]), dup2(Tab<float>::hank(m, k)), h);
            float2 eb = __fmul2_rn(make_float2(ga[m], gb[m]), h);
#pragma unroll
            for (int n = m; n <= N; ++n)
                eb = __ffma2_rn(make_float2(ga[n], gb[n]), make_float2(a[n - m], b[n - m]), eb);
            mb = fma(eb.x + eb.y, e[m - 1], mb);
        }
        mbar = mb;
        return;
    }
    T mb = T(0);
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        T ha = b[1] * Tab<T>::hank(m, 1);
        T hb = a[1] * Tab<T>::hank(m, 1);
#pragma unroll
        for (int k = 2; k <= N; ++k) {
            ha = fma(b[k], Tab<T>::hank(m, k), ha);
            hb = fma(a[k], Tab<T>::hank(m, k), hb);
        }
        T eb = fma(ga[m], ha, gb[m] * hb);
#pragma unroll
        for (int n = m; n <= N; ++n) {
            eb = fma(ga[n], a[n - m], eb);
            eb = fma(gb[n], b[n - m], eb);
        }
        mb = fma(eb, e[m - 1], mb);
    }
    mbar = mb;
}

// Adjoint of one approximation cell from the tape of output derivatives (cell_series_dm):
// dk/dM = sum_{n>=1} abar'_n d a'_n/dM + bbar'_n d b'_n/dM, 2N multiply-adds.
template <typename T, int N>
__device__ __forceinline__ void cell_adjoint_dm(const T (&da)[N], const T (&db)[N], const T (&e)[N + 1],
                                                const T (&ga)[N + 1], const T (&gb)[N + 1], T (&ra)[N + 1],
                                                T (&rb)[N + 1], T& mbar) {
    cell_adjoint_edges<T, N>(e, ga, gb, ra, rb);
    if constexpr (std::is_same<T, float>::value) {
        float2 acc = __fmul2_rn(make_float2(ga[1], gb[1]), make_float2(da[0], db[0]));
#pragma unroll
        for (int n = 2; n <= N; ++n) acc = __ffma2_rn(make_float2(ga[n], gb[n]), make_float2(da[n - 1], db[n - 1]), acc);
        mbar = acc.x + acc.y;
        return;
    }
    T mb = ga[1] * da[0];
    mb = fma(gb[1], db[0], mb);
#pragma unroll
    for (int n = 2; n <= N; ++n) {
        mb = fma(ga[n], da[n - 1], mb);
        mb = fma(gb[n], db[n - 1], mb);
    }
    mbar = mb;
}

// Adjoint of one interpolation cell.  The forward (cell_series<INTERP>, then project) computes,
// for n = 0..NE,
//   ct_n = e_n ha_n + sum_{k <= min(n, N)} a_k  e_{n-k},   ha_n = sum_{k=1..N} b_k n!/(n+k)!
//   cr_n = e_n hb_n + sum_{k <= min(n, N)} b'_k e_{n-k},   hb_n = sum_{k=1..N} a_k n!/(n+k)!
// with b'_0 = a_0 (the printed corner term of eq. (interpformula)) and b'_k = b_k, and then
// a' = P ct, b' = P cr.  Given the adjoints gt = ct_bar and gr = cr_bar (after the transpose of
// P), it returns a_bar (ra), b_bar (rb; b_0 does not enter) and M_bar = sum_m e_bar_m e_{m-1}.
template <typename T, int N, int NE>
__device__ __forceinline__ void cell_adjoint_interp(const T (&a)[N + 1], const T (&b)[N + 1], const T (&e)[NE + 1],
                                                    const T (&gt)[NE + 1], const T (&gr)[NE + 1], T (&ra)[N + 1],
                                                    T (&rb)[N + 1], T& mbar) {
    if constexpr (std::is_same<T, float>::value) {
        // FP32: a- and b-sides as packed pairs through the two-wide FP32 instructions, as in
        // cell_adjoint; the corner term and the dk/dM halves are summed once.
        float2 w[NE + 1];  // (gr_n e_n, gt_n e_n)
        float corner = 0.f;
#pragma unroll
        for (int n = 0; n <= NE; ++n) {
            w[n] = __fmul2_rn(make_float2(gr[n], gt[n]), dup2(e[n]));
            corner += w[n].x;  // a_0 as the right edge's b'_0
        }
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            float2 v = make_float2(k == 0 ? corner : 0.f, 0.f);  // (ra_k, rb_k)
            if (k >= 1) {
#pragma unroll
                for (int n = 0; n <= NE; ++n) v = __ffma2_rn(w[n], dup2(Tab<float>::hank(n, k)), v);
            }
#pragma unroll
            for (int n = k; n <= NE; ++n)
                v = __ffma2_rn(make_float2(gt[n], k >= 1 ? gr[n] : 0.f), dup2(e[n - k]), v);
            ra[k] = v.x;
            rb[k] = v.y;
        }
        float mb = 0.f;
#pragma unroll
        for (int m = 1; m <= NE; ++m) {
            float2 h = __fmul2_rn(make_float2(b[1], a[1]), dup2(Tab<float>::hank(m, 1)));  // (ha, hb)
#pragma unroll
            for (int k = 2; k <= N; ++k) h = __ffma2_rn(make_float2(b[k], a[k]), dup2(Tab<float>::hank(m, k)), h);
            float2 eb = __fmul2_rn(make_float2(gt[m], gr[m]), h);
#pragma unroll
            for (int k = 0; k <= N && m + k <= NE; ++k)
                eb = __ffma2_rn(make_float2(gt[m + k], gr[m + k]), make_float2(a[k], k == 0 ? a[0] : b[k]), eb);
            mb = fma(eb.x + eb.y, e[m - 1], mb);
        }
        mbar = mb;
        return;
    }
    T al[NE + 1], be[NE + 1];  // gr_n e_n (weights of hb and of the corner), gt_n e_n (of ha)
#pragma unroll
    for (int n = 0; n <= NE; ++n) { al[n] = gr[n] * e[n]; be[n] = gt[n] * e[n]; }
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        T va = T(0), vb = T(0);
        if (k >= 1) {
#pragma unroll
            for (int n = 0; n <= NE; ++n) {
                va = fma(al[n], Tab<T>::hank(n, k), va);
                vb = fma(be[n], Tab<T>::hank(n, k), vb);
            }
        } else {
#pragma unroll
            for (int n = 0; n <= NE; ++n) va += al[n];  // a_0 as the right edge's b'_0
        }
#pragma unroll
        for (int n = k; n <= NE; ++n) {
            va = fma(gt[n], e[n - k], va);
            if (k >= 1) vb = fma(gr[n], e[n - k], vb);
        }
        ra[k] = va;
        rb[k] = vb;
    }
    T mb = T(0);
#pragma unroll
    for (int m = 1; m <= NE; ++m) {
        T ha = b[1] * Tab<T>::hank(m, 1);
        T hb = a[1] * Tab<T>::hank(m, 1);
#pragma unroll
        for (int k = 2; k <= N; ++k) {
            ha = fma(b[k], Tab<T>::hank(m, k), ha);
            hb = fma(a[k], Tab<T>::hank(m, k), hb);
        }
        T eb = fma(gt[m], ha, gr[m] * hb);
#pragma unroll
        for (int k = 0; k <= N && m + k <= NE; ++k) {
            eb = fma(gt[m + k], a[k], eb);
            eb = fma(gr[m + k], k == 0 ? a[0] : b[k], eb);
        }
        mb = fma(eb, e[m - 1], mb);
    }
    mbar = mb;
}

// Transpose of the interpolation projection: c_bar_n = g_n (n <= N), c_bar_j = sum_n g_n P[n][j]
// (j > N), for the adjoint g of a projected edge.
template <typename T, int N, int NE>
__device__ __forceinline__ void project_transpose(const T (&g)[N + 1], T (&c)[NE + 1]) {
#pragma unroll
    for (int n = 0; n <= N; ++n) c[n] = g[n];
#pragma unroll
    for (int j = N + 1; j <= NE; ++j) {
        T v = T(0);
#pragma unroll
        for (int n = 0; n <= N; ++n) v = fma(g[n], Tab<T>::proj(N, n, j - N - 1), v);
        c[j] = v;
    }
}

// Shared memory of one warp: a ring of K steps of the strip tape (each lane copies its own row
// of a step ahead of the reverse walk), then each lane's dk/dx accumulator of its row
// ([32][dpad + 1]; the odd stride puts the lanes' scalar accesses in distinct banks).
template <typename T, int N, int K>
__host__ __device__ constexpr int bwd_stack_bytes() {
    return K * fwd_tape_step_bytes<T, N, false>();
}
template <typename T>
__host__ __device__ constexpr int bwd_xacc_bytes(int dpad) { return 32 * (dpad + 1) * static_cast<int>(sizeof(T)); }

template <typename T, int N, int K, int DMAX>
constexpr int bwd_min_blocks() {
    return sizeof(T) == 8 ? 1 : (DMAX <= 8 ? 5 : 3);
}

template <typename T, int N, int K, int DMAX>
__global__ void __launch_bounds__(kFwdWarps * 32, (bwd_min_blocks<T, N, K, DMAX>()))
    bwd_approx_kernel(BwdParams B) {
    constexpr bool kRescale = std::is_same<T, float>::value;
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const Launch& L = B.L;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t slot = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wib;
    char* base = static_cast<char*>(L.scratch) + slot * L.scratch_stride;
    // the strip tape: per step of the current strip, the 32 lanes' rows of output derivatives,
    // exponent and M (the layout of the forward tape, store_dm_row)
    char* stape = base;
    constexpr int kStep = fwd_tape_step_bytes<T, N, false>();
    constexpr int TR = tape_row<T>(N, false);
    T* fbuf = reinterpret_cast<T*>(base + B.off_fbuf);          // [strip][col][N+1]
    int* fexp = reinterpret_cast<int*>(base + B.off_fexp);      // [strip][col]
    T* rbuf = reinterpret_cast<T*>(base + B.off_rbuf);          // [col][N+1]
    int* rexp = reinterpret_cast<int*>(base + B.off_rexp);      // [col]
    T* ybar = reinterpret_cast<T*>(base + B.off_ybar);          // [coarse col][dpad]
    const int dpad = L.dpad;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* wsm = smem_raw + wib * (bwd_stack_bytes<T, N, K>() + bwd_xacc_bytes<T>(dpad));
    unsigned char* ring = wsm;  // K slots of kStep bytes: step t of the strip in slot t % K
    T* xacc = reinterpret_cast<T*>(wsm + bwd_stack_bytes<T, N, K>()) + lane * (dpad + 1);
    const T* __restrict__ incX = static_cast<const T*>(L.X.inc);
    const T* __restrict__ incY = static_cast<const T*>(L.Y.inc);

    for (;;) {
        const int64_t item = next_item(L);
        if (item < 0) break;
        const PairDesc P = decode_pair(L, item);
        if (P.lx < 0 || P.ly < 0) {
            if (lane == 0) record_error(SK_ERR_BAD_LENGTH);
            continue;
        }
        if (P.lx == 0 || P.ly == 0) continue;  // k = 1 does not depend on the paths
        double gbar;
        if (L.mode == kPairsList) gbar = B.gout[item];
        else if (L.mode == kGramFull) gbar = B.gout[P.a * L.ldo + P.b];
        else gbar = B.gout[P.a * L.ldo + P.b] + (P.a != P.b ? B.gout[P.b * L.ldo + P.a] : 0.0);
        if (gbar == 0.0) continue;

        const int lam = L.lam;
        const int rows = static_cast<int>(P.lx << lam);
        const int cols = static_cast<int>(P.ly << lam);
        const int period = cols > 32 ? cols : 32;
        const int nstrips = (rows + 31) >> 5;
        const int last_lane = (rows - 1) - ((nstrips - 1) << 5);
        const int nsteps = (nstrips - 1) * period + last_lane + cols;
        const T sub = pow2t<T>(-2 * lam);
        const T* xbase = incX + P.xs * dpad;
        const T* ybase = incY + P.ys * dpad;

        // ------------------------------------------------------------------ F
        int ek = 0;
        {
            T a[N + 1], bo[N + 1];
#pragma unroll
            for (int n = 0; n <= N; ++n) { a[n] = T(0); bo[n] = T(0); }
            int ea = 0, eo = 0;
            int jj = -lane, s = 0;
            for (int step = 0; step < nsteps; ++step) {
                T b[N + 1];
#pragma unroll
                for (int n = 0; n <= N; ++n) b[n] = __shfl_up_sync(kFull, bo[n], 1);
                int eb = kRescale ? __shfl_up_sync(kFull, eo, 1) : 0;
                const int row = (s << 5) + lane;
                const bool active = jj >= 0 && jj < cols && row < rows;
                if (active) {
                    if (lane == 0) {
                        if (s == 0) {
                            set_unit<T, N>(b);
                            eb = 0;
                        } else {
                            const T* src = fbuf + (static_cast<int64_t>(s - 1) * B.cols_max + jj) * (N + 1);
#pragma unroll
                            for (int n = 0; n <= N; ++n) b[n] = src[n];
                            if (kRescale) eb = fexp[static_cast<int64_t>(s - 1) * B.cols_max + jj];
                        }
                    }
                    if (jj == 0) {
                        set_unit<T, N>(a);
                        ea = 0;
                    }
                    if (kRescale) align_inputs<T, N>(a, ea, b, eb);
                    const T M = row_dot<T>(xbase + static_cast<int64_t>(row >> lam) * dpad,
                                           ybase + static_cast<int64_t>(jj >> lam) * dpad, L.nvec) * sub;
                    fwd_cell<T, N>(a, b, M, L.tau, bo, ea);
                    if (row == rows - 1 && jj == cols - 1) {
                        double v = 0.5 * (series_at_one<T, N>(a) + series_at_one<T, N>(bo));
                        int e2 = 0;
                        if (v != 0.0) frexp(v, &e2);
                        ek = ea + e2;
                    }
                    eo = ea;
                    if (lane == 31 && s + 1 < nstrips) {
                        T* dst = fbuf + (static_cast<int64_t>(s) * B.cols_max + jj) * (N + 1);
#pragma unroll
                        for (int n = 0; n <= N; ++n) dst[n] = bo[n];
                        if (kRescale) fexp[static_cast<int64_t>(s) * B.cols_max + jj] = eo;
                    }
                }
                __syncwarp();
                if (++jj == period) { jj = 0; ++s; }
            }
        }
        ek = __shfl_sync(kFull, ek, last_lane);
        const double gscale = gbar * pow2d(ek);

        // adjoint state of the lane
        T gra[N + 1], gbo[N + 1];
        int gea = kZeroExp, gbe = kZeroExp;
        T ysum[DMAX];
#pragma unroll
        for (int n = 0; n <= N; ++n) { gra[n] = T(0); gbo[n] = T(0); }
#pragma unroll
        for (int c = 0; c < DMAX; ++c) ysum[c] = T(0);
        for (int c = 0; c < dpad; ++c) xacc[c] = T(0);
        // dk/dy of the pair's columns, summed over its strips in T (lane 0 adds each strip's
        // column sum as the adjoint leaves the column) and added to the gradient once at the end
        for (int q = lane; q < P.ly * dpad; q += 32) ybar[q] = T(0);
        __syncwarp();

        for (int s = nstrips - 1; s >= 0; --s) {
            const int row = (s << 5) + lane;
            const int ts = (s == nstrips - 1 ? last_lane : 31) + cols;  // steps of this strip
            const T* xrow = xbase + static_cast<int64_t>(min(row, rows - 1) >> lam) * dpad;
            // -------------------------------------------------------------- R1
            // the strip's forward from its hand-off column, each active cell's row of output
            // derivatives, exponent and M to the strip tape
            {
                T a[N + 1], bo[N + 1];
#pragma unroll
                for (int n = 0; n <= N; ++n) { a[n] = T(0); bo[n] = T(0); }
                int ea = 0, eo = 0;
                for (int tt = 0; tt < ts; ++tt) {
                    T b[N + 1];
#pragma unroll
                    for (int n = 0; n <= N; ++n) b[n] = __shfl_up_sync(kFull, bo[n], 1);
                    int eb = kRescale ? __shfl_up_sync(kFull, eo, 1) : 0;
                    const int jj = tt - lane;
                    const bool active = jj >= 0 && jj < cols && row < rows;
                    if (active) {
                        if (lane == 0) {
                            if (s == 0) {
                                set_unit<T, N>(b);
                                eb = 0;
                            } else {
                                const T* src = fbuf + (static_cast<int64_t>(s - 1) * B.cols_max + jj) * (N + 1);
#pragma unroll
                                for (int n = 0; n <= N; ++n) b[n] = src[n];
                                if (kRescale) eb = fexp[static_cast<int64_t>(s - 1) * B.cols_max + jj];
                            }
                        }
                        if (jj == 0) {
                            set_unit<T, N>(a);
                            ea = 0;
                        }
                        if (kRescale) align_inputs<T, N>(a, ea, b, eb);
                        const T M = row_dot<T>(xrow, ybase + static_cast<int64_t>(jj >> lam) * dpad, L.nvec) * sub;
                        T e[N + 1], ct[N + 1], cr[N + 1], da[N], db[N];
                        build_exp_series<T, N>(M, L.tau, e);
                        cell_series_dm<T, N>(a, b, e, ct, cr, da, db);  // ct, cr: fwd_cell's outputs
                        store_dm_row<T, N>(stape, tt, lane, da, db, ea, M);
#pragma unroll
                        for (int n = 0; n <= N; ++n) { a[n] = ct[n]; bo[n] = cr[n]; }
                        rescale_edges<T, N>(a, bo, ea);
                        eo = ea;
                    }
                }
            }
            __syncwarp();
            __threadfence_block();  // each lane's stores of its rows before its copies of them
            // -------------------------------------------------------------- R2
            // the strip's steps backward; each lane copies its own row of step t into ring slot
            // t % K, K steps ahead of its use (one commit group per step, empty past step 0)
            auto fetch = [&](int t) {
                if (t >= 0) {
                    const char* src = stape + static_cast<int64_t>(t) * kStep;
                    unsigned char* dst = ring + (t % K) * kStep;
#pragma unroll
                    for (int v = 0; v < TR / W; ++v) cp_async16(dst + (v * 32 + lane) * 16, src + (v * 32 + lane) * 16);
                    if constexpr (TR % W != 0)
                        cp_async8(dst + (TR / W) * 512 + lane * 8, src + (TR / W) * 512 + lane * 8);
                }
                cp_async_commit();
            };
#pragma unroll
            for (int k = 0; k < K; ++k) fetch(ts - 1 - k);
#pragma unroll 1
            for (int tt = ts - 1; tt >= 0; --tt) {
                cp_async_wait<K - 1>();  // step tt's group has landed
                T da[N], db[N], M = T(0);
                int ef = 0;
                {
                    const unsigned char* r = ring + (tt % K) * kStep;
                    auto put = [&](int q, T x) {
                        if (q < N) da[q] = x;
                        else if (q < 2 * N) db[q - N] = x;
                        else if (q == 2 * N) ef = exponent_from<T>(x);
                        else M = x;
                    };
#pragma unroll
                    for (int v = 0; v < TR / W; ++v) {
                        const V t = reinterpret_cast<const V*>(r)[v * 32 + lane];
                        const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
                        for (int w = 0; w < W; ++w) put(v * W + w, tp[w]);
                    }
                    if constexpr (TR % W != 0) {
                        const float2 t = reinterpret_cast<const float2*>(r + (TR / W) * 512)[lane];
                        put((TR / W) * W, t.x);
                        put((TR / W) * W + 1, t.y);
                    }
                }
                const int jj = tt - lane;
                const bool active = jj >= 0 && jj < cols && row < rows;
                T gb_in[N + 1];
#pragma unroll
                for (int n = 0; n <= N; ++n) gb_in[n] = __shfl_down_sync(kFull, gbo[n], 1);
                int gbe_in = __shfl_down_sync(kFull, gbe, 1);
#pragma unroll
                for (int c = 0; c < DMAX; ++c) ysum[c] = __shfl_down_sync(kFull, ysum[c], 1);
                if (active) {
                    if (row == rows - 1) {             // no row above: the top edge is final
#pragma unroll
                        for (int n = 0; n <= N; ++n) gb_in[n] = T(0);
                        gbe_in = kZeroExp;
                    } else if (lane == 31) {           // from lane 0 of the strip above
                        const T* src = rbuf + static_cast<int64_t>(jj) * (N + 1);
#pragma unroll
                        for (int n = 0; n <= N; ++n) gb_in[n] = src[n];
                        gbe_in = kRescale ? rexp[jj] : 0;
                    }
                    if (row == rows - 1 || lane == 31) {
#pragma unroll
                        for (int c = 0; c < DMAX; ++c) ysum[c] = T(0);
                    }
                    T ga_in[N + 1];
                    int gae_in = gea;
#pragma unroll
                    for (int n = 0; n <= N; ++n) ga_in[n] = gra[n];
                    if (jj == cols - 1) {              // right edge of the grid
#pragma unroll
                        for (int n = 0; n <= N; ++n) ga_in[n] = T(0);
                        gae_in = kZeroExp;
                    }
                    if (row == rows - 1 && jj == cols - 1) {  // seed from the endpoint average
#pragma unroll
                        for (int n = 0; n <= N; ++n) {
                            ga_in[n] = static_cast<T>(0.5 * cx_rfact(n));
                            gb_in[n] = ga_in[n];
                        }
                        gae_in = 0;
                        gbe_in = 0;
                    }
                    int eg = 0;
                    if (kRescale) {
                        eg = max(gae_in, gbe_in);
                        if (gae_in != eg) {
                            const T f = pow2c<T>(gae_in - eg);
#pragma unroll
                            for (int n = 0; n <= N; ++n) ga_in[n] *= f;
                        }
                        if (gbe_in != eg) {
                            const T f = pow2c<T>(gbe_in - eg);
#pragma unroll
                            for (int n = 0; n <= N; ++n) gb_in[n] *= f;
                        }
                    }
                    unit_scale_dm<T, N>(da, db, ef);
                    T e[N + 1];
                    build_exp_series<T, N>(M, L.tau, e);
                    T mbar;
                    cell_adjoint_dm<T, N>(da, db, e, ga_in, gb_in, gra, gbo, mbar);
                    // dk/dM of the coarse cell, relative to 2^ek
                    const T mrel = mbar * pow2c<T>(eg + ef - ek - 2 * lam);
                    {
                        const V* yv = reinterpret_cast<const V*>(ybase + static_cast<int64_t>(jj >> lam) * dpad);
                        const V* xv = reinterpret_cast<const V*>(xrow);
#pragma unroll
                        for (int c4 = 0; c4 < DMAX / W; ++c4) {
                            if (c4 * W < dpad) {
                                const V yy = __ldg(yv + c4);
                                const V xx = __ldg(xv + c4);
                                const T* yp = reinterpret_cast<const T*>(&yy);
                                const T* xp = reinterpret_cast<const T*>(&xx);
#pragma unroll
                                for (int w = 0; w < W; ++w) {
                                    xacc[c4 * W + w] = fma(mrel, yp[w], xacc[c4 * W + w]);
                                    ysum[c4 * W + w] = fma(mrel, xp[w], ysum[c4 * W + w]);
                                }
                            }
                        }
                    }
                    gea = eg;
                    if (kRescale) {
                        float mag = 0.f;
#pragma unroll
                        for (int n = 0; n <= N; ++n)
                            mag = fmaxf(mag, fmaxf(fabsf(static_cast<float>(gra[n])), fabsf(static_cast<float>(gbo[n]))));
                        if (mag == 0.f) {
                            gea = kZeroExp;
                        } else if (mag > 0x1p64f || mag < 0x1p-64f) {
                            const int sh = mag > 0x1p64f ? -64 : 64;
#pragma unroll
                            for (int n = 0; n <= N; ++n) { gra[n] *= pow2t<T>(sh); gbo[n] *= pow2t<T>(sh); }
                            gea -= sh;
                        }
                    }
                    gbe = gea;
                    if (lane == 0) {
                        if (s > 0) {  // hand the left-edge adjoint to lane 31 of the strip below
                            T* dst = rbuf + static_cast<int64_t>(jj) * (N + 1);
#pragma unroll
                            for (int n = 0; n <= N; ++n) dst[n] = gbo[n];
                            if (kRescale) rexp[jj] = gbe;
                        }
                        // the column's partial dk/dy over this strip is complete
                        T* yb = ybar + static_cast<int64_t>(jj >> lam) * dpad;
#pragma unroll
                        for (int c = 0; c < DMAX; ++c)
                            if (c < dpad) yb[c] += ysum[c];
                    }
                    if (jj == 0) {  // the row is finished: flush dk/dx of its increment
                        double* gx = B.gincX + (P.xs + (row >> lam)) * dpad;
                        for (int c = 0; c < dpad; ++c) {
                            if (xacc[c] != T(0)) atomicAdd(gx + c, static_cast<double>(xacc[c]) * gscale);
                            xacc[c] = T(0);
                        }
                    }
                }
                fetch(tt - K);  // into the slot this step's row came from
                __syncwarp();
            }
        }
        __syncwarp();  // lane 0's column sums are visible to the warp
        {
            double* gy = B.gincY + P.ys * dpad;
            for (int q = lane; q < P.ly * dpad; q += 32)
                if (ybar[q] != T(0)) atomicAdd(gy + q, static_cast<double>(ybar[q]) * gscale);
        }
        __syncwarp();
    }
}


// ---------------------------------------------------------------------------------------------
// Adjoint from a forward tape.  The forward kernel recorded, for every warp step, the 32 lanes'
// cell inputs (a, b, exponent, M; laid out [vector][lane]) and the exponent of k_hat; this kernel
// walks the same steps backward (the reverse of the forward schedule, strips overlapping exactly
// as there) and needs neither forward recomputation nor the increments.  The steps stream into a
// ring of kTapeRing shared-memory slots per warp with bulk copies issued kTapeRing steps ahead by
// lane 0, each slot completing on its own mbarrier.  Each cell's dk/dM (relative to 2^ek, with
// the 4^-lambda of the sub-cell M folded in) is written to a per-item buffer of 32-element rows,
// one per step, lane r's value at position (r + step) mod 32 (zero where a lane is idle); the
// skew lets bwd_contract_kernel read both rows and columns of a cell tile without bank
// conflicts.  That kernel turns the buffer into dk/dx and dk/dy.
// ---------------------------------------------------------------------------------------------
// Four slots measured fastest on the 128x128 Gram of 257-point paths: 15.6 ms, against 16.3 ms
// with three and 19.1 ms with eight.  Per-lane streaming loads of the tape one step ahead (no
// ring, no shared memory) took 18.9 ms.
constexpr int kTapeRing = 4;

template <typename T, int N, bool INTERP>
__host__ __device__ constexpr int bwd_tape_min_blocks() {
    return sizeof(T) == 8 ? (INTERP ? 1 : 2) : (INTERP ? 3 : 4);
}

// Series terms of a cell's adjoint: N + 1, or N + 1 + J for the interpolation scheme.
template <typename T, int N, bool INTERP>
__host__ __device__ constexpr int bwd_series_top() {
    return INTERP ? N + (sizeof(T) == 8 ? kJF64 : kJF32) : N;
}

// Shared memory of one warp for the tape adjoint: the ring and its mbarriers.
// Each warp's region is padded to 128 bytes, so that every warp's ring (a bulk-copy destination,
// which must be 16-byte aligned) starts aligned whatever the slot count.
__host__ __device__ constexpr int bwd_tape_warp_bytes(int step_bytes) {
    return (kTapeRing * step_bytes + kTapeRing * 8 + 127) / 128 * 128;
}
template <typename T, int N, bool INTERP>
__host__ __device__ constexpr int bwd_tape_warp_bytes() {
    return bwd_tape_warp_bytes(fwd_tape_step_bytes<T, N, INTERP>());
}

// Gradient seed and exponent of k_hat for item `item` (shared by the adjoint and the contraction).
__device__ __forceinline__ double item_gbar(const BwdParams& B, int64_t item, const PairDesc& P) {
    const Launch& L = B.L;
    if (L.mode == kPairsList) return B.gout[item];
    if (L.mode == kGramFull) return B.gout[P.a * L.ldo + P.b];
    return B.gout[P.a * L.ldo + P.b] + (P.a != P.b ? B.gout[P.b * L.ldo + P.a] : 0.0);
}

template <typename T, int N, bool INTERP>
__global__ void __launch_bounds__(kFwdWarps * 32, (bwd_tape_min_blocks<T, N, INTERP>()))
    bwd_tape_kernel(BwdParams B) {
    constexpr int NE = bwd_series_top<T, N, INTERP>();
    constexpr bool kRescale = std::is_same<T, float>::value;
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int TR = tape_row<T>(N, INTERP);
    const Launch& L = B.L;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t slot = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wib;
    char* base = static_cast<char*>(L.scratch) + slot * L.scratch_stride;
    T* rbuf = reinterpret_cast<T*>(base + B.off_rbuf);          // [col][N+1]
    int* rexp = reinterpret_cast<int*>(base + B.off_rexp);      // [col]
    constexpr int kStepBytes = fwd_tape_step_bytes<T, N, INTERP>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* ring = smem_raw + wib * bwd_tape_warp_bytes<T, N, INTERP>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kTapeRing * kStepBytes);
    if (lane == 0) {
        for (int k = 0; k < kTapeRing; ++k) mbar_init(bars + k, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;  // bit k: phase of slot k's barrier awaited next (warp-uniform)
    bool stuck = false;

    for (;;) {
        const int64_t item = stuck ? -1 : next_item(L);
        if (item < 0) break;
        const PairDesc P = decode_pair(L, item);
        if (P.lx < 0 || P.ly < 0) {
            if (lane == 0) record_error(SK_ERR_BAD_LENGTH);
            continue;
        }
        if (P.lx == 0 || P.ly == 0) continue;
        if (item_gbar(B, item, P) == 0.0) continue;  // bwd_contract_kernel skips it too

        const int lam = L.lam;
        const int rows = static_cast<int>(P.lx << lam);
        const int cols = static_cast<int>(P.ly << lam);
        const int period = cols > 32 ? cols : 32;
        const int nstrips = (rows + 31) >> 5;
        const int last_lane = (rows - 1) - ((nstrips - 1) << 5);
        const int nsteps = (nstrips - 1) * period + last_lane + cols;
        const int ek = L.tape_ek[item];
        const char* tape = static_cast<const char*>(L.tape) + item * L.tape_stride;
        T* mout = reinterpret_cast<T*>(static_cast<char*>(B.mbuf) + item * B.mb_stride);
        if constexpr (std::is_same<T, float>::value) {
            if (B.gtile) gtile_zero_padding(mout, rows, cols, B.gt_ncb);  // cells outside the grid hold zero
        }

        // Edge conditions of the reverse sweep.  A lane's right-edge input (no cell to the right)
        // is zero: gra starts at zero and is cleared whenever the lane moves down a strip.  The top
        // row's upper input is zero: it comes from a lane beyond the last row, never active in
        // this item, whose gbo stays zero (lane 31 is handled where it reads the hand-off).  The
        // corner cell (rows-1, cols-1), run by lane last_lane at the first reverse step, is
        // seeded from the endpoint average: for the approximation scheme both output edges get
        // 1/(2 n!); for the interpolation scheme the unprojected series do (n = 0..N+J).
        T gra[N + 1], gbo[N + 1];
        int gea = kZeroExp, gbe = kZeroExp;
#pragma unroll
        for (int n = 0; n <= N; ++n) {
            gra[n] = (!INTERP && lane == last_lane) ? static_cast<T>(0.5 * cx_rfact(n)) : T(0);
            gbo[n] = T(0);
        }
        if (!INTERP && lane == last_lane) gea = 0;

        // fill the ring with the last kTapeRing steps (step t lives in slot t % kTapeRing); the
        // slots were read by the previous item's steps
        if (lane == 0) {
            fence_proxy_async_smem();
            for (int k = 0; k < kTapeRing && nsteps - 1 - k >= 0; ++k) {
                const int t = nsteps - 1 - k;
                const int sl = t % kTapeRing;
                mbar_arrive_expect_tx(bars + sl, kStepBytes);
                bulk_load(ring + sl * kStepBytes, tape + static_cast<int64_t>(t) * kStepBytes, kStepBytes, bars + sl);
            }
        }
        // position of this lane at the last step, then walked backward one step at a time
        int tt = nsteps - 1 - lane;
        int s = tt >= 0 ? tt / period : -1;
        int jj = tt >= 0 ? tt - s * period : -1;
        int stuck_step = -1;
        for (int step = nsteps - 1; step >= 0; --step) {
            const int sl = step % kTapeRing;
            if (!mbar_wait(bars + sl, (parity >> sl) & 1u)) {
                stuck = true;  // the device error word is set; drain what is in flight and stop
                stuck_step = step;
                break;
            }
            parity ^= 1u << sl;
            // The lane's tape row.  Interpolation: the cell inputs fa = a, fb = b.  Approximation:
            // fa[0..N-1] = d a'_{n+1}/dM and fb[0..N-1] = d b'_{n+1}/dM (its whole 16-byte vectors
            // [vector][lane], then an 8-byte remainder [lane] for FP32 with N even).
            T fa[N + 1], fb[N + 1];
            int ef;
            T M;
            {
                const V* src = reinterpret_cast<const V*>(ring + sl * kStepBytes);
                auto put = [&](int q, T x) {
                    if constexpr (INTERP) {
                        if (q <= N) fa[q] = x;
                        else if (q <= 2 * N + 1) fb[q - N - 1] = x;
                        else if (q == 2 * N + 2) ef = exponent_from<T>(x);
                        else if (q == 2 * N + 3) M = x;
                    } else {
                        if (q < N) fa[q] = x;
                        else if (q < 2 * N) fb[q - N] = x;
                        else if (q == 2 * N) ef = exponent_from<T>(x);
                        else M = x;
                    }
                };
#pragma unroll
                for (int v = 0; v < TR / W; ++v) {
                    const V t = src[v * 32 + lane];
                    const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
                    for (int w = 0; w < W; ++w) put(v * W + w, tp[w]);
                }
                if constexpr (TR % W != 0) {
                    const float2 t = reinterpret_cast<const float2*>(ring + sl * kStepBytes + (TR / W) * 32 * 16)[lane];
                    put((TR / W) * W, t.x);
                    put((TR / W) * W + 1, t.y);
                }
            }
            __syncwarp();  // every lane has its row: the slot can be refilled
            if (lane == 0 && step - kTapeRing >= 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bars + sl, kStepBytes);
                bulk_load(ring + sl * kStepBytes, tape + static_cast<int64_t>(step - kTapeRing) * kStepBytes,
                          kStepBytes, bars + sl);
            }
            T gb_in[N + 1];
#pragma unroll
            for (int n = 0; n <= N; ++n) gb_in[n] = __shfl_down_sync(kFull, gbo[n], 1);
            int gbe_in = __shfl_down_sync(kFull, gbe, 1);
            const int row = (s << 5) + lane;
            const bool active = s >= 0 && jj < cols && row < rows;
            T mrel = T(0);
            if (active) {
                if (lane == 31) {                  // from lane 0 of the strip above, if any
                    if (row == rows - 1) {
#pragma unroll
                        for (int n = 0; n <= N; ++n) gb_in[n] = T(0);
                        gbe_in = kZeroExp;
                    } else {
                        const T* src = rbuf + static_cast<int64_t>(jj) * (N + 1);
#pragma unroll
                        for (int n = 0; n <= N; ++n) gb_in[n] = src[n];
                        gbe_in = kRescale ? rexp[jj] : 0;
                    }
                }
                if (!INTERP && step == nsteps - 1) {  // warp-uniform: the corner cell's upper input
#pragma unroll
                    for (int n = 0; n <= N; ++n) gb_in[n] = static_cast<T>(0.5 * cx_rfact(n));
                    gbe_in = 0;
                }
                int eg = 0;
                if (kRescale) {
                    eg = max(gea, gbe_in);
                    if (gea != eg) {
                        const T f = pow2c<T>(gea - eg);
#pragma unroll
                        for (int n = 0; n <= N; ++n) gra[n] *= f;
                    }
                    if (gbe_in != eg) {
                        const T f = pow2c<T>(gbe_in - eg);
#pragma unroll
                        for (int n = 0; n <= N; ++n) gb_in[n] *= f;
                    }
                }
                T da[N], db[N];  // approximation: the row's derivatives (fa, fb hold them in 0..N-1)
#pragma unroll
                for (int n = 0; n < N; ++n) { da[n] = fa[n]; db[n] = fb[n]; }
                if constexpr (INTERP) unit_scale<T, N>(fa, fb, ef);
                else unit_scale_dm<T, N>(da, db, ef);
                T e[NE + 1];
                build_exp_series<T, NE>(M, L.tau, e);
                T mbar;
                T ga_in[N + 1];
#pragma unroll
                for (int n = 0; n <= N; ++n) ga_in[n] = gra[n];
                if constexpr (INTERP) {
                    T gt[NE + 1], gr[NE + 1];
                    project_transpose<T, N, NE>(ga_in, gt);
                    project_transpose<T, N, NE>(gb_in, gr);
                    if (step == nsteps - 1) {  // warp-uniform: the corner's endpoint seed
#pragma unroll
                        for (int n = 0; n <= NE; ++n) {
                            gt[n] = static_cast<T>(0.5 * cx_rfact(n));
                            gr[n] = gt[n];
                        }
                        eg = 0;
                    }
                    cell_adjoint_interp<T, N, NE>(fa, fb, e, gt, gr, gra, gbo, mbar);
                } else {
                    cell_adjoint_dm<T, N>(da, db, e, ga_in, gb_in, gra, gbo, mbar);
                }
                mrel = mbar * pow2c<T>(eg + ef - ek - 2 * lam);
                gea = eg;
                if (kRescale && (step & 3) == 0) {  // keep the adjoints within [2^-64, 2^64]
                    float mag = 0.f;
#pragma unroll
                    for (int n = 0; n <= N; ++n)
                        mag = fmaxf(mag, fmaxf(fabsf(static_cast<float>(gra[n])), fabsf(static_cast<float>(gbo[n]))));
                    if (mag > 0x1p64f || (mag < 0x1p-64f && mag > 0.f)) {
                        const int sh = mag > 0x1p64f ? -64 : 64;
#pragma unroll
                        for (int n = 0; n <= N; ++n) { gra[n] *= pow2t<T>(sh); gbo[n] *= pow2t<T>(sh); }
                        gea -= sh;
                    }
                }
                gbe = gea;
                if (lane == 0 && s > 0) {  // hand the left-edge adjoint to lane 31 of the strip below
                    T* dst = rbuf + static_cast<int64_t>(jj) * (N + 1);
#pragma unroll
                    for (int n = 0; n <= N; ++n) dst[n] = gbo[n];
                    if (kRescale) rexp[jj] = gbe;
                }
            }
            bool tiled = false;
            if constexpr (std::is_same<T, float>::value) {
                if (B.gtile) {  // BF16 hi/lo tiles for the tensor-core contraction
                    tiled = true;
                    if (active) {
                        __nv_bfloat16 h, l;
                        split_bf16(mrel, h, l);
                        __nv_bfloat16* gt = reinterpret_cast<__nv_bfloat16*>(mout);
                        const int64_t q = gtile_index(row, jj, B.gt_ncb);
                        gt[q] = h;
                        gt[q + kGtilePlane] = l;
                    }
                }
            }
            if (!tiled) mout[static_cast<int64_t>(step) * 32 + ((lane + step) & 31)] = mrel;  // skewed row
            __syncwarp();
            if (s >= 0 && --jj < 0) {  // down one strip: the next row starts at the right edge
                jj = period - 1;
                --s;
#pragma unroll
                for (int n = 0; n <= N; ++n) gra[n] = T(0);
                gea = kZeroExp;
            }
        }
        if (stuck) {
            // Wait (bounded) for the copies still in flight into this warp's ring (steps stuck_step
            // down to stuck_step - kTapeRing + 1) before leaving.
            if (lane == 0)
                for (int k = 0; k < kTapeRing && stuck_step - k >= 0; ++k) {
                    const int sl = (stuck_step - k) % kTapeRing;
                    mbar_wait(bars + sl, (parity >> sl) & 1u);
                }
            __syncwarp();
            break;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// Chain rule through M_ij = <dx_i, dy_j> / 4^lambda (M_ij is the increments' inner product that
// drives the Goursat PDE of the kernel of piecewise linear paths):
//   dk/d(dx_i) = sum_j dk/dM_ij dy_j,   dk/d(dy_j) = sum_i dk/dM_ij dx_i,
// from the dk/dM buffer written by bwd_tape_kernel.  One block per work item (grid-stride), one
// warp per strip of 32 rows.  A strip is cut into tiles of 32 columns; cell (r, j0 + q) of tile
// j0 sits at step sP + j0 + r + q, so a tile spans 63 consecutive 32-element rows of the buffer.
// The warp streams halves of 32 rows (4 KB in FP32) into a circular ring of three halves (96 rows)
// with cp.async.bulk, one half ahead.  Per tile it stages the 32 dy rows in shared memory next to
// the strip's 32 dx rows (C coordinates each), and with the buffer's skew (lane r of step t at
// (r + t) mod 32):
//   * dk/dx: lane r walks its row (q = 0..31) against the dy rows;
//   * dk/dy: lane q walks its column (r = 0..31) against the broadcast dx rows;
// both conflict-free in FP32, every operand in shared memory, each cell's dk/dM read once for all
// C coordinates, and the products as two-wide FP32 instructions.  Row sums stay in registers
// across a strip's tiles and go to the FP64 gradients once per strip (strips own disjoint rows).
// Column sums are added to a shared per-column accumulator once per tile; the columns are taken a
// window at a time (as many as the accumulator holds), and the accumulator goes to the FP64
// gradients once per window, scaled by gbar 2^ek.  Coordinates beyond C are taken C at a time.
// ---------------------------------------------------------------------------------------------
constexpr int kContractWarps = 4;
constexpr int kContractSlack = 64;  // buffer rows past an item's last step that a tile may read
constexpr int kContractAccBytes = 32 << 10;  // per-block column accumulator

// Shared memory of one contraction warp, padded to 128 bytes so that every warp's ring (a bulk
// copy destination) starts 128-byte aligned.
template <typename T, int C>
__host__ __device__ constexpr int contract_warp_bytes() {
    return (3 * 32 * 32 * static_cast<int>(sizeof(T))    // ring of three halves
            + 2 * 32 * C * static_cast<int>(sizeof(T))   // dx of the strip's rows, dy of the tile's columns
            + 3 * 8                                      // mbarriers
            + 127) / 128 * 128;
}

// Columns of a window: the accumulator holds [C][window] elements.
template <typename T, int C>
__host__ __device__ constexpr int contract_window() {
    return kContractAccBytes / (C * static_cast<int>(sizeof(T))) / 32 * 32;
}

// C accumulators, acc += m v with v read from shared memory as 16-byte vectors (FP32: two-wide
// FMAs on coordinate pairs).
template <typename T, int C> struct ContractAcc;
template <int C> struct ContractAcc<float, C> {
    float2 s[C / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < C / 2; ++k) s[k] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void axpy(float m, const float* v) {
        const float2 m2 = make_float2(m, m);
        const float4* vv = reinterpret_cast<const float4*>(v);
#pragma unroll
        for (int k = 0; k < C / 4; ++k) {
            const float4 y = vv[k];
            s[2 * k] = __ffma2_rn(m2, make_float2(y.x, y.y), s[2 * k]);
            s[2 * k + 1] = __ffma2_rn(m2, make_float2(y.z, y.w), s[2 * k + 1]);
        }
    }
    __device__ __forceinline__ float get(int c) const { return (c & 1) ? s[c >> 1].y : s[c >> 1].x; }
};
template <int C> struct ContractAcc<double, C> {
    double s[C];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int c = 0; c < C; ++c) s[c] = 0.0;
    }
    __device__ __forceinline__ void axpy(double m, const double* v) {
        const double2* vv = reinterpret_cast<const double2*>(v);
#pragma unroll
        for (int k = 0; k < C / 2; ++k) {
            const double2 y = vv[k];
            s[2 * k] = fma(m, y.x, s[2 * k]);
            s[2 * k + 1] = fma(m, y.y, s[2 * k + 1]);
        }
    }
    __device__ __forceinline__ double get(int c) const { return s[c]; }
};

// One tile: cell (r, j0 + q) is at ring row hb + r + q (mod 96), position (2r + q + coff) mod 32
// with coff = (t0 + j0) mod 32.  nr, nc: valid rows and columns (FULL: 32 and 32; otherwise
// cells outside them, whose buffer entries may hold anything, count as zero).
template <typename T, int C, bool FULL, bool WRAP>
__device__ __forceinline__ void contract_tile(const T* __restrict__ ring, int hb, int coff, const T* __restrict__ xs,
                                              const T* __restrict__ ys, int nr, int nc, int lane, ContractAcc<T, C>& xa,
                                              ContractAcc<T, C>& ya) {
    // dk/dx: row `lane`.  The upper half-warp runs one column ahead (cyclically) so that the two
    // halves read banks of opposite parity.
#pragma unroll 8
    for (int q0 = 0; q0 < 32; ++q0) {
        const int q = (q0 + (lane >> 4)) & 31;
        const int u = lane + q;
        int row = hb + u;
        if (WRAP) row -= row >= 96 ? 96 : 0;
        T m = ring[(row << 5) + ((lane + u + coff) & 31)];
        if (!FULL) m = (lane < nr && q < nc) ? m : T(0);
        xa.axpy(m, ys + q * C);
    }
    // dk/dy: column `lane`, against the broadcast dx rows
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int u = r + lane;
        int row = hb + u;
        if (WRAP) row -= row >= 96 ? 96 : 0;
        T m = ring[(row << 5) + ((r + u + coff) & 31)];
        if (!FULL) m = (r < nr && lane < nc) ? m : T(0);
        ya.axpy(m, xs + r * C);
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(kContractWarps * 32) bwd_contract_kernel(BwdParams B) {
    constexpr int HB = 32 * 32 * static_cast<int>(sizeof(T));  // bytes of one half
    constexpr int WIN = contract_window<T, C>();
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const Launch& L = B.L;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int dpad = L.dpad;
    const int lam = L.lam;
    const T* __restrict__ incX = static_cast<const T*>(L.X.inc);
    const T* __restrict__ incY = static_cast<const T*>(L.Y.inc);
    extern __shared__ __align__(16) unsigned char csm[];
    unsigned char* wsm = csm + wib * contract_warp_bytes<T, C>();
    T* ring = reinterpret_cast<T*>(wsm);                                   // [96 rows][32], circular
    T* xs = reinterpret_cast<T*>(wsm + 3 * HB);                            // [32][C]
    T* ys = xs + 32 * C;                                                   // [32][C]
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + 3 * HB + 2 * 32 * C * sizeof(T));
    T* acc = reinterpret_cast<T*>(csm + kContractWarps * contract_warp_bytes<T, C>());  // [C][WIN]
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) mbar_init(bars + k, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;   // bit k: phase of slot k's barrier awaited next (warp-uniform)
    uint32_t pending = 0;  // bit k: a copy into slot k was issued and not yet awaited
    bool stuck = false;

    // Every warp visits every item and window of its block (a stuck warp skips its strips) so
    // that the block-wide barriers below are reached by all warps.
    for (int64_t item = blockIdx.x; item < L.npairs; item += gridDim.x) {
        const PairDesc P = decode_pair(L, item);
        if (P.lx <= 0 || P.ly <= 0) continue;
        const double gbar = item_gbar(B, item, P);
        if (gbar == 0.0) continue;
        const double gscale = gbar * pow2d(L.tape_ek[item]);
        const int rows = static_cast<int>(P.lx << lam);
        const int cols = static_cast<int>(P.ly << lam);
        const int period = cols > 32 ? cols : 32;
        const int nstrips = (rows + 31) >> 5;
        // Waits on slot k for the copy issued last into it; false when the wait ran out.
        auto await_slot = [&](int k) -> bool {
            if (!mbar_wait(bars + k, (parity >> k) & 1u)) return false;
            parity ^= 1u << k;
            pending &= ~(1u << k);
            return true;
        };
        const char* mb = static_cast<const char*>(B.mbuf) + item * B.mb_stride;
        const T* xbase = incX + P.xs * dpad;
        const T* ybase = incY + P.ys * dpad;
        double* gx = B.gincX + P.xs * dpad;
        double* gy = B.gincY + P.ys * dpad;
        for (int c0 = 0; c0 < dpad; c0 += C) {
            for (int w0 = 0; w0 < cols; w0 += WIN) {  // a window of columns [w0, w0 + WIN)
                const int wcols = min(WIN, cols - w0);
                const int ntiles = (wcols + 31) >> 5;
                // coarse columns the window touches: (w0 >> lam) .. ((w0 + wcols - 1) >> lam)
                const int ya0 = w0 >> lam;
                const int nya = ((w0 + wcols - 1) >> lam) - ya0 + 1;
                for (int q = threadIdx.x; q < C * nya; q += blockDim.x) acc[q] = T(0);
                __syncthreads();
                for (int s = wib; s < nstrips && !stuck; s += kContractWarps) {
                    const int t0 = s * period + w0;  // buffer row of the window's first tile
                    const int nr = min(32, rows - (s << 5));  // valid rows of the strip
                    // half h of the window = buffer rows t0 + 32h .. t0 + 32h + 31, in slot h % 3
                    if (lane == 0) fence_proxy_async_smem();  // the previous strip read these slots
                    for (int h = 0; h < 3 && h <= ntiles; ++h) {
                        if (lane == 0) {
                            mbar_arrive_expect_tx(bars + h, HB);
                            bulk_load(ring + h * 1024, mb + static_cast<int64_t>(t0 + 32 * h) * 32 * sizeof(T), HB,
                                      bars + h);
                        }
                        pending |= 1u << h;
                    }
                    __syncwarp();  // the previous strip's readers of xs are done
                    {
                        const int xi = min((s << 5) + lane, rows - 1) >> lam;
                        const V* xr = reinterpret_cast<const V*>(xbase + static_cast<int64_t>(xi) * dpad + c0);
                        V* xd = reinterpret_cast<V*>(xs + lane * C);
#pragma unroll
                        for (int k = 0; k < C / W; ++k) {
                            V v = {};
                            if (lane < nr && c0 + k * W < dpad) v = __ldg(xr + k);
                            xd[k] = v;
                        }
                    }
                    ContractAcc<T, C> xa;
                    xa.zero();
                    for (int b = 0; b < ntiles; ++b) {
                        // half b (slot b % 3) was awaited as the upper half of tile b - 1, except for b = 0
                        const int s0 = b % 3, s1 = (b + 1) % 3;
                        if (b == 0 && !await_slot(s0)) { stuck = true; break; }
                        if (!await_slot(s1)) { stuck = true; break; }
                        const int j0 = w0 + (b << 5);
                        const int nc = min(32, cols - j0);  // valid columns of the tile
                        __syncwarp();  // the previous tile's readers of ys are done
                        {
                            const int yi = min(j0 + lane, cols - 1) >> lam;
                            const V* yr = reinterpret_cast<const V*>(ybase + static_cast<int64_t>(yi) * dpad + c0);
                            V* yd = reinterpret_cast<V*>(ys + lane * C);
#pragma unroll
                            for (int k = 0; k < C / W; ++k) {
                                V v = {};
                                if (lane < nc && c0 + k * W < dpad) v = __ldg(yr + k);
                                yd[k] = v;
                            }
                        }
                        __syncwarp();
                        ContractAcc<T, C> ya;
                        ya.zero();
                        const int coff = (s * period + j0) & 31;
                        // slots 0-1 and 1-2 are contiguous in the ring; only slots 2-0 wrap
                        if (nr == 32 && nc == 32) {
                            if (s0 == 2) contract_tile<T, C, true, true>(ring, s0 * 32, coff, xs, ys, nr, nc, lane, xa, ya);
                            else contract_tile<T, C, true, false>(ring, s0 * 32, coff, xs, ys, nr, nc, lane, xa, ya);
                        } else {
                            contract_tile<T, C, false, true>(ring, s0 * 32, coff, xs, ys, nr, nc, lane, xa, ya);
                        }
                        if (lane < nc) {
                            const int yi = ((j0 + lane) >> lam) - ya0;
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                const T v = ya.get(c);
                                if (c0 + c < dpad && v != T(0)) atomicAdd(acc + c * nya + yi, v);
                            }
                        }
                        __syncwarp();  // slot s0 is read by every lane: refill it with half b + 3
                        if (b + 3 <= ntiles) {
                            if (lane == 0) {
                                fence_proxy_async_smem();
                                mbar_arrive_expect_tx(bars + s0, HB);
                                bulk_load(ring + s0 * 1024, mb + static_cast<int64_t>(t0 + 32 * (b + 3)) * 32 * sizeof(T),
                                          HB, bars + s0);
                            }
                            pending |= 1u << s0;
                        }
                    }
                    if (lane < nr) {  // this strip's rows are its own: straight to the gradients
                        const int xi = ((s << 5) + lane) >> lam;
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            const T v = xa.get(c);
                            if (c0 + c < dpad && v != T(0))
                                atomicAdd(gx + static_cast<int64_t>(xi) * dpad + c0 + c, static_cast<double>(v) * gscale);
                        }
                    }
                }
                __syncthreads();
                for (int q = threadIdx.x; q < C * nya; q += blockDim.x) {
                    const int c = q / nya, r = q - c * nya;
                    if (c0 + c >= dpad || acc[q] == T(0)) continue;
                    atomicAdd(gy + static_cast<int64_t>(ya0 + r) * dpad + c0 + c, static_cast<double>(acc[q]) * gscale);
                }
                __syncthreads();
            }
        }
    }
    if (stuck) {  // the device error word is set; wait (bounded) for this warp's copies in flight
        for (int k = 0; k < 3; ++k)
            if (pending & (1u << k)) mbar_wait(bars + k, (parity >> k) & 1u);
    }
}

}  // namespace sk
