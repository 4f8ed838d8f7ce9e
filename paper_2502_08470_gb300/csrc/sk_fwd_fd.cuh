// Forward wavefront of the finite-difference schemes on the dyadic grid P_lambda (Definition
// "dyadic scheme", Section 2; second-order explicit update eq. (secondexplicitscheme); implicit
// update of Remark "higherfd") for sm_103a.
//
// On a sub-cell of P_lambda with m = <dx_I, dy_J> = M_ij / 4^lambda (the refined increments are
// the coarse ones divided by 2^lambda), all three updates read
//     k(I+1, J+1) = (k(I+1, J) + k(I, J+1)) alpha - k(I, J) beta
// with alpha = 1 + m/2, beta = 1 (ORDER 1, first order); alpha = 1 + m/2 + m^2/12,
// beta = 1 - m^2/12 (ORDER 2, second order); alpha = (1 + m/4) / (1 - m/4), beta = 1 (ORDER 3,
// implicit: the four-corner trapezoid equation k11 = k10 + k01 - k00 + (m/4)(k00 + k10 + k01 +
// k11) solved for k11, which leaves the k00 terms cancelling to beta = 1).  All 4^lambda sub-cells
// of a cell share (alpha, beta).
//
// Difference form.  Writing v(I+1, J) = k(I+1, J) - k(I, J), the same update is
//     v(I+1, J+1) = v(I+1, J) + (alpha - 1)(k(I+1, J) + k(I, J+1)) - (beta - 1) k(I, J),
//     k(I+1, J+1) = k(I, J+1) + v(I+1, J+1).
// A lane carries v for its rows along the sweep and rebuilds k upward from the node below, so
// rounding in the long sweep direction is relative to |v| (small) rather than to |k|; in the
// direct form every node's O(eps |k|) rounding reaches the whole quadrant above and to its right.
//
// Parallel layout.  One warp owns one pair (or, for long pairs, a block of warps shares it with
// one strip per warp in a pipeline, as in the polynomial wavefront).  Lane r owns R = min(2^lambda, 16) consecutive node
// rows (a "row group"; all in one coarse row) and sweeps the refined columns; the top node of
// its group moves one lane up per step by __shfl_up_sync, and lane 31's top nodes are handed to
// lane 0 of the next strip through a per-warp buffer, as in the polynomial wavefront.  FP32 keeps
// a power-of-two exponent per lane (rescale by 2^-64 / 2^64 outside [2^-64, 2^64]).
#pragma once

#include <type_traits>

#include "sk_common.cuh"
#include "sk_fwd_poly.cuh"  // trivial_pair

namespace sk {

// One lane's row of the FD forward tape: its R node differences v (before the column's update),
// k0 = k(gR, J), k1 = k(gR, J+1), the sub-cell m and the exponent, padded to 16 bytes.  From it the
// adjoint rebuilds the lane's R sub-cells of column J (fd_tape_row elements per lane and step,
// laid out [vector][lane] like the polynomial tapes).
template <typename T>
__host__ __device__ constexpr int fd_tape_row(int R) {
    return ((R + 4) * static_cast<int>(sizeof(T)) + 15) / 16 * 16 / static_cast<int>(sizeof(T));
}

template <typename T>
__device__ __forceinline__ T fd_pow2(int e) {
    if constexpr (std::is_same<T, float>::value) return pow2f(e);
    else return pow2d(e);
}

// Sweep of one pair by one warp (CW = 1) or by warp w of a cooperative block of CW warps
// (strips w, w + CW, ...; hand-off ordering as in sweep_poly).
template <typename T, int ORDER, int R, int CW, bool TAPE = false>
__device__ __forceinline__ void sweep_fd(const Launch& L, int64_t item, const PairDesc& P, int w, char* own_buf,
                                         const char* prev_buf, int* prog, int64_t buf_cols) {
    constexpr bool kRescale = std::is_same<T, float>::value;
    const int lane = threadIdx.x & 31;
    T* hbuf = reinterpret_cast<T*>(own_buf);                          // [buf_cols]
    int* ebuf = reinterpret_cast<int*>(hbuf + buf_cols);              // [buf_cols]
    const T* hprev = reinterpret_cast<const T*>(prev_buf);
    const int* eprev = reinterpret_cast<const int*>(hprev + buf_cols);
    const int dpad = L.dpad;
    const T* __restrict__ incX = static_cast<const T*>(L.X.inc);
    const T* __restrict__ incY = static_cast<const T*>(L.Y.inc);

    const int lam = L.lam;
    const int nI = static_cast<int>(P.lx << lam);   // refined node rows 0..nI
    const int nJ = static_cast<int>(P.ly << lam);   // refined node columns 0..nJ
    const int groups = nI / R;
    // Period of a warp's strips.  Alone, a warp starts its next strip as soon as lane 0 is free
    // (P = max(cols, 32)).  In a cooperative block that overlap can deadlock: a warp whose lane 0
    // waits on the ring of other warps also holds back its lanes still publishing the previous
    // strip, which those warps need.  A warp therefore starts strip k + 1 only after finishing
    // strip k (P = cols + 31), unless the rows are longer than the ring's lag (cols > 31 CW),
    // where the overlapped schedule keeps every wait pointed at finished work.  A model of this
    // schedule (tests/test_pipeline_schedule.py) checks the rule and the deadlock it avoids.
    const int period = CW == 1 ? (nJ > 32 ? nJ : 32) : (nJ > 31 * CW ? nJ : nJ + 31);
    const int nstrips = (groups + 31) >> 5;
    const int last_lane = (groups - 1) - ((nstrips - 1) << 5);
    const int nloc = w < nstrips ? (nstrips - 1 - w) / CW + 1 : 0;
    if (nloc == 0) return;
    const bool has_last = (nstrips - 1) % CW == w;
    const int nsteps = (nloc - 1) * period + (has_last ? last_lane : 31) + nJ;
    const T sub = fd_pow2<T>(-2 * lam);
    const T* xbase = incX + P.xs * dpad;
    const T* ybase = incY + P.ys * dpad;

    T v[R];     // k(gR + 1 + r, jj) - k(gR + r, jj) for the lane's group g at its column jj
    T kb_prev = T(1), top = T(0);
    int ea = 0, eo = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = T(0);
    int jj = -lane, sl = 0, gs = w;     // column, local strip, global strip
    bool stuck = false;

    for (int step = 0; step < nsteps; ++step) {
        T kb = __shfl_up_sync(kFull, top, 1);            // k(gR, jj + 1) from the lane below
        int eb = kRescale ? __shfl_up_sync(kFull, eo, 1) : 0;
        const int g = (gs << 5) + lane;
        const bool active = jj >= 0 && jj < nJ && g < groups && sl < nloc;
        if (active) {
            if (lane == 0) {
                if (gs == 0) {
                    kb = T(1);                               // row 0: k(s_0, .) = 1
                    eb = 0;
                } else {
                    if constexpr (CW > 1) {
                        if (!stuck && !wait_progress(prog + (w + CW - 1) % CW, (gs - 1) * nJ + jj + 1, wait_polls(L)))
                            stuck = true;
                    }
                    kb = hprev[jj];
                    if (kRescale) eb = eprev[jj];
                }
            }
            if (jj == 0) {                               // column 0: k(., t_0) = 1, so v = 0
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = T(0);
                kb_prev = T(1);
                ea = 0;
            }
            if (kRescale && ea != eb) {
                if (ea > eb) {
                    kb *= (eb - ea < -126) ? T(0) : fd_pow2<T>(eb - ea);
                } else {
                    const T f = (ea - eb < -126) ? T(0) : fd_pow2<T>(ea - eb);
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] *= f;
                    kb_prev *= f;
                    ea = eb;
                }
            }
            const T m = row_dot<T>(xbase + static_cast<int64_t>((g * R) >> lam) * dpad,
                                   ybase + static_cast<int64_t>(jj >> lam) * dpad, L.nvec) * sub;
            if constexpr (TAPE) {  // the column's inputs for the adjoint (fd_tape_row)
                using V = typename Vec<T>::type;
                constexpr int W = Vec<T>::W;
                constexpr int TR = fd_tape_row<T>(R);
                V* dst = reinterpret_cast<V*>(static_cast<char*>(L.tape) + item * L.tape_stride +
                                              static_cast<int64_t>(step) * (32 * TR * static_cast<int>(sizeof(T))));
#pragma unroll
                for (int vv = 0; vv < TR / W; ++vv) {
                    V t;
                    T* tp = reinterpret_cast<T*>(&t);
#pragma unroll
                    for (int q2 = 0; q2 < W; ++q2) {
                        const int q = vv * W + q2;
                        tp[q2] = q < R ? v[q < R ? q : 0] : (q == R ? kb_prev : (q == R + 1 ? kb : (q == R + 2 ? m : T(0))));
                        if (q == R + 3) tp[q2] = exponent_as<T>(kRescale ? ea : 0);
                    }
                    __stcs(dst + vv * 32 + lane, t);
                }
            }
            T a1 = m * T(0.5);                           // alpha - 1
            if constexpr (ORDER == 3) a1 = a1 / (T(1) - m * T(0.25));
            T m2 = T(0);                                 // (1 - beta) = alpha - 1 - m/2 (ORDER 2)
            if constexpr (ORDER == 2) m2 = m * m * T(1.0 / 12.0);
            T k00 = kb_prev, k01 = kb;                   // k(I, J), k(I, J+1) for I = gR + r
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T k10 = k00 + v[r];                // k(I+1, J)
                const T sum = k10 + k01;
                T d2 = a1 * sum;
                if constexpr (ORDER == 2) d2 = fma(m2, sum + k00, d2);
                v[r] += d2;
                const T k11 = k01 + v[r];                // k(I+1, J+1)
                k00 = k10;
                k01 = k11;
            }
            kb_prev = kb;
            top = k01;
            if (g == groups - 1 && jj == nJ - 1) {
                double res = static_cast<double>(top);
                if (kRescale) res = ldexp(res, ea);
                if (!isfinite(res)) record_error(SK_ERR_NONFINITE);
                write_result(L, item, P, res);
                if (TAPE && L.tape_ek != nullptr) {  // exponent of k_hat for the adjoint's scaling
                    int e2 = 0;
                    const double t0 = static_cast<double>(top);
                    if (t0 != 0.0) frexp(t0, &e2);
                    L.tape_ek[item] = (kRescale ? ea : 0) + e2;
                }
            }
            if (kRescale) {
                const float mag = fmaxf(fabsf(static_cast<float>(kb_prev)), fabsf(static_cast<float>(top)));
                if (mag > 0x1p64f || (mag < 0x1p-64f && mag > 0.f)) {
                    const int sh = mag > 0x1p64f ? -64 : 64;
                    const T f = fd_pow2<T>(sh);
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] *= f;
                    kb_prev *= f;
                    top *= f;
                    ea -= sh;
                }
            }
            eo = ea;
            if (lane == 31 && gs + 1 < nstrips) {
                hbuf[jj] = top;
                if (kRescale) ebuf[jj] = eo;
                if constexpr (CW > 1) publish_progress(prog + w, gs * nJ + jj + 1);
            }
        }
        __syncwarp();
        if (++jj == period) {
            jj = 0;
            ++sl;
            gs += CW;
        }
    }
}

// One-warp blocks are compiled for 8 blocks per SM (64 registers, no spills): FD Grams of
// 128 x 128 pairs of 257-point paths ran 2.1x faster than at the 180-200 registers the
// unconstrained build took (2 blocks per SM).  The pipelined blocks keep their budget: capped at
// two blocks per SM they ran slower (64 oscillatory pairs at lambda = 4: 30.1 against 22.1 ms).
// TAPE (CW = 1): also record the forward tape of the FD adjoint (fd_tape_row, L.tape must be set).
template <typename T, int ORDER, int R, int CW, bool TAPE = false>
__global__ void __launch_bounds__((CW > 1 ? CW : kFwdWarps) * 32, (CW > 1 ? 1 : (TAPE ? 4 : 8)))
    fwd_fd_kernel(Launch L, int64_t buf_cols) {
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    char* block_base = static_cast<char*>(L.scratch) + static_cast<int64_t>(blockIdx.x) * nw * L.scratch_stride;
    char* own = block_base + wib * L.scratch_stride;
    if constexpr (CW > 1) {
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
            const int nstrips = P.lx > 0 ? static_cast<int>((((P.lx << L.lam) / R) + 31) >> 5) : 0;
            if (nstrips < L.coop_min_strips) {  // short pairs from here on: one warp each
                if (wib == 0 && !trivial_pair(L, item, P))
                    sweep_fd<T, ORDER, R, 1>(L, item, P, 0, own, own, nullptr, buf_cols);
                break;
            }
            if (!trivial_pair(L, item, P))
                sweep_fd<T, ORDER, R, CW>(L, item, P, wib, own, block_base + ((wib + CW - 1) % CW) * L.scratch_stride,
                                          s_prog, buf_cols);
        }
    }
    for (;;) {
        const int64_t item = next_item(L);
        if (item < 0) break;
        const PairDesc P = decode_pair(L, item);
        if (trivial_pair(L, item, P)) continue;
        sweep_fd<T, ORDER, R, 1, TAPE>(L, item, P, 0, own, own, nullptr, buf_cols);
    }
}

}  // namespace sk
