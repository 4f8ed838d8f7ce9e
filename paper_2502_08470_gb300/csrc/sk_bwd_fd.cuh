// Reverse-mode derivative (adjoint wavefront) of the finite-difference schemes (Definition "dyadic
// scheme", eq. (secondexplicitscheme), Remark "higherfd") from the forward tape of sweep_fd.
// The paper defines no gradient: this is the exact adjoint of the schemes' own arithmetic.
//
// The forward step of a lane (group g of R = 2^lambda node rows, column J) maps its state
// (differences v_r = k(gR+r+1, J) - k(gR+r, J), the bottom node k0 = k(gR, J)) and the input
// k1 = k(gR, J+1) from the lane below to the new differences v'_r and the top node k(gR+R, J+1):
//     k10 = k00 + v_r,  sum = k10 + k01,  d = a1 sum + m2 (sum + k00),  v'_r = v_r + d,
//     k11 = k01 + v'_r,  (k00, k01) <- (k10, k11),      starting from (k0, k1),
// with a1 = alpha - 1 and m2 = 1 - beta (m2 = 0 for first order and the implicit scheme).  The
// adjoint runs the same steps in reverse order (the reverse of the forward schedule, one warp per
// pair): from the adjoints of v' (carried from the lane's next column), of the top node (from the
// lane above, or lane 0 of the strip above through a per-warp buffer, or the endpoint seed 1) and
// of k1 as the next column's k0 (carried), it gives the adjoints of v, k0 and k1 (k1's goes down to
// the lane below) and, per sub-cell, dk/dm = abar1 da1/dm + mbar2 dm2/dm.  A coarse cell's
// 4^lambda sub-cells share m = M_ij / 4^lambda, so dk/dM_ij sums them over 4^-lambda; the lane
// covers the cell's 2^lambda rows in one step and its 2^lambda columns in consecutive steps, and
// writes the sum, relative to 2^ek, into the contraction's dk/dM buffer for the coarse grid (the
// skewed [step][lane] rows of bwd_contract_kernel, or the tiles of the tensor-core contraction).
// FP32 carries power-of-two exponents for the adjoints as the polynomial adjoint does.
//
// The tape rows stream through a per-warp ring in shared memory, kFdRing<R> steps ahead: each
// lane copies its own 16-byte vectors of a step with cp.async (one commit group per step) and
// waits for the oldest group only when it needs that step, so the row loads no longer stall
// every step (measured: the FD1 adjoint at lambda = 0 spent most cycles waiting on its per-step
// loads, issue 30%).  A lane reads only the vectors it copied itself, so cp.async.wait_group
// orders the copy before the read without any warp-wide barrier.
#pragma once

#include <type_traits>

#include "sk_bwd_poly.cuh"
#include "sk_fwd_fd.cuh"

namespace sk {

// Steps of tape rows in flight per warp: deeper for the short rows of few node rows per lane.
template <int R>
__host__ __device__ constexpr int kFdRing() {
    return R <= 1 ? 8 : (R <= 2 ? 6 : 4);
}
// Shared-memory bytes of one warp's ring.
template <typename T, int R>
__host__ __device__ constexpr int fd_ring_warp_bytes() {
    return kFdRing<R>() * 32 * fd_tape_row<T>(R) * static_cast<int>(sizeof(T));
}

template <typename T, int ORDER, int R>
__global__ void __launch_bounds__(kFwdWarps * 32) bwd_fd_tape_kernel(BwdParams B) {
    constexpr bool kRescale = std::is_same<T, float>::value;
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int TR = fd_tape_row<T>(R);
    const Launch& L = B.L;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t slot = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wib;
    char* base = static_cast<char*>(L.scratch) + slot * L.scratch_stride;
    T* rbuf = reinterpret_cast<T*>(base + B.off_rbuf);       // [col]: adjoint of lane 0's k1
    int* rexp = reinterpret_cast<int*>(base + B.off_rexp);   // [col]
    constexpr int D = kFdRing<R>();
    constexpr int kStepBytes = 32 * TR * static_cast<int>(sizeof(T));
    extern __shared__ __align__(16) unsigned char fd_smem[];
    unsigned char* ring = fd_smem + wib * fd_ring_warp_bytes<T, R>();  // [D][vector][lane]

    for (;;) {
        const int64_t item = next_item(L);
        if (item < 0) break;
        const PairDesc P = decode_pair(L, item);
        if (P.lx < 0 || P.ly < 0) {
            if (lane == 0) record_error(SK_ERR_BAD_LENGTH);
            continue;
        }
        if (P.lx == 0 || P.ly == 0) continue;
        if (item_gbar(B, item, P) == 0.0) continue;  // the contraction skips it too

        const int lam = L.lam;
        const int groups = static_cast<int>(P.lx);        // R = 2^lambda rows per lane: one coarse row
        const int nJ = static_cast<int>(P.ly << lam);     // refined columns
        const int period = nJ > 32 ? nJ : 32;
        const int nstrips = (groups + 31) >> 5;
        const int last_lane = (groups - 1) - ((nstrips - 1) << 5);
        const int nsteps = (nstrips - 1) * period + last_lane + nJ;
        const int ek = L.tape_ek[item];
        const char* tape = static_cast<const char*>(L.tape) + item * L.tape_stride;
        // coarse-grid schedule of the dk/dM buffer: cell (32 s + r, j) at row s P' + j + r
        const int cols_c = static_cast<int>(P.ly);
        const int period_c = cols_c > 32 ? cols_c : 32;
        char* mout = static_cast<char*>(B.mbuf) + item * B.mb_stride;
        if constexpr (std::is_same<T, float>::value) {
            if (B.gtile) gtile_zero_padding(mout, groups, cols_c, B.gt_ncb);  // coarse cells outside the grid
        }

        T vbar[R];                  // adjoints of the lane's v at the column after the current one
        T carry = T(0);             // adjoint of k0 of that column (= k1 of the current one)
        int ge = kZeroExp;          // exponent of vbar and carry
        T k1out = T(0);             // adjoint of this lane's k1 at its last active column (to lane - 1)
        int k1e = kZeroExp;
        T mcell = T(0);             // dk/dM of the current coarse cell, relative to 2^ek
#pragma unroll
        for (int r = 0; r < R; ++r) vbar[r] = T(0);

        // this lane's vectors of steps nsteps - 1 .. nsteps - D, one commit group per step (step t
        // in slot t % D; empty groups past step 0 keep the count uniform)
        auto fetch = [&](int t) {
            if (t >= 0) {
                const V* src = reinterpret_cast<const V*>(tape + static_cast<int64_t>(t) * kStepBytes);
                V* dst = reinterpret_cast<V*>(ring + (t % D) * kStepBytes);
#pragma unroll
                for (int vv = 0; vv < TR / W; ++vv) cp_async16(dst + vv * 32 + lane, src + vv * 32 + lane);
            }
            cp_async_commit();
        };
#pragma unroll
        for (int k = 0; k < D; ++k) fetch(nsteps - 1 - k);

        int tt = nsteps - 1 - lane;
        int s = tt >= 0 ? tt / period : -1;
        int jj = tt >= 0 ? tt - s * period : -1;
        for (int step = nsteps - 1; step >= 0; --step) {
            cp_async_wait<D - 1>();  // this step's group has landed (the D - 1 after it may not)
            const V* trow = reinterpret_cast<const V*>(ring + (step % D) * kStepBytes);
            T tb = __shfl_down_sync(kFull, k1out, 1);
            int tbe = __shfl_down_sync(kFull, k1e, 1);
            const int g = (s << 5) + lane;
            const bool active = s >= 0 && jj < nJ && g < groups;
            if (active) {
                if (g == groups - 1) {            // the top group: no lane above in this pair
                    tb = T(0);
                    tbe = kZeroExp;
                    if (jj == nJ - 1) {           // the endpoint k(nI, nJ): seed 1
                        tb = T(1);
                        tbe = 0;
                    }
                } else if (lane == 31) {          // from lane 0 of the strip above
                    tb = rbuf[jj];
                    tbe = kRescale ? rexp[jj] : 0;
                }
                // the tape row of this step
                T v[R], k0, k1, m;
                int ea = 0;
                {
#pragma unroll
                    for (int vv = 0; vv < TR / W; ++vv) {
                        const V t = trow[vv * 32 + lane];
                        const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
                        for (int q2 = 0; q2 < W; ++q2) {
                            const int q = vv * W + q2;
                            if (q < R) v[q < R ? q : 0] = tp[q2];
                            else if (q == R) k0 = tp[q2];
                            else if (q == R + 1) k1 = tp[q2];
                            else if (q == R + 2) m = tp[q2];
                            else if (q == R + 3) ea = exponent_from<T>(tp[q2]);
                        }
                    }
                }
                if (jj == nJ - 1) {  // the lane's first reverse column of this strip: nothing carried
#pragma unroll
                    for (int r = 0; r < R; ++r) vbar[r] = T(0);
                    carry = T(0);
                    ge = kZeroExp;
                }
                // bring the carried adjoints and the one from above to a common exponent
                int eg = 0;
                if (kRescale) {
                    eg = max(ge, tbe);
                    if (ge != eg) {
                        const T f = pow2c<T>(ge - eg);
#pragma unroll
                        for (int r = 0; r < R; ++r) vbar[r] *= f;
                        carry *= f;
                    }
                    if (tbe != eg) tb *= pow2c<T>(tbe - eg);
                }
                // forward recompute of the column (as sweep_fd runs it)
                T a1 = m * T(0.5);
                if constexpr (ORDER == 3) a1 = a1 / (T(1) - m * T(0.25));
                T m2 = T(0);
                if constexpr (ORDER == 2) m2 = m * m * T(1.0 / 12.0);
                T k00s[R], sums[R];
                {
                    T k00 = k0, k01 = k1;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const T k10 = k00 + v[r];
                        const T sum = k10 + k01;
                        T d2 = a1 * sum;
                        if constexpr (ORDER == 2) d2 = fma(m2, sum + k00, d2);
                        const T k11 = k01 + (v[r] + d2);
                        k00s[r] = k00;
                        sums[r] = sum;
                        k00 = k10;
                        k01 = k11;
                    }
                }
                // reverse of the column
                T k01b = tb, k00b = T(0), a1b = T(0), m2b = T(0);
#pragma unroll
                for (int r = R - 1; r >= 0; --r) {
                    const T k11b = k01b, k10b0 = k00b;
                    const T vpb = vbar[r] + k11b;         // v'_r: carried and through k11 = k01 + v'_r
                    T k01r = k11b;
                    T vb = vpb;                           // through v'_r = v_r + d
                    const T db = vpb;
                    T sumb = a1 * db;
                    T k00r = T(0);
                    a1b = fma(sums[r], db, a1b);
                    if constexpr (ORDER == 2) {
                        sumb = fma(m2, db, sumb);
                        k00r = m2 * db;
                        m2b = fma(sums[r] + k00s[r], db, m2b);
                    }
                    const T k10b = k10b0 + sumb;          // sum = k10 + k01
                    k01r += sumb;
                    k00r += k10b;                          // k10 = k00 + v_r
                    vb += k10b;
                    vbar[r] = vb;
                    k01b = k01r;
                    k00b = k00r;
                }
                // dk/dm of the column's R sub-cells: a1' and m2' of the scheme
                T mb;
                if constexpr (ORDER == 3) {
                    const T den = T(1) - m * T(0.25);
                    mb = a1b * (T(0.5) / (den * den));
                } else {
                    mb = a1b * T(0.5);
                    if constexpr (ORDER == 2) mb = fma(m2b, m * T(1.0 / 6.0), mb);
                }
                mcell = fma(mb, pow2c<T>(eg + ea - ek - 2 * lam), mcell);
                // k1 of this column: through this column's sub-cells and as the next column's k0
                const T k1b = k01b + carry;
                carry = k00b;
                ge = eg;
                k1out = k1b;
                k1e = eg;
                if (kRescale && (step & 3) == 0) {  // keep the adjoints within [2^-64, 2^64]
                    T mag = fabs(carry);
#pragma unroll
                    for (int r = 0; r < R; ++r) mag = fmax(mag, fabs(vbar[r]));
                    const float fm = static_cast<float>(mag);
                    if (fm > 0x1p64f || (fm < 0x1p-64f && fm > 0.f)) {
                        const int sh = fm > 0x1p64f ? -64 : 64;
#pragma unroll
                        for (int r = 0; r < R; ++r) vbar[r] *= pow2t<T>(sh);
                        carry *= pow2t<T>(sh);
                        ge -= sh;
                    }
                }
                if (lane == 0 && s > 0) {  // hand k1's adjoint to lane 31 of the strip below
                    rbuf[jj] = k1out;
                    if (kRescale) rexp[jj] = k1e;
                }
                if ((jj & ((1 << lam) - 1)) == 0) {  // the coarse cell's first column: its sum is complete
                    const int j = jj >> lam;
                    bool tiled = false;
                    if constexpr (std::is_same<T, float>::value) {
                        if (B.gtile) {
                            tiled = true;
                            __nv_bfloat16 h, l;
                            split_bf16(mcell, h, l);
                            __nv_bfloat16* gt = reinterpret_cast<__nv_bfloat16*>(mout);
                            const int64_t q = gtile_index(g, j, B.gt_ncb);
                            gt[q] = h;
                            gt[q + kGtilePlane] = l;
                        }
                    }
                    if (!tiled) {
                        const int64_t row = static_cast<int64_t>(s) * period_c + j + lane;
                        reinterpret_cast<T*>(mout)[row * 32 + ((lane + row) & 31)] = mcell;
                    }
                    mcell = T(0);
                }
            }
            fetch(step - D);  // into the slot this step's row came from
            __syncwarp();
            if (s >= 0 && --jj < 0) {  // down one strip
                jj = period - 1;
                --s;
            }
        }
        __syncwarp();
    }
}

}  // namespace sk
