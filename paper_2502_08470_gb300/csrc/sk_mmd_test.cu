// Two-sample permutation test on MMD^2 from a pooled Gram matrix (the paper names statistical
// hypothesis testing among the library's uses, Sections 1 and 4; the test is the standard one).
//
// K is the (na + nb) x (na + nb) Gram matrix of the pooled sample Z = (A, B), row-major FP64.  A
// relabelling marks na of the pooled paths as the first sample; with l_j = 1 for a marked path,
//     r_i = sum_j K_ij l_j,   t_i = sum_j K_ij,
//     S_11 = sum_{i: l_i = 1} r_i,   S_10 = sum_{i: l_i = 1} (t_i - r_i),   S_00 = sum_{i: l_i = 0} (t_i - r_i),
// and MMD^2 = S_11 / na^2 + S_00 / nb^2 - 2 S_10 / (na nb) (biased), or with the diagonals
// sum_{l_i = 1} K_ii, sum_{l_i = 0} K_ii taken out of S_11, S_00 and means over na (na - 1),
// nb (nb - 1) (unbiased).  Every statistic is one pass over K with masked FP64 additions: the
// labels enter as bit masks, so there is no multiplication, and K (2 MB for 512 pooled paths)
// stays in L2 across the blocks.
//
// Layout.  pack_labels_kernel turns the caller's uint8 rows into bit rows (one 32-bit word per 32
// pooled paths), with row 0 the given split (paths < na) and row q >= 1 the caller's row q - 1,
// and counts each row's marks.  mmd_perm_stats_kernel gives a block kPermPerBlock relabellings:
// each warp walks its rows of K once, lane j reading K_ij coalesced, and adds K_ij into the
// relabellings whose bit j is set (the mask word is a broadcast load), so every K row read serves
// kPermPerBlock statistics.  All sums run in a fixed order (lane-strided, xor-butterfly, rows of a
// warp in order, warps in order), so a statistic depends only on K and its own relabelling.
#include <algorithm>
#include <cstdint>

#include "sigkernel.h"
#include "sk_common.cuh"
#include "sk_dispatch.h"

namespace sk {

namespace {

constexpr int kPermPerBlock = 8;  // relabellings per block
constexpr int kPermWarps = 8;     // warps per block of the statistics kernel

// One warp per 32-path word of one relabelling row: bits[q * nw + w], counts[q] += marks.
__global__ void pack_labels_kernel(const uint8_t* __restrict__ labels, int64_t nq, int64_t n, int64_t na,
                                   uint32_t* __restrict__ bits, int* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 31) >> 5;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; t < nq * nw; t += warps) {
        const int64_t q = t / nw, w = t - q * nw;
        const int64_t j = (w << 5) + lane;
        bool mark = false;
        if (j < n) mark = q == 0 ? j < na : labels[(q - 1) * n + j] != 0;
        const uint32_t word = __ballot_sync(kFull, mark);
        if (lane == 0) {
            bits[t] = word;
            if (word) atomicAdd(counts + q, __popc(word));
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// stat[q] for q in [blockIdx.x * kPermPerBlock, ... + kPermPerBlock) ∩ [0, nq); written to
// out[0] for q = 0 and out[1 + q] otherwise.
__global__ void __launch_bounds__(kPermWarps * 32)
    mmd_perm_stats_kernel(const double* __restrict__ K, int64_t n, int64_t na, const uint32_t* __restrict__ bits,
                          const int* __restrict__ counts, int64_t nq, int unbiased, double* __restrict__ out) {
    constexpr int PB = kPermPerBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (n + 31) >> 5;
    const int64_t q0 = static_cast<int64_t>(blockIdx.x) * PB;
    const uint32_t* qbits[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) qbits[q] = bits + (q0 + q < nq ? q0 + q : q0) * nw;  // past the end: a copy of q0, unused

    double s11[PB], s00[PB], s10[PB], d11[PB], d00[PB];
#pragma unroll
    for (int q = 0; q < PB; ++q) s11[q] = s00[q] = s10[q] = d11[q] = d00[q] = 0.0;

    for (int64_t i = warp; i < n; i += kPermWarps) {
        const double* __restrict__ Ki = K + i * n;
        double r[PB], t = 0.0;
#pragma unroll
        for (int q = 0; q < PB; ++q) r[q] = 0.0;
        for (int64_t w = 0; w < nw; ++w) {
            const int64_t j = (w << 5) + lane;
            const double kij = j < n ? Ki[j] : 0.0;
            t += kij;
#pragma unroll
            for (int q = 0; q < PB; ++q)
                if ((__ldg(qbits[q] + w) >> lane) & 1u) r[q] += kij;
        }
        t = warp_sum(t);
#pragma unroll
        for (int q = 0; q < PB; ++q) r[q] = warp_sum(r[q]);
        const double kii = Ki[i];
        const int64_t wi = i >> 5;
        const int bi = static_cast<int>(i & 31);
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            if ((__ldg(qbits[q] + wi) >> bi) & 1u) {
                s11[q] += r[q];
                s10[q] += t - r[q];
                d11[q] += kii;
            } else {
                s00[q] += t - r[q];
                d00[q] += kii;
            }
        }
    }

    __shared__ double part[kPermWarps][PB][5];
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            part[warp][q][0] = s11[q];
            part[warp][q][1] = s00[q];
            part[warp][q][2] = s10[q];
            part[warp][q][3] = d11[q];
            part[warp][q][4] = d00[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < PB && q0 + threadIdx.x < nq) {
        const int q = threadIdx.x;
        double a11 = 0.0, a00 = 0.0, a10 = 0.0, e11 = 0.0, e00 = 0.0;
        for (int w = 0; w < kPermWarps; ++w) {
            a11 += part[w][q][0];
            a00 += part[w][q][1];
            a10 += part[w][q][2];
            e11 += part[w][q][3];
            e00 += part[w][q][4];
        }
        const int64_t gq = q0 + q;
        const double fa = static_cast<double>(na), fb = static_cast<double>(n - na);
        double stat;
        if (counts[gq] != na) {
            record_error(SK_ERR_BAD_LABELS);
            stat = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
        } else if (unbiased) {
            stat = (a11 - e11) / (fa * (fa - 1.0)) + (a00 - e00) / (fb * (fb - 1.0)) - 2.0 * a10 / (fa * fb);
        } else {
            stat = a11 / (fa * fa) + a00 / (fb * fb) - 2.0 * a10 / (fa * fb);
        }
        out[gq == 0 ? 0 : 1 + gq] = stat;
    }
}

// out[1] = (1 + #{p : out[2 + p] >= out[0]}) / (1 + nperm); one block, integer counts.
// The p-value is NaN when the observed statistic or any relabelling's statistic is NaN (a bad
// relabelling row, or non-finite Gram entries): a count over the others would look plausible.
__global__ void mmd_perm_pvalue_kernel(int64_t nperm, double* out) {
    __shared__ long long part[256];
    __shared__ int any_nan;
    if (threadIdx.x == 0) any_nan = 0;
    __syncthreads();
    const double obs = out[0];
    long long c = 0;
    bool nan_seen = isnan(obs);
    for (int64_t p = threadIdx.x; p < nperm; p += blockDim.x) {
        const double v = out[2 + p];
        c += v >= obs ? 1 : 0;
        nan_seen |= isnan(v);
    }
    if (nan_seen) atomicOr(&any_nan, 1);
    part[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (static_cast<int>(threadIdx.x) < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[1] = any_nan ? __longlong_as_double(0x7ff8000000000000LL)
                         : static_cast<double>(1 + part[0]) / static_cast<double>(1 + nperm);
}

// K[(na + b) n + a] = K[a n + na + b]: the K_BA block from K_AB.
__global__ void mirror_cross_kernel(double* K, int64_t n, int64_t na) {
    const int64_t nb = n - na;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < na * nb;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t / na, a = t - b * na;  // consecutive threads write consecutive a
        K[(na + b) * n + a] = K[a * n + na + b];
    }
}

}  // namespace

size_t mmd_perm_scratch_bytes(int64_t n, int64_t nperm) {
    const size_t nw = static_cast<size_t>((n + 31) >> 5);
    const size_t nq = static_cast<size_t>(nperm) + 1;
    return (nq * nw * 4 + 255) / 256 * 256 + (nq * 4 + 255) / 256 * 256;
}

cudaError_t launch_mmd_perm(double* K, int64_t n, int64_t na, const uint8_t* labels, int64_t nperm, int unbiased,
                            void* scratch, double* out, cudaStream_t st) {
    const int64_t nq = nperm + 1;
    const size_t nw = static_cast<size_t>((n + 31) >> 5);
    uint32_t* bits = static_cast<uint32_t*>(scratch);
    int* counts = reinterpret_cast<int*>(static_cast<char*>(scratch) + (static_cast<size_t>(nq) * nw * 4 + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(counts, 0, static_cast<size_t>(nq) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (n > na) {
        const int64_t cross = na * (n - na);
        mirror_cross_kernel<<<static_cast<unsigned>(std::min<int64_t>((cross + 255) / 256, 4096)), 256, 0, st>>>(K, n, na);
    }
    const int64_t words = nq * static_cast<int64_t>(nw);
    pack_labels_kernel<<<static_cast<unsigned>(std::min<int64_t>((words + 7) / 8, 65535)), 256, 0, st>>>(labels, nq, n, na,
                                                                                                        bits, counts);
    mmd_perm_stats_kernel<<<static_cast<unsigned>((nq + kPermPerBlock - 1) / kPermPerBlock), kPermWarps * 32, 0, st>>>(
        K, n, na, bits, counts, nq, unbiased, out);
    mmd_perm_pvalue_kernel<<<1, 256, 0, st>>>(nperm, out);
    return cudaGetLastError();
}

}  // namespace sk
