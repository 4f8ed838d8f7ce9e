// Chain rule through M_ij = <dx_i, dy_j> on the tensor cores (FP32 compute mode, BF16 x 3).
//
// For one pair with cell gradient G = dk/dM (rows x cols, refined grid, from the tape adjoint)
//     dk/dx_{i >> lambda} += sum_j G_ij dy_{j >> lambda}      (D1 = G . DY,   K = columns)
//     dk/dy_{j >> lambda} += sum_i G_ij dx_{i >> lambda}      (D2 = G^T . DX, K = rows)
// two GEMMs with a shared left operand.  G arrives as BF16 high and low parts in 128 x 128 blocks
// of 8 x 8 core matrices (gtile_index), which the tensor core reads as the K-major operand of D1
// and as the M-major (transposed) operand of D2 without any reshuffling; the increments come
// transposed and split the same way (tc_operand_offset), one 128-row block per operand tile.  Each
// product is hi*hi + hi*lo + lo*hi (relative error at most about 3 x 2^-16 per product: the
// rounding of each lo and the dropped lo*lo, each up to 2^-16), accumulated in FP32
// in tensor memory, and the sums go to the FP64 gradients with gbar 2^ek, as in the FMA
// contraction (bwd_contract_kernel).
//
// One CTA per SM, persistent over a contiguous range of items, warp-specialised:
//   warp 0     bulk copies of each 128 x 128 block of G (64 KB) and of the two increment tiles
//              into a two-stage shared-memory ring;
//   warp 1     allocates tensor memory (512 columns: two halves, so that the epilogue of one item
//              overlaps the MMAs of the next) and issues the MMAs (one thread);
//   warps 2-5  epilogue: tensor memory -> registers -> FP64 atomics.
// Every mbarrier wait is bounded; a wait that runs out records SK_ERR_DEVICE_TIMEOUT, the role
// stops, and the CTA drains its copies and MMAs in flight before freeing tensor memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"
#include "sk_umma.cuh"

namespace sk {

constexpr int kTcThreads = 192;
constexpr int kTmemCols = 512;
constexpr int kTmemHalf = 256;

// Byte offset of element (n, kk) of the (hi or lo) plane of one operand tile: N coordinates x 128
// rows of a path, K-major 8 x 8 core matrices (core matrix (n / 8, kk / 8) at ((n / 8) * 16 +
// kk / 8) * 128 bytes, element (n % 8, kk % 8) at (n % 8) * 16 + (kk % 8) * 2).
__device__ __forceinline__ uint32_t tc_operand_offset(int n, int kk) {
    return static_cast<uint32_t>(((n >> 3) * 16 + (kk >> 3)) * 128 + (n & 7) * 16 + (kk & 7) * 2);
}

// Operand tiles of one path set: for path p and 128-row block k (refined rows k*128..k*128+127),
// the hi plane then the lo plane of the N x 128 transposed increments (row i of the refined grid
// uses increment i >> lambda; rows past the path and coordinates past d are zero).
template <int N>
__global__ void tc_operand_kernel(PathSet S, int inc_mode, int lam, int dpad, int nblk, unsigned char* out) {
    constexpr int kPlane = N * 256;
    const float* __restrict__ inc = static_cast<const float*>(S.inc);
    for (int64_t pb = blockIdx.x; pb < S.count * nblk; pb += gridDim.x) {
        const int64_t p = pb / nblk;
        const int k = static_cast<int>(pb - p * nblk);
        int64_t start, len;
        path_span(S, p, inc_mode, start, len);
        const int64_t rows = len > 0 ? (len << lam) : 0;
        unsigned char* hi = out + pb * 2 * kPlane;
        unsigned char* lo = hi + kPlane;
        for (int e = threadIdx.x; e < N * 128; e += blockDim.x) {
            const int n = e >> 7, kk = e & 127;
            const int64_t i = static_cast<int64_t>(k) * 128 + kk;
            float v = 0.f;
            if (i < rows && n < dpad) v = inc[(start + (i >> lam)) * dpad + n];
            __nv_bfloat16 h, l;
            split_bf16(v, h, l);
            const uint32_t o = tc_operand_offset(n, kk);
            *reinterpret_cast<__nv_bfloat16*>(hi + o) = h;
            *reinterpret_cast<__nv_bfloat16*>(lo + o) = l;
        }
    }
}

struct TcItem {
    PairDesc P;
    int rows, cols, nrb, ncb;
    double gscale;
};

// The item's geometry, or false when the adjoint skipped it (no cells, invalid, zero weight).
__device__ __forceinline__ bool tc_item(const BwdParams& B, int64_t item, TcItem& t) {
    const Launch& L = B.L;
    t.P = decode_pair(L, item);
    if (t.P.lx <= 0 || t.P.ly <= 0) return false;
    const double gbar = item_gbar(B, item, t.P);
    if (gbar == 0.0) return false;
    t.gscale = gbar * pow2d(L.tape_ek[item]);
    t.rows = static_cast<int>(t.P.lx << L.lam);
    t.cols = static_cast<int>(t.P.ly << L.lam);
    t.nrb = (t.rows + 127) >> 7;
    t.ncb = (t.cols + 127) >> 7;
    return true;
}

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1) bwd_contract_tc_kernel(BwdParams B, int64_t per_cta, int nrb_max) {
    constexpr int kOper = 2 * N * 256;               // one operand tile: hi and lo planes
    constexpr int kStage = 65536 + 2 * kOper;        // G block (hi, lo), DY tile, DX tile
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, N);
    constexpr uint32_t kIdescT = kIdesc | (1u << 15);  // A (G) read M-major: its transpose
    const Launch& L = B.L;
    extern __shared__ __align__(16) unsigned char tc_raw[];
    const uint32_t raw = smem_u32(tc_raw);
    unsigned char* sm = tc_raw + (((raw + 1023) & ~1023u) - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + 2 * kStage);
    uint64_t* empty = full + 2;
    uint64_t* tfull = full + 4;
    uint64_t* tempty = full + 6;
    uint64_t* drain = full + 8;
    uint32_t* slot = reinterpret_cast<uint32_t*>(full + 9);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
            mbar_init(tfull + s, 1);
            mbar_init(tempty + s, 4);
        }
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *slot;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * per_cta;
    const int64_t i1 = min(i0 + per_cta, L.npairs);

    if (warp == 0) {
        if (lane == 0) {  // producer
            uint32_t it = 0;
            bool stuck = false;
            for (int64_t item = i0; item < i1 && !stuck; ++item) {
                TcItem t;
                if (!tc_item(B, item, t)) continue;
                const char* gsrc = static_cast<const char*>(B.mbuf) + item * B.mb_stride;
                const char* ysrc = static_cast<const char*>(B.yt) + t.P.b * static_cast<int64_t>(B.yt_nblk) * kOper;
                const char* xsrc = static_cast<const char*>(B.xt) + t.P.a * static_cast<int64_t>(B.xt_nblk) * kOper;
                for (int rb = 0; rb < t.nrb && !stuck; ++rb)
                    for (int cb = 0; cb < t.ncb; ++cb, ++it) {
                        const int s = it & 1;
                        const uint32_t u = it >> 1;
                        if (!mbar_wait(empty + s, (u & 1u) ^ 1u)) { stuck = true; break; }
                        unsigned char* st = sm + s * kStage;
                        mbar_arrive_expect_tx(full + s, kStage);
                        bulk_load(st, gsrc + (static_cast<int64_t>(rb) * B.gt_ncb + cb) * 65536, 65536, full + s);
                        bulk_load(st + 65536, ysrc + static_cast<int64_t>(cb) * kOper, kOper, full + s);
                        bulk_load(st + 65536 + kOper, xsrc + static_cast<int64_t>(rb) * kOper, kOper, full + s);
                    }
            }
            // copies still in flight land before the CTA leaves (their phase completes; bounded)
            for (uint32_t k = (it >= 2 ? it - 2 : 0); k < it; ++k) mbar_wait(full + (k & 1), (k >> 1) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            uint32_t it = 0, nitem = 0;
            bool stuck = false;
            for (int64_t item = i0; item < i1 && !stuck; ++item) {
                TcItem t;
                if (!tc_item(B, item, t)) continue;
                const uint32_t h = nitem & 1, v = nitem >> 1;
                if (!mbar_wait(tempty + h, (v & 1u) ^ 1u)) { stuck = true; break; }
                tc_fence_after();
                const uint32_t tb = taddr + h * kTmemHalf;
                for (int rb = 0; rb < t.nrb && !stuck; ++rb)
                    for (int cb = 0; cb < t.ncb; ++cb, ++it) {
                        const int s = it & 1;
                        const uint32_t u = it >> 1;
                        if (!mbar_wait(full + s, u & 1u)) { stuck = true; break; }
                        tc_fence_after();
                        const uint32_t g = smem_u32(sm + s * kStage), y = g + 65536, x = y + kOper;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {  // K slices of 16
                            // D1[rb] += G (rows x 16 columns) . DY^T
                            const uint64_t ah = desc_cm(g + 256 * k, 128, 2048), al = desc_cm(g + 32768 + 256 * k, 128, 2048);
                            const uint64_t bh = desc_cm(y + 256 * k, 128, 2048), bl = desc_cm(y + N * 256 + 256 * k, 128, 2048);
                            const uint32_t d1 = tb + rb * N;
                            umma_bf16(d1, ah, bh, kIdesc, (cb > 0 || k > 0) ? 1u : 0u);
                            umma_bf16(d1, ah, bl, kIdesc, 1u);
                            umma_bf16(d1, al, bh, kIdesc, 1u);
                            // D2[cb] += G^T (columns x 16 rows) . DX^T
                            const uint64_t th = desc_cm(g + 4096 * k, 2048, 128), tl = desc_cm(g + 32768 + 4096 * k, 2048, 128);
                            const uint64_t xh = desc_cm(x + 256 * k, 128, 2048), xl = desc_cm(x + N * 256 + 256 * k, 128, 2048);
                            const uint32_t d2 = tb + (nrb_max + cb) * N;
                            umma_bf16(d2, th, xh, kIdescT, (rb > 0 || k > 0) ? 1u : 0u);
                            umma_bf16(d2, th, xl, kIdescT, 1u);
                            umma_bf16(d2, tl, xh, kIdescT, 1u);
                        }
                        umma_commit(empty + s);  // the stage is free once these MMAs have read it
                    }
                umma_commit(tfull + h);  // the item's sums are complete
                ++nitem;
            }
            umma_commit(drain);  // every MMA of this CTA has finished before tensor memory is freed
            mbar_wait(drain, 0);
        }
    } else {  // epilogue warps 2..5: tensor-memory lanes 32 (warp % 4) ..
        const int q = warp & 3;
        const int lam = L.lam, dpad = L.dpad;
        uint32_t nitem = 0;
        for (int64_t item = i0; item < i1; ++item) {
            TcItem t;
            if (!tc_item(B, item, t)) continue;
            const uint32_t h = nitem & 1, v = nitem >> 1;
            if (!mbar_wait(tfull + h, v & 1u)) break;
            tc_fence_after();
            const uint32_t tb = taddr + h * kTmemHalf + ((32u * q) << 16);
            double* gx = B.gincX + t.P.xs * dpad;
            double* gy = B.gincY + t.P.ys * dpad;
            for (int blk = 0; blk < t.nrb + t.ncb; ++blk) {
                const bool isx = blk < t.nrb;
                const int b = isx ? blk : blk - t.nrb;
                const int r = b * 128 + 32 * q + lane;  // grid row (D1) or column (D2)
                const bool ok = r < (isx ? t.rows : t.cols);
                double* g = (isx ? gx : gy) + static_cast<int64_t>(ok ? (r >> lam) : 0) * dpad;
                const uint32_t col = isx ? b * N : (nrb_max + b) * N;
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float vals[16];
                    tmem_ld16(tb + col + c0, vals);
                    tmem_ld_wait();
                    if (ok) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (c0 + c < dpad && vals[c] != 0.f) atomicAdd(g + c0 + c, static_cast<double>(vals[c]) * t.gscale);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_one(tempty + h);
            ++nitem;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(taddr, kTmemCols);
    }
}

template <int N>
cudaError_t launch_tc(const BwdParams& B, int nrb_max, int sms, cudaStream_t st) {
    const int smem = 2 * (65536 + 4 * N * 256) + 1024 + 128;
    cudaError_t e = cudaFuncSetAttribute(bwd_contract_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(sms, std::max<int64_t>(B.L.npairs, 1));
    const int64_t per = (B.L.npairs + grid - 1) / grid;
    bwd_contract_tc_kernel<N><<<static_cast<int>(grid), kTcThreads, smem, st>>>(B, per, nrb_max);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_operands(const PathSet& S, int inc_mode, int lam, int dpad, int nblk, void* out, cudaStream_t st) {
    if (S.count == 0) return cudaSuccess;
    const int64_t nb = S.count * nblk;
    tc_operand_kernel<N><<<static_cast<int>(std::min<int64_t>(nb, 65535)), 256, 0, st>>>(
        S, inc_mode, lam, dpad, nblk, static_cast<unsigned char*>(out));
    return cudaGetLastError();
}

size_t tc_operand_bytes(int N, int64_t paths, int nblk) {
    return static_cast<size_t>(paths) * nblk * 2 * N * 256;
}

cudaError_t launch_tc_operands(int N, const PathSet& S, int inc_mode, int lam, int dpad, int nblk, void* out,
                               cudaStream_t st) {
    return N == 16 ? launch_operands<16>(S, inc_mode, lam, dpad, nblk, out, st)
                   : launch_operands<32>(S, inc_mode, lam, dpad, nblk, out, st);
}

cudaError_t launch_tc_contraction(int N, const BwdParams& B, int nrb_max, int sms, cudaStream_t st) {
    return N == 16 ? launch_tc<16>(B, nrb_max, sms, st) : launch_tc<32>(B, nrb_max, sms, st);
}

}  // namespace sk
