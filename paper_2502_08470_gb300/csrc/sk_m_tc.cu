// The increment inner products M_ij = <dx_i, dy_j> / 4^lambda of every cell of a batch of pairs on
// the tensor cores (tcgen05, FP32 compute mode with 4 < d <= 32), for the wavefront to read.
//
// For a pair (a, b) the cells' M is the product of the pair's increment rows, DX_a (rows x d) times
// DY_b^T (d x cols), with refined row i using increment i >> lambda.  Each FP32 increment is split
// into three BF16 parts, x = h + m + l with h = bf16(x), m = bf16(x - h), l = bf16(x - h - m): both
// differences are exact in FP32 and the last has at most 8 significant bits, so the split is exact
// for |x| >= 2^-110.  Each 128 x 128 tile of M accumulates, in FP32 in tensor memory, the six
// products whose parts carry at least 2^-16 of the value, smallest first: mm', hl', lh', hm', mh',
// hh'.  The dropped ml', lm', ll' are at most 2 x 2^-24 + 2^-32 (about 2^-23) of each product, the
// order of the FP32 inner product's own rounding (a two-part split left about 2^-16, which moved
// Gram entries by 1e-4 relative).  The operand tiles are prepared
// once per call: per path and 128-row block, the h, m and l planes of 128 rows x KP coordinates
// (KP = d rounded up to 16 or 32, zero padded) in K-major 8 x 8 core matrices.
//
// M is written in the order the wavefront consumes it: for the pair's warp schedule (strips of 32
// rows, cell (32 s + r, j) at warp step s P + j + r with P = max(cols, 32)), the steps go in groups
// of four, and group G holds lane r's M of steps 4G .. 4G + 3 as the float4 at (32 G + r) * 4, so
// one coalesced 512-byte load gives the warp four steps of M.
//
// One CTA per SM over a contiguous range of pairs, warp-specialised as the tensor-core contraction
// (sk_contract_tc.cu): warp 0 bulk-copies each tile's two operand tiles into a two-stage ring,
// warp 1 allocates the tensor memory (two 128-column accumulators) and issues the MMAs, warps 2..9
// move each accumulator through shared memory to the M buffer (two warps per 32-row strip of the
// tile, 64 columns each), one float4 per lane and store.  Every mbarrier wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>

#include "sk_bwd_poly.cuh"
#include "sk_dispatch.h"
#include "sk_umma.cuh"

namespace sk {

constexpr int kMtEpiWarps = 8;
constexpr int kMtThreads = 64 + 32 * kMtEpiWarps;
constexpr int kMtRow = 100;                 // staging floats per lane (64 + 31 + 3 steps, 16-byte rows)
constexpr int kMtStage = 32 * kMtRow * 4;  // staging bytes per epilogue warp
constexpr int kMtStages = 2;
constexpr int kMtParts = 3;  // BF16 parts per FP32 operand

// Byte offset of element (r, k) of one (hi or lo) plane of an operand tile: 128 rows x KP
// coordinates, core matrix (r / 8, k / 8) at ((r / 8) * (KP / 8) + k / 8) * 128 bytes, element
// (r % 8, k % 8) at (r % 8) * 16 + (k % 8) * 2.
template <int KP>
__device__ __forceinline__ uint32_t m_operand_offset(int r, int k) {
    return static_cast<uint32_t>(((r >> 3) * (KP / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Operand tiles of a path set: for path p and 128-row block k, the h, m and l parts of the refined
// rows' increments scaled by 2^-lambda (exact), so that the products are M_ij / 4^lambda.
template <int KP>
__global__ void m_operand_kernel(PathSet S, int inc_mode, int lam, int dpad, int nblk, unsigned char* out) {
    constexpr int kPlane = 128 * KP * 2;  // one part of a tile
    const float* __restrict__ inc = static_cast<const float*>(S.inc);
    const float scale = pow2f(-lam);
    for (int64_t pb = blockIdx.x; pb < S.count * nblk; pb += gridDim.x) {
        const int64_t p = pb / nblk;
        const int k = static_cast<int>(pb - p * nblk);
        int64_t start, len;
        path_span(S, p, inc_mode, start, len);
        const int64_t rows = len > 0 ? (len << lam) : 0;
        unsigned char* hi = out + pb * kMtParts * kPlane;
        for (int e = threadIdx.x; e < 128 * KP; e += blockDim.x) {
            const int r = e / KP, c = e - r * KP;
            const int64_t i = static_cast<int64_t>(k) * 128 + r;
            float v = 0.f;
            if (i < rows && c < dpad) v = inc[(start + (i >> lam)) * dpad + c] * scale;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const float r1 = v - __bfloat162float(h);
            const __nv_bfloat16 m = __float2bfloat16_rn(r1);
            const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
            const uint32_t o = m_operand_offset<KP>(r, c);
            *reinterpret_cast<__nv_bfloat16*>(hi + o) = h;
            *reinterpret_cast<__nv_bfloat16*>(hi + kPlane + o) = m;
            *reinterpret_cast<__nv_bfloat16*>(hi + 2 * kPlane + o) = l;
        }
    }
}

struct MtParams {
    const unsigned char* xt;  // operand tiles of X: [X.count][xt_nblk][hi, lo]
    const unsigned char* yt;  // of Y
    int32_t xt_nblk, yt_nblk;
    float* mx;                // per item: [steps][32] (the forward tape's layout)
    int64_t mx_stride;        // bytes per item
    int64_t per_cta;          // items per CTA
};

__device__ __forceinline__ bool m_item(const Launch& L, int64_t item, PairDesc& P, int& rows, int& cols) {
    P = decode_pair(L, item);
    if (P.lx <= 0 || P.ly <= 0) return false;
    rows = static_cast<int>(P.lx << L.lam);
    cols = static_cast<int>(P.ly << L.lam);
    return true;
}

template <int KP>
__global__ void __launch_bounds__(kMtThreads, 1) m_tc_kernel(Launch L, MtParams M) {
    constexpr int kPlane = 128 * KP * 2;
    constexpr int kTile = kMtParts * kPlane;          // one operand tile: its h, m and l parts
    constexpr int kStage = 2 * kTile;                  // the X tile and the Y tile
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, 128);
    constexpr uint32_t kSbo = (KP / 8) * 128;         // 8-row groups of a tile
    extern __shared__ __align__(16) unsigned char mt_raw[];
    const uint32_t raw = smem_u32(mt_raw);
    unsigned char* sm = mt_raw + (((raw + 1023) & ~1023u) - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kMtStages * kStage + kMtEpiWarps * kMtStage);
    uint64_t* empty = full + kMtStages;
    uint64_t* tfull = full + 2 * kMtStages;
    uint64_t* tempty = full + 3 * kMtStages;
    uint64_t* drain = full + 4 * kMtStages;
    uint32_t* slot = reinterpret_cast<uint32_t*>(drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMtStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
            mbar_init(tfull + s, 1);
            mbar_init(tempty + s, kMtEpiWarps);
        }
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(slot, 256);  // two 128-column accumulators
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *slot;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * M.per_cta;
    const int64_t i1 = min(i0 + M.per_cta, L.npairs);

    if (warp == 0) {
        if (lane == 0) {  // producer
            uint32_t it = 0;
            bool stuck = false;
            for (int64_t item = i0; item < i1 && !stuck; ++item) {
                PairDesc P;
                int rows, cols;
                if (!m_item(L, item, P, rows, cols)) continue;
                const int nrb = (rows + 127) >> 7, ncb = (cols + 127) >> 7;
                const unsigned char* xs = M.xt + P.a * static_cast<int64_t>(M.xt_nblk) * kTile;
                const unsigned char* ys = M.yt + P.b * static_cast<int64_t>(M.yt_nblk) * kTile;
                for (int rb = 0; rb < nrb && !stuck; ++rb)
                    for (int cb = 0; cb < ncb; ++cb, ++it) {
                        const int s = it % kMtStages;
                        const uint32_t u = it / kMtStages;
                        if (!mbar_wait(empty + s, (u & 1u) ^ 1u)) { stuck = true; break; }
                        unsigned char* st = sm + s * kStage;
                        mbar_arrive_expect_tx(full + s, kStage);
                        bulk_load(st, xs + static_cast<int64_t>(rb) * kTile, kTile, full + s);
                        bulk_load(st + kTile, ys + static_cast<int64_t>(cb) * kTile, kTile, full + s);
                    }
            }
            for (uint32_t k = (it >= kMtStages ? it - kMtStages : 0); k < it; ++k)
                mbar_wait(full + (k % kMtStages), (k / kMtStages) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer: one 128 x 128 accumulator per tile, four in rotation
            uint32_t it = 0;
            bool stuck = false;
            for (int64_t item = i0; item < i1 && !stuck; ++item) {
                PairDesc P;
                int rows, cols;
                if (!m_item(L, item, P, rows, cols)) continue;
                const int ntiles = ((rows + 127) >> 7) * ((cols + 127) >> 7);
                for (int t = 0; t < ntiles; ++t, ++it) {
                    const int s = it % kMtStages;
                    const uint32_t u = it / kMtStages;
                    if (!mbar_wait(tempty + s, (u & 1u) ^ 1u) || !mbar_wait(full + s, u & 1u)) {
                        stuck = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t x = smem_u32(sm + s * kStage), y = x + kTile;
                    const uint32_t d = taddr + s * 128;
                    // parts (of X, of Y), smallest products first: mm, hl, lh, hm, mh, hh
                    constexpr int kPx[6] = {1, 0, 2, 0, 1, 0}, kPy[6] = {1, 2, 0, 1, 0, 0};
#pragma unroll
                    for (int t = 0; t < 6; ++t)
#pragma unroll
                        for (int k = 0; k < KP / 16; ++k)
                            umma_bf16(d, desc_cm(x + kPx[t] * kPlane + 256 * k, 128, kSbo),
                                      desc_cm(y + kPy[t] * kPlane + 256 * k, 128, kSbo), kIdesc,
                                      (t | k) ? 1u : 0u);
                    umma_commit(empty + s);
                    umma_commit(tfull + s);
                }
            }
            umma_commit(drain);
            mbar_wait(drain, 0);
        }
    } else {  // epilogue warps 2..9: tensor-memory lanes 32 (warp % 4) .. (one strip of the tile)
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;  // columns 64 half .. 64 half + 63 of the tile
        // The warp's 32 x 64 block goes through shared memory indexed by warp step: lane r's cell
        // of column c, in warp step T0 + c + r, at float r * kMtRow + (c + r + (T0 mod 4)).  Lane r's
        // M of a group of four steps is then one aligned float4, read conflict-free (kMtRow / 4 is
        // odd), and the scalar writes from tensor memory are conflict-free as well (kMtRow + 1 is
        // odd modulo 32).
        float* stg = reinterpret_cast<float*>(sm + kMtStages * kStage + (warp - 2) * kMtStage) + lane * kMtRow;
        uint32_t it = 0;
        for (int64_t item = i0; item < i1; ++item) {
            PairDesc P;
            int rows, cols;
            if (!m_item(L, item, P, rows, cols)) continue;
            const int nrb = (rows + 127) >> 7, ncb = (cols + 127) >> 7;
            const int period = cols > 32 ? cols : 32;
            float4* mx = reinterpret_cast<float4*>(reinterpret_cast<char*>(M.mx) + item * M.mx_stride);
            bool stuck = false;
            for (int rb = 0; rb < nrb && !stuck; ++rb)
                for (int cb = 0; cb < ncb; ++cb, ++it) {
                    const int s = it % kMtStages;
                    const uint32_t u = it / kMtStages;
                    if (!mbar_wait(tfull + s, u & 1u)) { stuck = true; break; }
                    tc_fence_after();
                    const int sg = rb * 4 + q;                   // the strip's index in the pair
                    const int jb = cb * 128 + 64 * half;         // the block's first column
                    const int64_t T0 = static_cast<int64_t>(sg) * period + jb;  // step of cell (32 sg, jb)
                    const int a = static_cast<int>(T0 & 3);
#pragma unroll
                    for (int c0 = 0; c0 < 64; c0 += 16) {
                        float v[16];
                        tmem_ld16(taddr + ((32u * q) << 16) + s * 128 + 64 * half + c0, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int k = 0; k < 16; ++k) stg[c0 + k + lane + a] = v[k];
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_one(tempty + s);  // the accumulator is free again
                    const int ncol = min(64, cols - jb);         // the block's columns in the grid
                    if ((sg << 5) < rows && ncol > 0) {
                        const bool rows_full = (sg << 5) + 32 <= rows;
                        const bool row_ok = (sg << 5) + lane < rows;
                        const int ng = (ncol + 30 + a) / 4 + 1;  // groups of steps the block touches
                        float4* dst = mx + (T0 >> 2) * 32 + lane;
                        // group g holds cells c = 4 g + k - lane - a; all are in the block when
                        // 4 g >= 31 + a and 4 g + 3 - a < ncol
                        const int gin0 = (31 + a + 3) / 4, gin1 = (ncol - 4 + a) / 4;  // interior groups
#pragma unroll 4
                        for (int g = 0; g < ng; ++g) {
                            const float4 w = *reinterpret_cast<const float4*>(stg + 4 * g);
                            if (rows_full && g >= gin0 && g <= gin1) {
                                dst[static_cast<int64_t>(g) * 32] = w;
                            } else if (row_ok) {
                                float* d1 = reinterpret_cast<float*>(dst + static_cast<int64_t>(g) * 32);
                                const float wk[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const int c = 4 * g + k - lane - a;
                                    if (c >= 0 && c < ncol) d1[k] = wk[k];
                                }
                            }
                        }
                    }
                    __syncwarp();  // the staging block is read before the next tile overwrites it
                }
            if (stuck) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(taddr, 256);
    }
}

size_t m_operand_bytes(int KP, int64_t paths, int nblk) {
    return static_cast<size_t>(paths) * nblk * kMtParts * 128 * KP * 2;
}

cudaError_t launch_m_operands(int KP, const PathSet& S, int inc_mode, int lam, int dpad, int nblk, void* out,
                              cudaStream_t st) {
    if (S.count == 0) return cudaSuccess;
    const int blocks = static_cast<int>(std::min<int64_t>(S.count * nblk, 65535));
    if (KP == 16) m_operand_kernel<16><<<blocks, 256, 0, st>>>(S, inc_mode, lam, dpad, nblk, static_cast<unsigned char*>(out));
    else m_operand_kernel<32><<<blocks, 256, 0, st>>>(S, inc_mode, lam, dpad, nblk, static_cast<unsigned char*>(out));
    return cudaGetLastError();
}

cudaError_t launch_m_tc(int KP, const Launch& L, const void* xt, const void* yt, int xt_nblk, int yt_nblk, float* mx,
                        int64_t mx_stride, int sms, cudaStream_t st) {
    MtParams M;
    M.xt = static_cast<const unsigned char*>(xt);
    M.yt = static_cast<const unsigned char*>(yt);
    M.xt_nblk = xt_nblk;
    M.yt_nblk = yt_nblk;
    M.mx = mx;
    M.mx_stride = mx_stride;
    const int64_t grid = std::min<int64_t>(sms, std::max<int64_t>(L.npairs, 1));
    M.per_cta = (L.npairs + grid - 1) / grid;
    const int smem = kMtStages * 2 * (kMtParts * 128 * KP * 2) + kMtEpiWarps * kMtStage + 1024 + 256;
    cudaError_t e;
    if (KP == 16) {
        if ((e = cudaFuncSetAttribute(m_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        m_tc_kernel<16><<<static_cast<int>(grid), kMtThreads, smem, st>>>(L, M);
    } else {
        if ((e = cudaFuncSetAttribute(m_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        m_tc_kernel<32><<<static_cast<int>(grid), kMtThreads, smem, st>>>(L, M);
    }
    return cudaGetLastError();
}

}  // namespace sk
