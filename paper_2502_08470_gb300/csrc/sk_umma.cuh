// Fifth-generation tensor-core (tcgen05) helpers for sm_103a, as inline PTX: tensor-memory
// allocation, the shared-memory matrix and instruction descriptors of a BF16 MMA with FP32
// accumulation, the MMA itself, its completion on an mbarrier, and loads of the accumulator.
//
// Operand tiles live in shared memory in the K-major 128-byte-swizzle layout: a tile of R rows
// (R a multiple of 8) and 64 K-elements per 128-byte row; eight rows form a 1024-byte atom, and
// within an atom the 16-byte chunk c of row r sits at chunk position c ^ (r % 8).  Tiles with more
// than 64 K-elements are several such R-row blocks, one per 64 K-elements.  Every tile starts on a
// 1024-byte boundary, so the swizzle the tensor core applies to the address bits matches the one
// sw128_offset() applies when the tile is written.
//
// An MMA of shape M x N x 16 (M = 128: row m of the accumulator is tensor-memory lane m, column n
// is tensor-memory column n) reads a 32-byte slice of each row; successive K-slices of an atom
// are addressed by advancing the descriptor's start address by 32 bytes.
#pragma once

#include <stdint.h>

#include "sk_tma.cuh"

namespace sk {

// Byte offset of element (r, k) of a K-major BF16 tile of R rows in the 128-byte-swizzle layout.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int k, int R) {
    const uint32_t lin = static_cast<uint32_t>((k >> 6) * R * 128 + (r >> 3) * 1024 + (r & 7) * 128 + (k & 63) * 2);
    return lin ^ (((lin >> 7) & 7u) << 4);
}

// Shared-memory matrix descriptor of a K-major 128-byte-swizzle tile whose current K-slice starts
// at shared address `addr`: start address (bits 0-13, in 16-byte units), leading-dimension byte
// offset (bits 16-29; not used by swizzled K-major layouts, set to 16 bytes), stride-dimension
// byte offset (bits 32-45: the 1024 bytes between 8-row groups), descriptor version 1 (bits
// 46-47), base offset 0 (tiles are 1024-byte aligned), layout 2 = 128-byte swizzle (bits 61-63).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
    uint64_t d = static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(16 >> 4) << 16;
    d |= static_cast<uint64_t>(1024 >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// Non-swizzled shared-memory matrix descriptor (layout 0) of a tile of 8 x 8 core matrices (each
// 128 contiguous bytes, row r of a core matrix at 16 r): start address, the byte offset between
// core matrices adjacent along K (lbo) and along M / N (sbo), version 1.  For a K-major operand a
// K-slice of 16 elements is two core matrices along K, so slice k starts at addr + 2 k lbo.
__device__ __forceinline__ uint64_t desc_cm(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

__device__ __forceinline__ void mbar_arrive_one(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major), FP32 accumulator, dense:
// D format F32 (bits 4-5 = 1), A format BF16 (bits 7-9 = 1), B format BF16 (bits 10-12 = 1),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one M x N x 16 slice; issued by one thread.  accumulate = 0 overwrites.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Tensor-memory allocation of `ncols` columns (a power of two >= 32) by one whole warp; the base
// address is written to the shared-memory word `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tensor-core operations around thread synchronisation.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of the warp's 32 tensor-memory lanes (lane = thread): warp
// w % 4 may address lanes 32 (w % 4) .. 32 (w % 4) + 31 only.  Complete with tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// BF16 split of an FP32 value: hi = bf16(x), lo = bf16(x - hi); hi*y_hi + hi*y_lo + lo*y_hi
// reproduces x*y to within about 3 x 2^-16 relative: BF16 keeps 8 significant bits, so the
// rounding of each lo and the dropped lo*lo term are each up to 2^-16 of the product.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

}  // namespace sk
