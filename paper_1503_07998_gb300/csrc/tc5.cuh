// 5th-generation tensor core (tcgen05) building blocks in inline PTX for
// sm_103a: tensor-memory allocation, shared-memory matrix descriptors, the
// BF16 and TF32 MMAs with FP32 accumulation in tensor memory, their
// completion signal on an mbarrier, and tensor-memory loads and stores.
//
// Operand layouts (no swizzle).  A matrix is stored as 8 x 16-byte "core
// matrices" (8 rows of 8 BF16 or 4 TF32 values); a descriptor gives the start address,
// the byte stride between core matrices adjacent along K (LBO field) and the
// byte stride between core matrices adjacent along M or N (SBO field), for
// K-major and MN-major operands alike.
//   K-major  element (row r, k):  (r % 8) * 16 + (r / 8) * SBO + (k % 8) * 2 + (k / 8) * LBO   (BF16)
//                                 (r % 8) * 16 + (r / 8) * SBO + (k % 4) * 4 + (k / 4) * LBO   (TF32)
//   MN-major element (row r, k):  (r % 8) * 2  + (r / 8) * SBO + (k % 8) * 16 + (k / 8) * LBO   (BF16)
// Tensor memory: 128 lanes x 512 columns of 32 bits per SM; for M = 128 the
// accumulator row m sits in lane m, column n in column base + n.  A warp can
// read only the 32 lanes of its quarter (warp index mod 4).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mvd {
namespace tc5 {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle (layout field 0), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 accumulator,
// M x N tile, A/B K-major (false) or MN-major (true).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// Instruction descriptor of kind::tf32: TF32 A and B (format code 2 in both
// type fields), FP32 accumulator, M x N tile, both operands K-major.  One MMA
// covers K = 8 (32 bytes of a row, two core matrices).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// Whole warp: allocate `ncols` (power of two >= 32) tensor-memory columns and
// write the base address to shared memory.
__device__ __forceinline__ void alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// One thread: D (tensor memory) = A * B (+ D if accumulate), A and B from
// shared memory.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One thread: arrive once on `bar` when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Warp: 32 lanes x 32 consecutive columns; thread i receives its lane's
// columns in r[0..31].
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Warp: 32 lanes x 8 consecutive columns.
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Warp: 32 lanes x 16 consecutive columns.
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One thread: D (tensor memory) = A * B (+ D), A from tensor memory (BF16,
// column c of a row holding k = 2c in its low and 2c+1 in its high half), B
// from shared memory.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One thread: D (tensor memory) = A * B (+ D), kind::tf32, A from tensor
// memory (one TF32 value per 32-bit column), B from shared memory.
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// FP32 -> TF32 (10 explicit mantissa bits), round to nearest, ties away from
// zero; the result is an FP32 bit pattern whose low 13 bits are zero.  On the
// sign-magnitude bit pattern, adding half a TF32 unit (bit 12) and clearing
// the 13 dropped bits rounds the magnitude half away from zero; a carry out
// of the mantissa correctly bumps the exponent.  Two integer operations,
// equal to cvt.rna.tf32.f32 for finite inputs (checked bit for bit on the
// tensor-route workloads).
__device__ __forceinline__ uint32_t to_tf32(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// Warp: write N consecutive columns of each thread's lane (N = 16, 8, 4, 2, 1).
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t *w) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
        "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
        : "memory");
}
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t *w) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}
__device__ __forceinline__ void st4(uint32_t taddr, const uint32_t *w) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3])
                 : "memory");
}
__device__ __forceinline__ void st2(uint32_t taddr, const uint32_t *w) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(w[0]), "r"(w[1]) : "memory");
}

// N (compile time, even) consecutive columns from w[0..N).
template <int N>
__device__ __forceinline__ void st_cols(uint32_t taddr, const uint32_t *w) {
    static_assert(N % 2 == 0, "even column counts");
    int c = 0;
#pragma unroll
    for (; c + 16 <= N; c += 16) st16(taddr + c, w + c);
    if constexpr (N % 16 >= 8) {
        st8(taddr + c, w + c);
        c += 8;
    }
    if constexpr (N % 8 >= 4) {
        st4(taddr + c, w + c);
        c += 4;
    }
    if constexpr (N % 4 >= 2) st2(taddr + c, w + c);
}

__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace tc5
}  // namespace mvd
