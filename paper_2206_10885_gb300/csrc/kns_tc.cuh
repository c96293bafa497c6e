// kns_tc.cuh -- Blackwell (sm_100 family) tensor-core building blocks in inline PTX: tensor memory
// (TMEM) allocation, shared-memory matrix descriptors in the canonical no-swizzle K-major layout,
// tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulation in TMEM), commit to an mbarrier, and
// tcgen05.ld of the accumulator back into registers.
//
// Canonical K-major layout without swizzle (both operands): the matrix is cut into "core matrices"
// of 8 rows x 16 bytes (8 BF16 values along K), each stored as 128 contiguous bytes (row r at byte
// 16 r).  Core matrices adjacent along K are LBO bytes apart, 8-row groups adjacent along M (or N)
// are SBO bytes apart.  Here LBO = 128 (the K-chunks of one row group are contiguous) and
// SBO = 16 K bytes (one row group holds all K columns), so element (row, k) of a K-column matrix
// lives at byte  (row / 8) * 16 K + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2.
// One MMA consumes K = 16 (two core matrices along K); the next K-slice starts 256 bytes later.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace kns {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a K-major canonical matrix with K columns.
__host__ __device__ constexpr int canon_off(int row, int k, int K) {
    return (row >> 3) * (16 * K) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Byte layout of one cell's tensor-core trace weights, the same in global and in shared memory (the
// host writes it, one bulk copy moves it): for a grid of SDF width W, H hidden layers and an
// encoding of IN values (K0 = IN rounded up to 16):
//   layer 0:          W0 hi, W0 lo   (W x K0 each, canonical K-major, zero columns beyond IN);
//   layer l=1..H-1:   Wl hi, Wl lo   (W x W);
//   FP32:             biases b_l[W] for l = 0..H-1, the d row of the last layer [W], its bias.
__host__ __device__ constexpr int k0_of(int IN) { return (IN + 15) / 16 * 16; }
__host__ __device__ constexpr int w_hi(int l, int W, int K0) { return l == 0 ? 0 : 4 * W * K0 + (l - 1) * 4 * W * W; }
__host__ __device__ constexpr int w_lo(int l, int W, int K0) { return w_hi(l, W, K0) + (l == 0 ? 2 * W * K0 : 2 * W * W); }
__host__ __device__ constexpr int bias_off(int W, int H, int K0) { return w_hi(H, W, K0); }
__host__ __device__ constexpr int drow_off(int W, int H, int K0) { return bias_off(W, H, K0) + 4 * H * W; }
__host__ __device__ constexpr int cell_bytes(int W, int H, int K0) {
    return (drow_off(W, H, K0) + 4 * W + 16 + 127) / 128 * 128;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and stride (M/N) byte
// offsets, each >> 4 in 14 bits; bits 46..47 = 1 (descriptor version of the sm_100 family);
// base offset 0, relative LBO mode, layout type 0 = no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D format F32 (bits 4..5 = 1), A and B BF16 (bits 7..9 and
// 10..12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17..22, M >> 4 in bits 24..28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp; the base address is
// written to *slot in shared memory.  The permit is released at once (one allocation per CTA).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's generic-proxy shared-memory writes visible to the tensor cores (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, M x N x 16, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, M x N x 16, issued by one thread.  A lives in tensor memory: row m
// of A in lane m, K along the columns, two BF16 values per 32-bit column (the lower k in the low half).
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier receives one arrival when every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w of a warpgroup reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31; taddr carries lane << 16 | column).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane (as tmem_ld32).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stores 8 consecutive 32-bit columns of this thread's TMEM lane (every thread of the warp takes part).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
// Waits until this thread's tcgen05.st have completed (before a barrier that hands the data to an MMA).
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// hi = bf16(x), lo = bf16(x - hi) (both round to nearest): hi + lo carries ~16 significant bits.
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = *reinterpret_cast<const uint16_t *>(&h);
    lo = *reinterpret_cast<const uint16_t *>(&l);
}

}  // namespace tc
}  // namespace kns
