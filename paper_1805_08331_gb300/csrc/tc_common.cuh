// tc_common.cuh -- Blackwell (sm_100 family) tensor-core helpers in inline PTX:
// TMEM allocation, shared-memory matrix descriptors, tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulation), commit to an mbarrier, TMEM loads.
//
// Operand layout used throughout: K-major, 128-byte swizzle.  A tile of R rows
// x 128 K-elements (BF16) is stored as two halves of 64 K-elements; each half
// is R rows of 128 bytes, in atoms of 8 rows (1024 bytes, 1024-byte aligned).
// Inside an atom the 16-byte chunk c of row r is stored at chunk position
// c ^ (r % 8).  One MMA consumes K = 16 (32 bytes of a row): step s starts at
// half s/4, byte offset 32 (s % 4) inside the row.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row r, k) in a K-major SW128 tile with 128 K-elements.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k, int rows) {
    const int h = k >> 6, kk = k & 63, chunk = kk >> 3, within = kk & 7;
    return (uint32_t)(h * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) + within * 2);
}

// Shared-memory matrix descriptor: start address, leading byte offset 16 (not
// used by swizzled K-major layouts), stride byte offset 1024 (8-row atoms),
// descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// D[tmem] (+)= A[adesc] * B[bdesc]^T  (both K-major), issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// Arrive on the mbarrier once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;");
}
// Bounded wait for the mbarrier phase `parity` to complete; returns false if
// the iteration limit ran out (the caller records an error and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_spins = 1u << 26) {
    const uint32_t a = smem_u32(mbar);
    for (uint32_t it = 0; it < max_spins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// Make generic-proxy shared-memory writes visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }

// Load 32 consecutive FP32 columns of this thread's TMEM lane (32x32b shape, x32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Pack two floats to BF16x2 with round-to-nearest, saturating to the finite range.
__device__ __forceinline__ uint32_t pack_bf16x2_sat(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.satfinite.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// One 128 x 128 x 128 GEMM step: D (TMEM, 128 lanes x 128 FP32 columns) =
// A (128 x 128, K-major SW128 at sa) * B (128 x 128, K-major SW128 at sb)^T,
// as 8 MMAs of K = 16.  Issued by one thread; commit to mbar.
__device__ __forceinline__ void gemm128_issue(uint32_t tmem_d, uint32_t sa, uint32_t sb, uint64_t* mbar) {
    constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const uint32_t off = (uint32_t)((s >> 2) * 128 * 128 + (s & 3) * 32);
        mma_bf16(tmem_d, sw128_desc(sa + off), sw128_desc(sb + off), idesc, s > 0 ? 1u : 0u);
    }
    mma_commit(mbar);
}
