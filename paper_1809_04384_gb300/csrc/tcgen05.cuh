// Inline-PTX helpers for the 5th-generation tensor cores (tcgen05) of sm_103a: TF32 and BF16
// matrix products from shared-memory operands into Tensor Memory (TMEM), completion
// through an mbarrier, and TMEM reads.
//
// Operand layout (both A and B "K-major", no swizzle): a matrix of R rows (M or N) and a
// chunk of KC columns (K) is stored as core matrices of 8 rows x 16 bytes (4 FP32/TF32
// values), the core matrices ordered with the row direction fastest.  Element (r, k) then
// sits at float offset kmaj_off(r, k, R).  In the shared-memory matrix descriptor the
// leading byte offset is the distance between core matrices adjacent in K ((R/8) * 128 B)
// and the stride byte offset the distance between core matrices adjacent in M/N (128 B);
// one MMA of K = 8 reads two core matrices along K.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dh2 {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__host__ __device__ __forceinline__ int kmaj_off(int r, int k, int R) {
    return ((k >> 2) * (R >> 3) + (r >> 3)) * 32 + (r & 7) * 4 + (k & 3);
}

// The same layout with 4 spare floats (16 B) after every K-direction group of core
// matrices: leading byte offset (R/8) * 128 + 16.  Stores whose K index runs across the
// lanes of a warp then fall into different banks.
__host__ __device__ __forceinline__ int kmaj_off_pad(int r, int k, int R) {
    return (k >> 2) * ((R >> 3) * 32 + 4) + (r >> 3) * 32 + (r & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte
// units), descriptor version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// The K-major layout for 16-bit operands: a core matrix is 8 rows x 8 values (16 B), one MMA
// of K = 16 reads two core matrices along K.  Offset in 16-bit elements.
__host__ __device__ __forceinline__ int kmaj_off16(int r, int k, int R) {
    return ((k >> 3) * (R >> 3) + (r >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// D (TMEM) (+)= A * B with BF16 operands (kind::f16); issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate ? 1u : 0u));
}

// D (TMEM) (+)= A * B; issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate ? 1u : 0u));
}

// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival on the mbarrier (release at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(mbar)) : "memory");
}

// waits for the phase of the given parity to complete; gives up after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    }
    return done != 0;
}

// TMEM allocation of `ncols` columns (power of two, >= 32) by one whole warp; the address
// is written to shared memory
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit columns of the TMEM lane (32 * quarter + lane) of this warp
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// x = hi + lo for the 3xTF32 products hi*hi + hi*lo + lo*hi: hi is x with the 13 low
// mantissa bits cleared (exactly representable in TF32), lo = x - hi is exact in FP32;
// the kind::tf32 MMA reads only the top 10 mantissa bits of lo, which leaves an error of
// about 2^-21 |x| per operand.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

}  // namespace tc
}  // namespace dh2
