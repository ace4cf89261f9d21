// Device helpers shared by the tcgen05 kernels (translate_tc.cu, leaf_tc.cu):
// shared-memory matrix descriptors for the no-swizzle K-major layout, bounded
// mbarrier waits, tensor-memory loads and group-wide decisions.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace fda_tc {

constexpr int KC = 32;                // real K per stage (two MMA k-steps of 16)
constexpr int ABYTES = 128 * KC * 2;  // one bf16 operand panel stage (hi or lo, 128 rows): 8 KB
constexpr long long SPIN = 20000000;  // bounded mbarrier polls

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;   // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                        // descriptor version
    return d;
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long long it = 0; it < SPIN && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
    return done != 0;
}

// byte offset of element (row, k) inside a [rows x 32] K-major bf16 stage
__device__ inline int core_off(int row, int k) { return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

__device__ inline bool mbar_wait_ab(uint32_t bar, uint32_t parity, const volatile int *abort)
{
    uint32_t done = 0;
    for (long long it = 0; it < SPIN; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    return false;
}

// 16 consecutive accumulator columns at each of two TMEM addresses (this
// warp's 32 lanes); the wait is inside the same statement, so the results
// cannot be used before the loads have completed
__device__ inline void tmem_ld16x2(uint32_t addr_a, uint32_t addr_b, uint32_t (&a)[16], uint32_t (&b)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
                   "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
                   "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
                   "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
                 : "r"(addr_a), "r"(addr_b));
}

// true on every thread of named barrier `id` (n threads) if pred holds on any
// of them: a group's decision to stop is taken together, so no thread is
// left waiting at a later barrier of the group
__device__ inline bool bar_any(int id, int n, bool pred)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)pred), "r"(id), "r"(n));
    return r != 0;
}


}  // namespace fda_tc
