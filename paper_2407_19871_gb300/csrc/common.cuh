// Shared definitions of the CUDA path: parameters, NTT primes, PTX helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/locpir.h"

namespace lp {

// Ring degree and gadget shape this build supports (N = 1024, k = 1, lg = 3, Bgbit = 10,
// key switch t = 8 digits of basebit = 2).  The LWE dimension n is a runtime value.
constexpr int RING_N = 1024;
constexpr int LOG_N = 10;
constexpr int LG = 3;
constexpr int BGBIT = 10;
constexpr int ROWS = 2 * LG;           // TRGSW rows (k + 1) lg
constexpr int KS_T = 8;
constexpr int KS_BASEBIT = 2;
constexpr int KS_BASE = 1 << KS_BASEBIT;
constexpr int MAX_LWE_N = 639;        // key-switch rows of n + 1 words fit 640 words
constexpr int EXT_STRIDE = 1028;       // words per extracted N-LWE row (N + 1, padded to 16 B)

// Gadget offset: sum_p (Bg/2) 2^(32 - Bgbit p) + 2^(31 - Bgbit lg) (rounding + recentring).
constexpr uint32_t GADGET_OFF = (512u << 22) + (512u << 12) + (512u << 2) + 2u;
constexpr uint32_t T_EIGHTH = 0x20000000u;
constexpr uint32_t T_QUARTER = 0x40000000u;

// The two NTT primes: p = c 2^11 + 1 (so Z_p holds a primitive 2048-th root of unity) and
// 22 p < 2^32, so that a forward transform needs no reduction between its 10 stages (see
// ntt.cuh).  Their product (~2^55.1) exceeds twice the largest |sum_r sum_j d b| =
// 6 * 1024 * 512 * 2^31 ~ 2^52.6 of one external product (digits |d| <= 512, key words
// centred in [-2^31, 2^31)), so the centred CRT lift recovers every coefficient exactly.
constexpr uint32_t PRIME0 = 195198977u;  // 95312 * 2^11 + 1
constexpr uint32_t PRIME1 = 195188737u;  // 95307 * 2^11 + 1

// Number of per-lane twiddles of the five lane-dependent stages.
constexpr int LANE_TW = 31;

__device__ __forceinline__ uint32_t umin_u32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// Modulus switch of a torus32 word to Z_2N (2N = 2048), rounding half up: ((x + 2^20) mod 2^32) >> 21.
__device__ __forceinline__ uint16_t modswitch_2048(uint32_t x) { return (uint16_t)((x + (1u << 20)) >> 21); }

// ---------------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk async copy, timers.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// Every wait in this library gives up after this long and reports LP_ETIMEOUT.
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

// Bounded wait for the phase of the given parity; returns false after limit_ns or when
// *abort (a CTA-wide flag in shared memory) is raised by another warp.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort,
                                                  uint64_t limit_ns = WAIT_LIMIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*abort) return false;
            if (global_timer_ns() - t0 > limit_ns) return false;
        }
    }
}

// 1-D bulk copy global -> shared through the TMA engine, completing on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (and those it has
// observed) before its later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier over `threads` threads with an OR-reduction of pred across them.
__device__ __forceinline__ bool bar_red_or(int id, int threads, bool pred)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, "
        "po;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)pred), "r"(id), "r"(threads)
        : "memory");
    return out != 0u;
}

// Device error word bits (read by the host after synchronising).
constexpr int DEV_ERR_TIMEOUT = 1;
constexpr int DEV_ERR_BOUNDS = 2;

}  // namespace lp
