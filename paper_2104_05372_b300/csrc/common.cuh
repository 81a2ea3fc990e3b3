// Shared device helpers for libgpa (sm_103a): status reporting, bounded
// mbarrier waits, 1-D bulk (TMA) copies, warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gpa.h"

namespace gpa {

// Every bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 1000ull * 1000ull * 1000ull;  // 1 s

__device__ __forceinline__ void report(int32_t* status, int code) {
    if (status) atomicOr(status, code);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete. Gives up after
// limit_ns (kWaitLimitNs unless a caller asks for less), reports
// GPA_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* status,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            report(status, GPA_ERR_TIMEOUT);
            return false;
        }
    }
}

// Warp-uniform variant: every lane polls, the warp leaves together (all lanes
// see the phase complete, or all give up after limit_ns by lane 0's clock).
// Use it wherever the warp runs .sync.aligned instructions or __syncwarp next.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, int32_t* status,
                                               unsigned long long limit_ns = kWaitLimitNs) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;  // already complete: no clock read
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        int late = (globaltimer_ns() - t0 > limit_ns) ? 1 : 0;
        late = __shfl_sync(0xffffffffu, late, 0);
        if (late) {
            if ((threadIdx.x & 31) == 0) report(status, GPA_ERR_TIMEOUT);
            return false;
        }
    }
}

// 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled on `bar` as transaction bytes. dst, src 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- cp.async (global -> shared without registers) ---------------------------
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Wait until at most N of this thread's most recent commit groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- warp helpers ----------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int32_t warp_sum(int32_t v) { return __reduce_add_sync(0xffffffffu, v); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Online log-sum-exp state (running max m, scaled sum l).
struct Lse {
    float m, l;
    __device__ __forceinline__ void init() {
        m = -INFINITY;
        l = 0.f;
    }
    __device__ __forceinline__ void add(float v) {
        if (v > m) {
            l = (m == -INFINITY ? 0.f : l * expf(m - v)) + 1.f;
            m = v;
        } else {
            l += expf(v - m);
        }
    }
    __device__ __forceinline__ void merge(float m2, float l2) {
        if (m2 == -INFINITY) return;
        if (m == -INFINITY) {
            m = m2;
            l = l2;
            return;
        }
        const float mx = fmaxf(m, m2);
        l = l * expf(m - mx) + l2 * expf(m2 - mx);
        m = mx;
    }
    __device__ __forceinline__ float value() const { return m + logf(l); }
};

}  // namespace gpa

// Host-side launch check: returns GPA_ERR_CUDA if the last launch failed.
#define GPA_LAUNCH_CHECK()                                   \
    do {                                                     \
        if (cudaPeekAtLastError() != cudaSuccess) {          \
            (void)cudaGetLastError();                        \
            return GPA_ERR_CUDA;                             \
        }                                                    \
    } while (0)
