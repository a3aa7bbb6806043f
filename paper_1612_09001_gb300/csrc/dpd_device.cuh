// Device-side building blocks shared by the libdpd kernels: shared-memory
// barriers, one-dimensional bulk copies (TMA engine), bounded waits and the
// per-handle error word.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpd_internal.h"

namespace dpd {

// Wall-clock limit for any single barrier wait inside a kernel.  A correct
// kernel waits microseconds; this only bounds a hang.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// FP32 (hi, lo) pairs: hi + lo carries a sum to about 2^-48 relative accuracy
// with FP32 arithmetic only.  two_sum_acc adds x to the pair, keeping the
// rounding error of the addition exactly (Knuth's two-sum) and summing it into
// lo; pair_add adds two pairs and renormalises the result.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    const float t = hi + x, z = t - hi;
    lo += (hi - (t - z)) + (x - z);
    hi = t;
}

__device__ __forceinline__ float2 pair_add(float2 a, float2 b)
{
    const float t = a.x + b.x, z = t - a.x;
    const float e = ((a.x - (t - z)) + (b.x - z)) + (a.y + b.y);
    const float s = t + e;
    return make_float2(s, e - (s - t));
}

__device__ __forceinline__ float2 shfl_xor_pair(float2 v, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete.  Gives up after
// kWaitLimitNs, records kFlagTimeout in *status and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
            atomicOr(status, kFlagTimeout);
            return false;
        }
    }
}

// One-dimensional bulk copy global -> shared through the TMA engine; completion
// is signalled on `bar` as transaction bytes.  src and dst 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Same, with an L2 eviction-priority hint for data read exactly once.
__device__ __forceinline__ void bulk_copy_g2s_stream(uint32_t dst, const void *src, uint32_t bytes,
                                                     uint32_t bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Programmatic dependent launch.  grid_dep_wait: block until the grids this one
// depends on (earlier work in the stream) have completed and their memory
// operations are visible; returns at once when there are none.
// grid_dep_launch_dependents: allow the next grid in the stream to start
// launching (its CTAs still wait in their own grid_dep_wait).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Streaming (evict-first) 16-byte global store.
__device__ __forceinline__ void st_stream_f4(float4 *p, float4 v)
{
    asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

}  // namespace dpd
