// Device-side helpers shared by the kernels of libneat.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace neat {

// tanh of a node, from the identity tanh(z) = 1 - 2 / (exp(2z) + 1) with
// the hardware base-2 exponential and reciprocal approximations (PTX
// ex2.approx, rcp.approx): z * 2/ln 2, one exponential, one add, one
// reciprocal, one multiply-add, a shorter dependent chain than an accurate
// library tanh.  The absolute error stays below about 4e-7 (relative errors
// of ex2 and rcp near 2^-22, times |2 r| <= 2), far inside the float
// tolerance; both limits and NaN pass through the identity.
__device__ __forceinline__ float node_tanh(float z)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z * 2.88539008177792681472f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
    return fmaf(-2.0f, r, 1.0f);
}

// Node activation of the node rule (Section 3.3, f_n); ids as in neat.h.
// tanh as above; the others with CUDA's accurate single-precision functions.
__device__ __forceinline__ float activate(uint32_t act, float z)
{
    switch (act) {
    case 1: return node_tanh(z);
    case 2: return 1.0f / (1.0f + expf(-z));
    case 3: return fmaxf(z, 0.0f);
    case 4: return sinf(z);
    case 5: return expf(-(z * z));
    case 6: return fabsf(z);
    default: return z;
    }
}

// Programmatic dependent launch controls (PTX griddepcontrol).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Hint: bring the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// A node or connection key: an exact integer in [0, 2^24).
__device__ __forceinline__ bool is_key(float k)
{
    return !isnan(k) && k >= 0.0f && k < 16777216.0f && floorf(k) == k;
}

// In-place ascending bitonic sort of n2 (a power of two) keys in shared
// memory; every thread of the block must call it.
template <typename T>
__device__ void bitonic_sort(T *a, int n2)
{
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const T x = a[i], y = a[ixj];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Read-only 16-byte global load.
__device__ __forceinline__ uint4 ldg16(const uint4 *p) { return __ldg(p); }

}  // namespace neat

namespace neat {

// ---- shared-memory mbarrier + TMA bulk copy (global -> shared), sm_90+ PTX

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Retire an mbarrier whose phases are complete before its memory is re-initialised.
__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// completing on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `phase` of `bar`: false once about kWaitLimitNs of
// wall time have passed without the phase completing.  Each try suspends
// the thread for up to kWaitHintNs instead of spinning.
constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s
constexpr uint32_t kWaitHintNs = 2000;
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t phase, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0;; ++i) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(bar), "r"(phase), "r"(kWaitHintNs) : "memory");
        if (ok) return true;
        if ((i & 63u) == 0) {
            const uint64_t t = global_ns();
            if (i == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) { return mbar_wait_for(bar, phase, kWaitLimitNs); }

// Order earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bits of a translation unit's device error word.
constexpr unsigned int kErrWaitExpired = 1u;

}  // namespace neat
