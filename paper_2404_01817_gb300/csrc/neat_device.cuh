// Device-side helpers shared by the kernels of libneat.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace neat {

// Node activation of the node rule (Section 3.3, f_n); ids as in neat.h.
// CUDA's accurate single-precision functions, no fast-math approximations.
__device__ __forceinline__ float activate(uint32_t act, float z)
{
    switch (act) {
    case 1: return tanhf(z);
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
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

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

// Bounded wait for phase `phase` of `bar`; false if the bound ran out.
constexpr uint32_t kWaitIters = 1u << 22;
constexpr uint32_t kWaitHintNs = 2000;   // suspend up to this long per try instead of spinning
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (uint32_t i = 0; i < kWaitIters; ++i) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(bar), "r"(phase), "r"(kWaitHintNs) : "memory");
        if (ok) return true;
    }
    return false;
}

// Bits of a translation unit's device error word.
constexpr unsigned int kErrWaitExpired = 1u;

}  // namespace neat
