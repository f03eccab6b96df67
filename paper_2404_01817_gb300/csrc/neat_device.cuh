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
