// Many forwards of one transformed population in a single launch, for input
// sequences known in advance (a fixed evaluation set, or observations that
// do not depend on the previous step's outputs).  Section 3.3 transforms a
// network once and calculates many times; here each group also keeps its
// genome's record in shared memory across the steps, so the record is read
// from memory once per launch instead of once per step, and there is one
// launch instead of one per step.  Same node rule, order and aggregation as
// every other forward (bit-identical outputs).
//
// GB300 mapping: the work items and shared-memory layout of the forward
// kernel; per step, the next step's inputs are loaded into registers before
// the current step's level walk, so their memory latency overlaps the walk.
#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"
#include "neat_item.cuh"

namespace neat {
namespace {

__device__ unsigned int g_fused_error;

struct FusedArgs {
    ForwardArgs f;
    int steps;
    long long in_step_stride;    // floats between consecutive steps' inputs
    long long out_step_stride;   // floats between consecutive steps' outputs
};

template <bool T1>
__global__ void __launch_bounds__(1024, 1) fused_kernel(const FusedArgs fa)
{
    const ForwardArgs &a = fa.f;
    extern __shared__ __align__(16) uint4 smem[];
    const int G = a.group, lgG = ilog2(G);
    const int gpb = blockDim.x >> lgG;
    const int gi = threadIdx.x >> lgG;
    const int lane = threadIdx.x & (G - 1);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int *flags = reinterpret_cast<int *>(bars + gpb);
    uint4 *srec = smem + forward_header_words(gpb) + (size_t)gi * (a.rec_words + a.val_floats / 4);
    float *v = reinterpret_cast<float *>(srec + a.rec_words);

    const long item = (long)blockIdx.x * gpb + gi;
    if (item >= (long)a.pop * a.tiles) return;
    const int k = (int)(item / a.tiles);
    const int g = a.order ? __ldg(a.order + k) : k;
    const int b0 = (int)(item - (long)k * a.tiles) * a.tile;
    const int bt = T1 ? 1 : min(a.tile, a.B - b0);
    const int lgT = T1 ? 0 : ilog2(a.tile);
    const uint8_t *grec = a.rec + (size_t)g * a.stride;
    const uint32_t bar = smem_addr(bars + gi);
    uint32_t bytes = (uint32_t)a.rec_copy_bytes;
    if (bytes == 0) bytes = min(align16(__ldg(reinterpret_cast<const uint32_t *>(grec) + 4)),
                                (uint32_t)a.rec_words * 16u);
    if (lane == 0) {
        flags[gi] = 0;
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(srec), grec, bytes, bar);
    }
    const size_t xoff = ((size_t)g * a.B + b0) * a.I, yoff = ((size_t)g * a.B + b0) * a.O;
    const int nx = bt * a.I;
    float xr[kInputRegs];
#pragma unroll
    for (int q = 0; q < kInputRegs; ++q) {
        const int i = lane + q * G;
        xr[q] = (fa.steps > 0 && i < nx) ? __ldg(a.x + xoff + i) : 0.0f;
    }
    group_sync(G, gi);
    if (!mbar_wait(bar, 0)) flags[gi] = 1;
    group_sync(G, gi);
    const uint4 h0 = srec[0], h1 = srec[1];
    // a failed copy or an invalid genome writes NaN at every step but stays
    // in the step loop, so that the groups sharing its warp keep in step
    const bool dead = flags[gi] || (h0.z & NEAT_G_ERROR_MASK);
    if (flags[gi]) {
        if (lane == 0) atomicOr(&g_fused_error, kErrWaitExpired);
        mbar_wait(bar, 0);
    }
    // groups smaller than a warp: the lanes of this warp's groups that have
    // work items meet at the end of every step, so the genomes sharing a warp
    // run each step's walk together instead of drifting into divergent paths
    unsigned wmask = 0xffffffffu;
    if (G < 32) {
        wmask = 0u;
        const int g0 = (threadIdx.x & ~31) >> lgG;                 // first group of this warp
        for (int j = 0; j < 32 / G; ++j)
            if (g0 + j < gpb && (long)blockIdx.x * gpb + g0 + j < (long)a.pop * a.tiles)
                wmask |= ((1u << G) - 1u) << (j * G);
    }
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
    const bool col_ok = T1 || (lane & (a.tile - 1)) < bt;
    const bool fast = (h0.w & 0xffffu) == kTraitsSumTanh;
    for (int s = 0; s < fa.steps; ++s) {
        const float *xb = a.x + (size_t)s * fa.in_step_stride + xoff;
        float *yb = a.y + (size_t)s * fa.out_step_stride + yoff;
        if (dead) {
            for (int i = lane; i < bt * a.O; i += G) yb[i] = __int_as_float(0x7fc00000);
            if (G < 32) __syncwarp(wmask);
            continue;
        }
        // this step's inputs (prefetched) into the value tile
#pragma unroll
        for (int q = 0; q < kInputRegs; ++q) {
            const int i = lane + q * G;
            if (i < nx) {
                if (T1) v[io[i]] = xr[q];
                else {
                    const int b = i / a.I, j = i - b * a.I;
                    v[((int)io[j] << lgT) + b] = xr[q];
                }
            }
        }
        for (int i = lane + kInputRegs * G; i < nx; i += G) {
            if (T1) v[io[i]] = __ldg(xb + i);
            else {
                const int b = i / a.I, j = i - b * a.I;
                v[((int)io[j] << lgT) + b] = __ldg(xb + i);
            }
        }
        // the next step's inputs, in flight during this step's walk
        if (s + 1 < fa.steps) {
#pragma unroll
            for (int q = 0; q < kInputRegs; ++q) {
                const int i = lane + q * G;
                if (i < nx) xr[q] = __ldg(xb + fa.in_step_stride + i);
            }
        }
        group_sync(G, gi);
        if (fast) walk_levels<T1, true>(srec, v, G, gi, lane, lgT, a.lg_split, col_ok);
        else walk_levels<T1, false>(srec, v, G, gi, lane, lgT, a.lg_split, col_ok);
        for (int i = lane; i < bt * a.O; i += G) {
            if (T1) yb[i] = v[io[a.I + i]];
            else {
                const int b = i / a.O, j = i - b * a.O;
                yb[i] = v[((int)io[a.I + j] << lgT) + b];
            }
        }
        // outputs read before the next walk overwrites them; warp lockstep
        if (G < 32) __syncwarp(wmask);
        else group_sync(G, gi);
    }
}

}  // namespace

int read_fused_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_fused_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "fused error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_fused_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "fused error word: clear");
    }
    return NEAT_OK;
}

}  // namespace neat

using namespace neat;

extern "C" int neat_forward_fused(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                  int64_t in_step_stride, int32_t batch, float *outputs_dev, int64_t out_step_stride,
                                  int32_t steps, const neat_launch *launch_host, void *stream)
{
    TraceRange trace_range("neat_forward_fused");
    clear_error();
    if (steps < 0) return invalid("neat_forward_fused: steps < 0");
    if (steps == 0) return NEAT_OK;
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch(pop, d, batch, &L);
        if (rc) return rc;
    }
    ForwardArgs f;
    int rc = make_forward_args(transformed_dev, pop, d, inputs_dev, batch, outputs_dev, L, &f);
    if (rc) return rc;
    const long items = (long)f.pop * f.tiles;
    if (items == 0) return NEAT_OK;
    if (in_step_stride < (int64_t)pop * batch * d.num_inputs || out_step_stride < (int64_t)pop * batch * d.num_outputs)
        return invalid("neat_forward_fused: step strides smaller than one step");
    FusedArgs fa;
    fa.f = f;
    fa.steps = steps;
    fa.in_step_stride = in_step_stride;
    fa.out_step_stride = out_step_stride;
    const size_t per_group = (size_t)f.rec_words * 16 + (size_t)f.val_floats * 4;
    const size_t smem = per_group * L.groups_per_block + 16u * (size_t)forward_header_words(L.groups_per_block);
    if (smem > kMaxSmemPerBlock)
        return invalid("neat_forward_fused: shared memory per block exceeds 227 KB; lower tile or groups_per_block");
    auto kern = (L.tile == 1) ? fused_kernel<true> : fused_kernel<false>;
    rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_forward_fused: shared memory per block");
    if (rc) return rc;
    const long grid = (items + L.groups_per_block - 1) / L.groups_per_block;
    if (grid > 0x7fffffffL) return invalid("neat_forward_fused: too many work items");
    kern<<<(unsigned)grid, L.group * L.groups_per_block, smem, as_stream(stream)>>>(fa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_fused: launch");
    return NEAT_OK;
}
