// Recurrent networks: K synchronous iterations of the node rule over every
// non-input node (the paper divides networks into feedforward and recurrent
// ones, Section 3.3, and names network_type among its hyperparameters; it
// gives no recurrent algorithm, so this library fixes one): input nodes hold
// their inputs, every other node starts at 0, and iteration k computes all
// nodes from iterate k-1,
//   v_k[n] = act_n(bias_n + response_n * agg_n(w_c v_{k-1}[src_c])).
// Records come from neat_transform_recurrent: positions in row order (no
// topological sort: cycles are allowed), the same incoming edge lists.
//
// GB300 mapping: as the feedforward kernel (one group per (genome, tile),
// one bulk copy of the record into shared memory issued before the
// programmatic-dependence wait), with two value tiles that swap roles every
// iteration; every node of an iteration is independent, so all of the
// group's threads work on one iteration at a time and one group barrier
// separates iterations.
#include <algorithm>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"
#include "neat_item.cuh"

namespace neat {
namespace {

__device__ unsigned int g_rnn_error;

template <bool T1, bool FAST>
__device__ __forceinline__ float *rnn_iterate(const uint4 *srec, float *cur, float *nxt, int G, int gi, int lane,
                                              int lgT, bool col_ok, int K)
{
    const uint4 h0 = srec[0], h1 = srec[1];
    const int n = (int)(h0.x & 0xffffu);
    const int first = (int)(h0.w >> 16);
    const uint4 *nodes = srec + 2;
    const uint2 *edges = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(srec) + h1.y);
    const int col = T1 ? 0 : (lane & ((1 << lgT) - 1));
    const int sub = T1 ? lane : (lane >> lgT);
    const int nsub = T1 ? G : (G >> lgT);
    for (int k = 0; k < K; ++k) {
        if (col_ok) {
            for (int p = first + sub; p < n; p += nsub) {
                const uint4 ne = nodes[p];
                const uint32_t act = ne.w & 0xffu;
                if (act == kInputAct) continue;
                const uint32_t agg = FAST ? kAggSum : ((ne.w >> 8) & 0xffu);
                const uint32_t ec = ne.z >> 16;
                const float a = partials<T1, FAST>(agg, edges + (ne.z & 0xffffu), ec, cur, lgT, col, 0, 4);
                nxt[vslot<T1>(p, lgT, col)] =
                    FAST ? node_tanh(fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)))
                         : node_output(ne, agg, act, ec, a);
            }
        }
        group_sync(G, gi);
        float *t = cur;
        cur = nxt;
        nxt = t;
    }
    return cur;
}

struct RnnArgs {
    ForwardArgs f;      // val_floats holds both value tiles
    int iterations;
};

template <bool PDL, bool T1>
__global__ void __launch_bounds__(1024, 1) rnn_kernel(const RnnArgs ra)
{
    const ForwardArgs &a = ra.f;
    extern __shared__ __align__(16) uint4 smem[];
    const int G = a.group, lgG = ilog2(G);
    const int gpb = blockDim.x >> lgG;
    const int gi = threadIdx.x >> lgG;
    const int lane = threadIdx.x & (G - 1);
    // [mbarriers][flags][group 0: record | values | values][group 1: ...]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int *flags = reinterpret_cast<int *>(bars + gpb);
    uint4 *srec = smem + forward_header_words(gpb) + (size_t)gi * (a.rec_words + a.val_floats / 4);
    const int tilefl = a.val_floats / 2;                 // floats of one value tile (a multiple of 4)
    float *v0 = reinterpret_cast<float *>(srec + a.rec_words);
    float *v1 = v0 + tilefl;

    const long item = (long)blockIdx.x * gpb + gi;
    if (item >= (long)a.pop * a.tiles) return;
    const int k = (int)(item / a.tiles);
    const int g = a.order ? __ldg(a.order + k) : k;
    const int b0 = (int)(item - (long)k * a.tiles) * a.tile;
    const int bt = T1 ? 1 : min(a.tile, a.B - b0);
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
    for (int i = lane; i < tilefl; i += G) v0[i] = 0.0f;  // non-input nodes start at 0
    // records do not depend on the previous kernel in the stream; inputs and
    // outputs do, so they are touched only after the dependence wait
    if constexpr (PDL) {
        pdl_wait();
        pdl_trigger();
    }
    const float *xb = a.x + ((size_t)g * a.B + b0) * a.I;
    float *yb = a.y + ((size_t)g * a.B + b0) * a.O;
    group_sync(G, gi);
    if (!mbar_wait(bar, 0)) flags[gi] = 1;
    group_sync(G, gi);
    if (flags[gi]) {
        if (lane == 0) atomicOr(&g_rnn_error, kErrWaitExpired);
        mbar_wait(bar, 0);
        for (int i = lane; i < bt * a.O; i += G) yb[i] = __int_as_float(0x7fc00000);
        return;
    }
    const uint4 h0 = srec[0], h1 = srec[1];
    if (h0.z & NEAT_G_ERROR_MASK) {
        for (int i = lane; i < bt * a.O; i += G) yb[i] = __int_as_float(0x7fc00000);
        return;
    }
    const int lgT = T1 ? 0 : ilog2(a.tile);
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
    for (int i = lane; i < bt * a.I; i += G) {           // inputs, held in both tiles
        const int b = T1 ? 0 : i / a.I, j = T1 ? i : i - b * a.I;
        const int slot = T1 ? (int)io[j] : (((int)io[j] << lgT) + b);
        const float x = __ldg(xb + i);
        v0[slot] = x;
        v1[slot] = x;
    }
    group_sync(G, gi);
    const bool col_ok = T1 || (lane & (a.tile - 1)) < bt;
    const float *fin = ((h0.w & 0xffffu) == kTraitsSumTanh)
                           ? rnn_iterate<T1, true>(srec, v0, v1, G, gi, lane, lgT, col_ok, ra.iterations)
                           : rnn_iterate<T1, false>(srec, v0, v1, G, gi, lane, lgT, col_ok, ra.iterations);
    for (int i = lane; i < bt * a.O; i += G) {
        if (T1) yb[i] = fin[io[a.I + i]];
        else {
            const int b = i / a.O, j = i - b * a.O;
            yb[i] = fin[((int)io[a.I + j] << lgT) + b];
        }
    }
}

using RnnFn = void (*)(RnnArgs);

RnnFn pick_rnn(bool pdl, bool t1)
{
    if (pdl) return t1 ? rnn_kernel<true, true> : rnn_kernel<true, false>;
    return t1 ? rnn_kernel<false, true> : rnn_kernel<false, false>;
}

size_t rnn_per_group(const ForwardArgs &f) { return (size_t)f.rec_words * 16 + (size_t)f.val_floats * 4; }

}  // namespace

int read_rnn_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_rnn_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "recurrent error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_rnn_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "recurrent error word: clear");
    }
    return NEAT_OK;
}

}  // namespace neat

using namespace neat;

extern "C" int neat_default_launch_recurrent(int32_t pop, neat_dims d, int32_t batch, neat_launch *out)
{
    if (!out) return invalid("neat_default_launch_recurrent: null pointer");
    neat_launch L;
    int rc = neat_default_launch(pop, d, batch, &L);   // tile as for the feedforward kernel
    if (rc) return rc;
    if (L.tile == 1) {
        // every non-input node is evaluated in every iteration: one thread
        // per non-input node (8..128 threads per genome)
        int g = 8;
        while (g < d.max_nodes - d.num_inputs && g < 128) g <<= 1;
        L.group = g;
    } else {
        // two value tiles (current and next iteration) beside the record
        const size_t rec = record_max_bytes(d.num_inputs, d.num_outputs, d.max_nodes, d.max_conns);
        while (L.tile > 1 && rec + 8u * (size_t)d.max_nodes * L.tile > kMaxGroupSmem) {
            L.tile >>= 1;
            L.group >>= 1;
        }
    }
    const size_t per_group = record_max_bytes(d.num_inputs, d.num_outputs, d.max_nodes, d.max_conns) +
                             8u * (size_t)((d.max_nodes * L.tile + 3) & ~3);
    const long items = (long)std::max(pop, 1) * ((std::max(batch, 1) + L.tile - 1) / L.tile);
    L.groups_per_block = groups_per_block_for(items, L.group, per_group);
    *out = L;
    return NEAT_OK;
}

extern "C" int neat_forward_recurrent_ex(const void *transformed_dev, int32_t pop, neat_dims d,
                                         const float *inputs_dev, int32_t batch, int32_t iterations,
                                         float *outputs_dev, const neat_launch *launch_host, void *stream)
{
    TraceRange trace_range("neat_forward_recurrent");
    clear_error();
    if (iterations < 0) return invalid("neat_forward_recurrent: iterations < 0");
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch_recurrent(pop, d, batch, &L);
        if (rc) return rc;
    }
    if (L.split != 1) return invalid("neat_forward_recurrent: split must be 1");
    ForwardArgs f;
    int rc = make_forward_args(transformed_dev, pop, d, inputs_dev, batch, outputs_dev, L, &f);
    if (rc) return rc;
    const long items = (long)f.pop * f.tiles;
    if (items == 0) return NEAT_OK;
    f.val_floats = 2 * ((d.max_nodes * L.tile + 3) & ~3);          // two value tiles
    const size_t smem = rnn_per_group(f) * L.groups_per_block + 16u * (size_t)forward_header_words(L.groups_per_block);
    if (smem > 227u * 1024u)
        return invalid("neat_forward_recurrent: shared memory per block exceeds 227 KB; lower tile or groups_per_block");
    const long grid = (items + L.groups_per_block - 1) / L.groups_per_block;
    if (grid > 0x7fffffffL) return invalid("neat_forward_recurrent: too many work items");
    RnnArgs ra;
    ra.f = f;
    ra.iterations = iterations;
    RnnFn kern = pick_rnn(L.pdl != 0, L.tile == 1);
    rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_forward_recurrent: shared memory per block");
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(L.group * L.groups_per_block));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = as_stream(stream);
    cudaLaunchAttribute attr[1];
    if (L.pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ra);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_recurrent: launch");
    return NEAT_OK;
}

extern "C" int neat_forward_recurrent(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                      int32_t batch, int32_t iterations, float *outputs_dev, void *stream)
{
    return neat_forward_recurrent_ex(transformed_dev, pop, d, inputs_dev, batch, iterations, outputs_dev, nullptr,
                                     stream);
}
