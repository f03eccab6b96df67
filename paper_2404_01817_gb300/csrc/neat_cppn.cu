// CPPN query of a HyperNEAT substrate (the CPPN / HyperNEAT extensions of
// Section 4.3): every CPPN genome is evaluated at every (source, target) node
// pair of consecutive substrate layers, with inputs (x_s, y_s, x_t, y_t, 1),
// and its output becomes the connection weight, zeroed when |w| < threshold.
//
// Substrate: `layers` layers of res x res nodes on the grid -1 + 2 i / (res-1)
// of [-1,1]^2, node index = res * iy + ix.  Output layout
// weights[genome][block][source][target], block l joining layer l to l+1.
//
// GB300 mapping: a block of 256 threads takes (genome, chunk of queries),
// bulk-copies the genome's record into shared memory once (TMA + mbarrier),
// and each thread evaluates its own queries one after another in its own
// column of the value tile v[position][256]: node and edge reads are the same
// for the whole warp (broadcasts), value reads hit 32 distinct banks, and no
// barrier is needed between nodes.  The work is bound by FP32 and SFU issue
// (edges and transcendentals per query), not by memory: the only traffic is
// the 4-byte output per query.
#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"
#include "neat_item.cuh"

namespace neat {
namespace {

constexpr int kCppnThreads = 256;
constexpr int kCppnQueriesPerThread = 16;

struct CppnArgs {
    const uint8_t *rec;
    size_t stride;
    float *out;
    int pop, N;
    int res, layers;
    long queries;            // per genome
    int chunks;              // blocks per genome
    float threshold;
    int rec_words;           // 16-byte words of the record region
    int use_xy;              // node coordinate table in shared memory (res^2 <= 4096)
};

__device__ unsigned int g_cppn_error;

// QPT: queries per thread evaluated together (1, or 2 in columns tid and
// tid + 256 of a 512-column tile, sharing each node's entry, dispatch and
// edge entries); every query's value is bit-equal either way.
template <int QPT>
__global__ void __launch_bounds__(kCppnThreads) cppn_kernel(const CppnArgs a)
{
    extern __shared__ __align__(16) uint4 smem[];
    __shared__ uint64_t bar_mem;
    __shared__ float coord[NEAT_MAX_NODES];
    const int tid = threadIdx.x;
    const int g = (int)(blockIdx.x / a.chunks);
    const long q0 = (long)(blockIdx.x - (long)g * a.chunks) * (kCppnThreads * kCppnQueriesPerThread);
    uint4 *srec = smem;
    float *v = reinterpret_cast<float *>(smem + a.rec_words);
    float2 *nodexy = reinterpret_cast<float2 *>(v + (size_t)a.N * kCppnThreads * QPT);   // (x, y) of node i
    const uint32_t bar = smem_addr(&bar_mem);
    const uint8_t *grec = a.rec + (size_t)g * a.stride;
    if (tid == 0) {
        const uint32_t bytes = min(align16(__ldg(reinterpret_cast<const uint32_t *>(grec) + 4)),
                                   (uint32_t)a.rec_words * 16u);
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(srec), grec, bytes, bar);
    }
    for (int i = tid; i < a.res; i += kCppnThreads)
        coord[i] = (float)(-1.0 + 2.0 * (double)i / (double)(a.res - 1));
    __syncthreads();
    if (a.use_xy)
        for (int i = tid; i < a.res * a.res; i += kCppnThreads) nodexy[i] = make_float2(coord[i % a.res], coord[i / a.res]);
    __shared__ int failed;
    if (tid == 0) failed = 0;
    __syncthreads();
    if (!mbar_wait(bar, 0)) failed = 1;
    __syncthreads();
    float *out = a.out + (size_t)g * a.queries;
    const long qend = min(a.queries, q0 + (long)kCppnThreads * kCppnQueriesPerThread);
    if (failed) {
        if (tid == 0) atomicOr(&g_cppn_error, kErrWaitExpired);
        mbar_wait(bar, 0);
        for (long q = q0 + tid; q < qend; q += kCppnThreads) out[q] = __int_as_float(0x7fc00000);
        return;
    }
    const uint4 h0 = srec[0], h1 = srec[1];
    if (h0.z & NEAT_G_ERROR_MASK) {
        for (long q = q0 + tid; q < qend; q += kCppnThreads) out[q] = __int_as_float(0x7fc00000);
        return;
    }
    const int n_nodes = (int)(h0.x & 0xffffu);
    const int first = (int)(h0.w >> 16);               // leading input positions need no evaluation
    const bool sum_only = ((h0.w >> 8) & 0xffu) == 0u;  // uniform sum aggregation
    const uint4 *nodes = srec + 2;
    const uint2 *edges = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(srec) + h1.y);
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
    constexpr int lgT = QPT == 2 ? 9 : 8;               // value slot = (p << lgT) + column
    static_assert((1 << lgT) == kCppnThreads * QPT, "tile of the CPPN value array");
    const int pin0 = io[0], pin1 = io[1], pin2 = io[2], pin3 = io[3], pin4 = io[4], pout = io[5];
    const int per_block = a.res * a.res * a.res * a.res;
    const int rr = a.res * a.res;
    // (source, target) of this thread's first query; later queries advance
    // it by kCppnThreads without dividing
    int r = (int)((q0 + tid) % per_block);
    int s = r / rr, t = r - s * rr;
    auto advance = [&](int &r_, int &s_, int &t_) {
        r_ += kCppnThreads;
        t_ += kCppnThreads;
        if (r_ >= per_block) {                         // into the next layer block
            r_ -= per_block;
            s_ = r_ / rr;
            t_ = r_ - s_ * rr;
        } else {
            while (t_ >= rr) {
                t_ -= rr;
                ++s_;
            }
        }
    };
    auto put_inputs = [&](int s_, int t_, int col) {
        float2 ps, pt;
        if (a.use_xy) {
            ps = nodexy[s_];
            pt = nodexy[t_];
        } else {
            ps = make_float2(coord[s_ % a.res], coord[s_ / a.res]);
            pt = make_float2(coord[t_ % a.res], coord[t_ / a.res]);
        }
        v[(pin0 << lgT) + col] = ps.x;
        v[(pin1 << lgT) + col] = ps.y;
        v[(pin2 << lgT) + col] = pt.x;
        v[(pin3 << lgT) + col] = pt.y;
        v[(pin4 << lgT) + col] = 1.0f;
    };
    for (long q = q0 + tid; q < qend; q += (long)kCppnThreads * QPT) {
        put_inputs(s, t, tid);
        if (QPT == 2) {
            int r2 = r, s2 = s, t2 = t;
            advance(r2, s2, t2);                       // the thread's next query, in column tid + 256
            put_inputs(s2, t2, tid + kCppnThreads);
            if (sum_only) {
                for (int p = first; p < n_nodes; ++p)
                    eval_node_sum_by_count2(nodes[p], edges, v, p, lgT, tid, kCppnThreads);
            } else {
                for (int p = first; p < n_nodes; ++p) {
                    eval_node_tile<false>(nodes[p], edges, v, p, lgT, tid);
                    eval_node_tile<false>(nodes[p], edges, v, p, lgT, tid + kCppnThreads);
                }
            }
            const float w = v[(pout << lgT) + tid];
            out[q] = (fabsf(w) < a.threshold) ? 0.0f : w;
            if (q + kCppnThreads < qend) {
                const float w2 = v[(pout << lgT) + tid + kCppnThreads];
                out[q + kCppnThreads] = (fabsf(w2) < a.threshold) ? 0.0f : w2;
            }
            r = r2;
            s = s2;
            t = t2;
            advance(r, s, t);
        } else {
            if (sum_only)
                for (int p = first; p < n_nodes; ++p) eval_node_sum_by_count<false>(nodes[p], edges, v, p, lgT, tid);
            else
                for (int p = first; p < n_nodes; ++p) eval_node_tile<false>(nodes[p], edges, v, p, lgT, tid);
            const float w = v[(pout << lgT) + tid];
            out[q] = (fabsf(w) < a.threshold) ? 0.0f : w;
            advance(r, s, t);
        }
    }
}

}  // namespace
}  // namespace neat

using namespace neat;

extern "C" int neat_cppn_query(const void *transformed_dev, int32_t pop, neat_dims d, neat_substrate sub,
                               float threshold, float *weights_dev, void *stream)
{
    TraceRange trace_range("neat_cppn_query");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_cppn_query: invalid dims");
    if (d.num_inputs != 5 || d.num_outputs != 1)
        return invalid("neat_cppn_query: a CPPN has 5 inputs (x_s, y_s, x_t, y_t, 1) and 1 output");
    if (sub.resolution < 2 || sub.resolution > 181 || sub.layers < 2)
        return invalid("neat_cppn_query: substrate resolution must be in 2..181 and layers >= 2");
    if (pop < 0) return invalid("neat_cppn_query: pop < 0");
    if (pop == 0) return NEAT_OK;
    if (!transformed_dev || !weights_dev) return invalid("neat_cppn_query: null pointer");
    if (reinterpret_cast<uintptr_t>(transformed_dev) & 15u)
        return invalid("neat_cppn_query: transformed must be 16-byte aligned");
    CppnArgs a;
    a.rec = static_cast<const uint8_t *>(transformed_dev);
    a.stride = record_stride(d);
    a.out = weights_dev;
    a.pop = pop;
    a.N = d.max_nodes;
    a.res = sub.resolution;
    a.layers = sub.layers;
    const long r2 = (long)sub.resolution * sub.resolution;
    a.queries = (long)(sub.layers - 1) * r2 * r2;
    const long per_block = (long)kCppnThreads * kCppnQueriesPerThread;
    a.chunks = (int)((a.queries + per_block - 1) / per_block);
    a.threshold = threshold;
    a.rec_words = (int)(record_max_bytes(5, 1, d.max_nodes, d.max_conns) / 16);
    a.use_xy = (r2 <= 4096) ? 1 : 0;
    // two queries per thread where the doubled value tile fits, else one
    auto smem_for = [&](int qpt) {
        return (size_t)a.rec_words * 16 + 4u * (size_t)d.max_nodes * kCppnThreads * qpt +
               (a.use_xy ? 8u * (size_t)r2 : 0u);
    };
    const int qpt = smem_for(2) <= 200u * 1024u ? 2 : 1;
    const size_t smem = smem_for(qpt);
    if (smem > 200u * 1024u) return invalid("neat_cppn_query: genome too large for one block (max_nodes <= 160)");
    const long blocks = (long)pop * a.chunks;
    if (blocks > 0x7fffffffL) return invalid("neat_cppn_query: too many queries");
    auto kern = qpt == 2 ? cppn_kernel<2> : cppn_kernel<1>;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_cppn_query: shared memory per block");
    if (rc) return rc;
    kern<<<(unsigned)blocks, kCppnThreads, smem, as_stream(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_cppn_query: launch");
    return NEAT_OK;
}

namespace neat {
int read_cppn_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_cppn_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "cppn error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_cppn_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "cppn error word: clear");
    }
    return NEAT_OK;
}
}  // namespace neat
