// HyperNEAT substrate evaluation (the CPPN / HyperNEAT extensions of Section
// 4.3): the weight blocks written by neat_cppn_query define a layered
// network over the substrate grid, evaluated here for a batch of input
// vectors per genome: layer 0 = the R = res^2 inputs, layer l+1 node
// t = act(sum_s W_l[s][t] v_l[s]) (no bias; hidden_act inside, output_act on
// the last layer).
//
// GB300 mapping: for the control setting (one or a few input vectors per
// genome) this is a batched matrix-vector product whose cost is reading the
// fp32 weight blocks once from HBM (2 x 256 KB per genome at 16 x 16), so it
// runs on the FP32 pipes at the bandwidth roofline rather than on tensor
// cores, which would also round the weights below the float tolerance.  One
// block per (genome, batch chunk of NB vectors): each thread owns VEC
// adjacent target columns of one slice of the sources (the slices are
// equal runs of consecutive rows), keeps NB x VEC accumulators in registers,
// and the slices are summed in a fixed order through shared memory, where
// the layer's values also stay, so the result is a function of the inputs
// alone.  The weights stream through shared memory by TMA bulk copies of
// whole source rows (substrate_tma_kernel, tiles of up to 4 vectors, near
// the HBM roofline at one vector per genome); shapes it cannot take (R not a
// multiple of 4) use per-thread VEC-wide read-only loads (substrate_kernel).
// Both accumulate compensated dot products and give the same bits.
#include <algorithm>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"

namespace neat {
namespace {

constexpr int kSubThreads = 256;

struct SubArgs {
    const float *w;        // [pop][L-1][R][R]
    const float *x;        // [pop][B][R]
    float *y;              // [pop][B][R]
    int R, L, B;
    int hidden_act, output_act;
    int groups;            // slices of the source range (threads per column group)
    int cols;              // column groups per pass (cols * groups <= threads)
    int stage_rows;        // bulk-copy path: source rows per shared-memory stage
};

__device__ unsigned int g_substrate_error;

// Compensated dot products.  Error-free transformations of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005):
// TwoSum (after Knuth) and TwoProduct by one FMA.  dot2_step adds x*w to the
// pair (s, c), s the rounded running sum and c the sum of the rounding
// errors; s + c is as accurate as the dot product in twice the working
// precision, so sums of large weights stay within the float tolerance.  The
// _rn intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void dot2_step(float &s, float &c, float x, float w)
{
    const float p = __fmul_rn(x, w);
    const float pe = __fmaf_rn(x, w, -p);                  // x*w - p, exactly
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

// The slices' (s, c) pairs added in slice order, rounded once at the end.
__device__ __forceinline__ float combine_slices(const float *ps, const float *pc, size_t stride, int groups)
{
    float S = ps[0], C = pc[0];
    for (int j = 1; j < groups; ++j) {
        float t, e;
        two_sum(S, ps[(size_t)j * stride], t, e);
        S = t;
        C = __fadd_rn(C, __fadd_rn(e, pc[(size_t)j * stride]));
    }
    return __fadd_rn(S, C);
}

template <int VEC>
struct VecT;
template <>
struct VecT<1> {
    using T = float;
    static __device__ __forceinline__ float get(const float &v, int) { return v; }
};
template <>
struct VecT<4> {
    using T = float4;
    static __device__ __forceinline__ float get(const float4 &v, int i)
    {
        return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    }
};

template <int NB, int VEC>
__global__ void __launch_bounds__(kSubThreads) substrate_kernel(const SubArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const int R = a.R;
    float *cur = sm;                       // [NB][R]
    float *nxt = cur + NB * R;             // [NB][R]
    float *ps = nxt + NB * R;              // [groups][NB][R] slice sums
    float *pc = ps + (size_t)a.groups * NB * R;   // [groups][NB][R] their rounding errors
    const int g = blockIdx.x, b0 = blockIdx.y * NB;
    const int nb = min(NB, a.B - b0);
    const int tid = threadIdx.x;
    const float *xg = a.x + ((size_t)g * a.B + b0) * R;
    for (int i = tid; i < NB * R; i += kSubThreads) cur[i] = (i < nb * R) ? __ldg(xg + i) : 0.0f;
    __syncthreads();
    const int ncols = R / VEC;                              // column groups in a row
    const int slice = (R + a.groups - 1) / a.groups;        // sources per slice
    const int col_in_pass = tid % a.cols, grp = tid / a.cols;
    using V = typename VecT<VEC>::T;
    for (int l = 0; l + 1 < a.L; ++l) {
        const float *Wl = a.w + ((size_t)g * (a.L - 1) + l) * (size_t)R * R;
        const int act = (l + 2 == a.L) ? a.output_act : a.hidden_act;
        for (int c0 = 0; c0 < ncols; c0 += a.cols) {
            const int c = c0 + col_in_pass;
            if (grp < a.groups && c < ncols) {
                float as[NB][VEC], ac[NB][VEC];
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) as[b][v] = ac[b][v] = 0.0f;
                const int s0 = grp * slice, s1 = min(R, s0 + slice);
                const V *col = reinterpret_cast<const V *>(Wl) + c;
#pragma unroll 8
                for (int s = s0; s < s1; ++s) {
                    const V wv = __ldg(col + (size_t)s * ncols);
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const float xv = cur[b * R + s];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) dot2_step(as[b][v], ac[b][v], xv, VecT<VEC>::get(wv, v));
                    }
                }
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        ps[((size_t)grp * NB + b) * R + c * VEC + v] = as[b][v];
                        pc[((size_t)grp * NB + b) * R + c * VEC + v] = ac[b][v];
                    }
            }
            __syncthreads();
            // sum the slices in order, apply the activation
            for (int i = tid; i < NB * a.cols * VEC; i += kSubThreads) {
                const int b = i / (a.cols * VEC), t = c0 * VEC + i % (a.cols * VEC);
                if (t >= R) continue;
                nxt[b * R + t] = activate((uint32_t)act, combine_slices(ps + (size_t)b * R + t, pc + (size_t)b * R + t,
                                                                         (size_t)NB * R, a.groups));
            }
            __syncthreads();
        }
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    float *yg = a.y + ((size_t)g * a.B + b0) * R;
    for (int i = tid; i < nb * R; i += kSubThreads) yg[i] = cur[i];
}

// The same layers with the weights streamed through shared memory by bulk
// copies (TMA): each stage is `stage_rows` consecutive source rows, which
// are contiguous in the source-major block; two stages are in flight, each
// completing on its own mbarrier (bounded waits).  The sources are split
// into `groups` slices (equal runs of consecutive rows) and a stage holds
// the next stage_rows / groups rows of every slice, one bulk copy each, so
// every thread works on every stage: thread (col, grp) owns the 4 target
// columns col*4 .. col*4+3 and adds the rows of slice grp, in increasing s,
// for its NB vectors; the slices' partial sums are added in order through
// shared memory.  The operations and their order are those of
// substrate_kernel, so the bits are the same.  Needs R % 4 == 0, R / 4
// dividing the block, and the per-slice stage rows dividing the slice.
template <int NB>
__global__ void __launch_bounds__(kSubThreads) substrate_tma_kernel(const SubArgs a)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int failed;
    const int R = a.R, rows = a.stage_rows;
    float *stage = sm;                                      // [2][rows][R]
    float *cur = stage + 2 * (size_t)rows * R;              // [NB][R]
    float *nxt = cur + NB * R;                              // [NB][R]
    float *ps = nxt + NB * R;                               // [groups][NB][R] slice sums
    float *pc = ps + (size_t)(kSubThreads / (R / 4)) * NB * R;   // [groups][NB][R] their rounding errors
    const int g = blockIdx.x, b0 = blockIdx.y * NB;
    const int nb = min(NB, a.B - b0);
    const int tid = threadIdx.x;
    const int ncols = R / 4, groups = kSubThreads / ncols;
    const int slen = R / groups;                            // sources per slice (R % groups == 0)
    const int col = tid % ncols, grp = tid / ncols;
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
    const int rps = rows / groups;                          // rows of each slice per stage
    const uint32_t slice_bytes = (uint32_t)rps * (uint32_t)R * 4u;
    const uint32_t stage_bytes = slice_bytes * (uint32_t)groups;
    const int nstages = slen / rps;
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        failed = 0;
    }
    const float *xg = a.x + ((size_t)g * a.B + b0) * R;
    for (int i = tid; i < NB * R; i += kSubThreads) cur[i] = (i < nb * R) ? __ldg(xg + i) : 0.0f;
    __syncthreads();
    // copies issued into and completions seen on each buffer (every thread
    // counts; thread 0 issues)
    uint32_t issued0 = 0u, issued1 = 0u, seen0 = 0u, seen1 = 0u;
    // stage st of layer block Wl: rows st*rps .. st*rps+rps-1 of every slice
    // (one bulk copy per slice), slice j's rows at buffer rows j*rps ..
    auto issue = [&](int buf, const float *Wl, int st) {
        if (tid == 0) {
            fence_proxy_async_smem();                       // the buffer's earlier reads come first
            const uint32_t bar = buf ? bar1 : bar0;
            mbar_arrive_expect_tx(bar, stage_bytes);
            for (int j = 0; j < groups; ++j)
                bulk_g2s(smem_addr(stage + (size_t)buf * rows * R + (size_t)j * rps * R),
                         Wl + ((size_t)j * slen + (size_t)st * rps) * R, slice_bytes, bar);
        }
        if (buf) ++issued1; else ++issued0;
    };
    for (int l = 0; l + 1 < a.L && !failed; ++l) {
        const float *Wl = a.w + ((size_t)g * (a.L - 1) + l) * (size_t)R * R;
        const int act = (l + 2 == a.L) ? a.output_act : a.hidden_act;
        for (int st = 0; st < 2 && st < nstages; ++st) issue(st, Wl, st);
        float as[NB][4], ac[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int v = 0; v < 4; ++v) as[b][v] = ac[b][v] = 0.0f;
        for (int st = 0; st < nstages; ++st) {
            const int buf = st & 1;
            if (mbar_wait(buf ? bar1 : bar0, (buf ? seen1 : seen0) & 1u)) {
                if (buf) ++seen1; else ++seen0;
            } else {
                failed = 1;
            }
            // this thread's rows: sources grp*slen + st*rps .. + rps - 1
            const float4 *W4 = reinterpret_cast<const float4 *>(stage + (size_t)buf * rows * R +
                                                                (size_t)grp * rps * R);
            const float *xs = cur + grp * slen + st * rps;
            for (int r = 0; r < rps; ++r) {
                const float4 w = W4[(size_t)r * ncols + col];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const float xv = xs[b * R + r];
                    dot2_step(as[b][0], ac[b][0], xv, w.x);
                    dot2_step(as[b][1], ac[b][1], xv, w.y);
                    dot2_step(as[b][2], ac[b][2], xv, w.z);
                    dot2_step(as[b][3], ac[b][3], xv, w.w);
                }
            }
            __syncthreads();                                // every thread is done with the buffer
            if (failed) break;
            if (st + 2 < nstages) issue(buf, Wl, st + 2);
        }
        if (failed) break;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                ps[((size_t)grp * NB + b) * R + col * 4 + v] = as[b][v];
                pc[((size_t)grp * NB + b) * R + col * 4 + v] = ac[b][v];
            }
        __syncthreads();
        for (int i = tid; i < NB * R; i += kSubThreads) {
            const int b = i / R, t = i - b * R;
            nxt[i] = activate((uint32_t)act, combine_slices(ps + (size_t)b * R + t, pc + (size_t)b * R + t,
                                                             (size_t)NB * R, groups));
        }
        __syncthreads();
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    float *yg = a.y + ((size_t)g * a.B + b0) * R;
    if (failed) {
        // a stage did not arrive in time: let every copy in flight land
        // before the block's shared memory is released, then report
        for (; seen0 < issued0; ++seen0) mbar_wait(bar0, seen0 & 1u);
        for (; seen1 < issued1; ++seen1) mbar_wait(bar1, seen1 & 1u);
        if (tid == 0) atomicOr(&g_substrate_error, kErrWaitExpired);
        for (int i = tid; i < nb * R; i += kSubThreads) yg[i] = __int_as_float(0x7fc00000);
        return;
    }
    for (int i = tid; i < nb * R; i += kSubThreads) yg[i] = cur[i];
}

template <int NB, int VEC>
int launch_sub(const SubArgs &a, int pop, cudaStream_t s)
{
    const size_t smem = sizeof(float) * ((size_t)2 * NB * a.R + 2 * (size_t)a.groups * NB * a.R);
    auto kern = substrate_kernel<NB, VEC>;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_substrate_forward: shared memory");
    if (rc) return rc;
    const dim3 grid((unsigned)pop, (unsigned)((a.B + NB - 1) / NB));
    kern<<<grid, kSubThreads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_substrate_forward: launch");
    return NEAT_OK;
}

template <int NB>
int launch_tma(const SubArgs &a, int pop, cudaStream_t s)
{
    const size_t smem = sizeof(float) * (2 * (size_t)a.stage_rows * a.R + 2 * (size_t)NB * a.R +
                                         2 * (size_t)(kSubThreads / (a.R / 4)) * NB * a.R);
    auto kern = substrate_tma_kernel<NB>;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_substrate_forward: shared memory");
    if (rc) return rc;
    const dim3 grid((unsigned)pop, (unsigned)((a.B + NB - 1) / NB));
    kern<<<grid, kSubThreads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_substrate_forward: launch");
    return NEAT_OK;
}

template <int VEC>
int launch_vec(const SubArgs &a, int pop, int nb, cudaStream_t s)
{
    switch (nb) {
    case 1: return launch_sub<1, VEC>(a, pop, s);
    case 2: return launch_sub<2, VEC>(a, pop, s);
    case 4: return launch_sub<4, VEC>(a, pop, s);
    case 8: return launch_sub<8, VEC>(a, pop, s);
    default: return launch_sub<16, VEC>(a, pop, s);
    }
}

}  // namespace
}  // namespace neat

using namespace neat;

extern "C" int neat_substrate_forward(const float *weights_dev, int32_t pop, neat_substrate sub, const float *inputs_dev,
                                      int32_t batch, int32_t hidden_act, int32_t output_act, float *outputs_dev,
                                      void *stream)
{
    TraceRange trace_range("neat_substrate_forward");
    clear_error();
    if (sub.resolution < 2 || sub.resolution > 181 || sub.layers < 2)
        return invalid("neat_substrate_forward: substrate resolution must be in 2..181 and layers >= 2");
    if (pop < 0 || batch < 0) return invalid("neat_substrate_forward: sizes must be >= 0");
    if (hidden_act < 0 || hidden_act > 6 || output_act < 0 || output_act > 6)
        return invalid("neat_substrate_forward: activation ids are 0..6");
    if (pop == 0 || batch == 0) return NEAT_OK;
    if (!weights_dev || !inputs_dev || !outputs_dev) return invalid("neat_substrate_forward: null pointer");
    if ((batch + 15) / 16 > 65535) return invalid("neat_substrate_forward: batch too large");
    SubArgs a;
    a.w = weights_dev;
    a.x = inputs_dev;
    a.y = outputs_dev;
    a.R = sub.resolution * sub.resolution;
    a.L = sub.layers;
    a.B = batch;
    a.hidden_act = hidden_act;
    a.output_act = output_act;
    const bool vec4 = (a.R % 4 == 0) && (reinterpret_cast<uintptr_t>(weights_dev) % 16 == 0);
    const int ncols = vec4 ? a.R / 4 : a.R;
    a.cols = std::min(ncols, kSubThreads);
    a.groups = std::max(1, kSubThreads / a.cols);
    int nb = 1;
    while (nb < batch && nb < 16) nb <<= 1;
    // shared memory: two value tiles and the slice partials
    while (sizeof(float) * ((size_t)2 * nb * a.R + 2 * (size_t)a.groups * nb * a.R) > 200u * 1024u && a.groups > 1)
        a.groups >>= 1;
    while (sizeof(float) * ((size_t)2 * nb * a.R + 2 * (size_t)a.groups * nb * a.R) > 200u * 1024u && nb > 1)
        nb >>= 1;
    if (sizeof(float) * ((size_t)4 * nb * a.R) > 200u * 1024u)
        return invalid("neat_substrate_forward: substrate too large for one block");
    // bulk-copy path: 32 KB stages of whole source rows, tiles of up to 4
    // vectors (with the compensated sums, larger batches are bound by
    // arithmetic, not by streaming the weights once per tile), when R / 4
    // divides the block and the stages, values and partial sums fit 112 KB
    // (two or more blocks per SM).  Both kernels split the sources into the
    // same slices, so their results are identical
    if (vec4 && kSubThreads % (a.R / 4) == 0) {
        const int groups = kSubThreads / (a.R / 4);
        // stage rows: about 32 KB, a multiple of the slices, each slice's
        // share dividing the slice
        const int slen = a.R / groups;
        int rows = std::max(groups, std::min(a.R, (32 * 1024) / (4 * a.R)));
        while (rows > groups && (rows % groups || slen % (rows / groups))) --rows;
        const int nbt = std::min(nb, 4);
        const size_t smem = sizeof(float) * (2 * (size_t)rows * a.R + 2 * (size_t)nbt * a.R +
                                             2 * (size_t)groups * nbt * a.R);
        // the same slices as substrate_kernel: groups = kSubThreads / (R / 4)
        // there too while its shared memory needs no fewer (true for nb <= 4)
        if (a.R % groups == 0 && rows % groups == 0 && slen % (rows / groups) == 0 && groups == a.groups &&
            smem <= 112u * 1024u) {
            a.stage_rows = rows;
            switch (nbt) {
            case 1: return launch_tma<1>(a, pop, as_stream(stream));
            case 2: return launch_tma<2>(a, pop, as_stream(stream));
            default: return launch_tma<4>(a, pop, as_stream(stream));
            }
        }
    }
    return vec4 ? launch_vec<4>(a, pop, nb, as_stream(stream)) : launch_vec<1>(a, pop, nb, as_stream(stream));
}

namespace neat {
int read_substrate_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_substrate_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "substrate error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_substrate_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "substrate error word: clear");
    }
    return NEAT_OK;
}
}  // namespace neat
