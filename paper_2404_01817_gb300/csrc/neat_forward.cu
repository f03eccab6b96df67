// Calculation stage of tensorized NEAT inference (Section 3.3): node values
// are computed in topological order, v[k] = act(bias + response * agg(w v[src])).
//
// GB300 mapping.  A work item is (genome, tile of input vectors).  A group of
// G threads owns one item: the group stages the genome's packed record
// (neat.h) into shared memory with 16-byte read-only loads, scatters the
// item's inputs into a shared value tile v[position][tile], then walks the
// levels of the layered order.  Thread (col, sub) of the group computes column
// `col` of the nodes sub, sub + G/tile, ... of each level; the group
// synchronises between levels (warp-level when G <= 32).  When tile == G the
// levels need no barrier at all: each thread only reads its own column.
// Every node value is produced by one thread summing its incoming edges in
// the record's fixed order, so results are independent of the launch shape.
// The path is bound by on-chip latency and L2/HBM bandwidth, not by any
// dense contraction, so no tensor-core instruction is involved.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"
#include "neat_item.cuh"

namespace neat {
namespace {

// Library error word: a bounded wait in a forward kernel expired.
__device__ unsigned int g_forward_error;

// One work item per group of a.group threads.  T1: one input vector per
// genome (tile 1), the case of a control loop that steps every genome once.
template <bool PDL, bool T1>
__global__ void __launch_bounds__(1024, 1) forward_kernel(const ForwardArgs a)
{
    extern __shared__ __align__(16) uint4 smem[];
    const int G = a.group, lgG = ilog2(G);
    const int gpb = blockDim.x >> lgG;
    const int gi = threadIdx.x >> lgG;
    const int lane = threadIdx.x & (G - 1);
    // [mbarriers][flags][group 0: record | values][group 1: ...]
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

    // one bulk copy of the genome's record into shared memory; records do
    // not depend on the previous kernel in the stream, so it is issued
    // before the programmatic-dependence wait
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
    if constexpr (PDL) {
        // the item's inputs into L2 while the previous kernel finishes, so
        // that their loads after the wait are L2 hits.  Only a hint: L2 is
        // the point of coherence, so whatever the previous kernel writes to
        // them is what the loads after the wait see (no L1 line is filled)
        const char *xp = reinterpret_cast<const char *>(a.x + ((size_t)g * a.B + b0) * a.I);
        const int nbytes = bt * a.I * 4;
        for (int off = lane * 128; off < nbytes; off += G * 128) prefetch_l2(xp + off);
        if (lane == G - 1 && nbytes > 0) prefetch_l2(xp + nbytes - 1);
        pdl_wait();
        pdl_trigger();
    }
    run_item<T1>(srec, v, bar, flags + gi, G, gi, lane, a.x + ((size_t)g * a.B + b0) * a.I,
                 a.y + ((size_t)g * a.B + b0) * a.O, a.I, a.O, bt, a.tile, a.lg_split, &g_forward_error);
}

// One thread per genome (group 1, tile 1): each thread walks the positions
// of its own genome in order, so no barrier is needed between levels; the
// loops run warp-uniform trip counts (the warp's largest position count and,
// per position, its largest in-degree) with predicated edge loads, which
// keeps the warp converged while 32 genomes advance together.  Same
// aggregation order as every other shape (four partials, fixed tree).
constexpr int kSerialInputs = 32;

template <bool FAST>
__device__ __forceinline__ void walk_serial(const uint4 *srec, float *v, int npos, int first, unsigned mask)
{
    const uint4 h1 = srec[1];
    const uint4 *nodes = srec + 2;
    const uint2 *edges = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(srec) + h1.y);
    const int maxpos = (int)__reduce_max_sync(mask, (unsigned)max(npos, 0));
    for (int it = 0; it < maxpos; ++it) {
        const int p = first + it;
        uint4 ne = make_uint4(0u, 0u, 0u, (uint32_t)kInputAct);
        if (it < npos) ne = nodes[p];
        const uint32_t act = ne.w & 0xffu;
        const bool live = act != kInputAct;
        const uint32_t ec = live ? (ne.z >> 16) : 0u;
        const uint32_t agg = FAST ? kAggSum : ((ne.w >> 8) & 0xffu);
        const uint2 *e = edges + (ne.z & 0xffffu);
        const uint32_t ecmax = __reduce_max_sync(mask, ec);
        const float id = FAST ? 0.0f : agg_identity(agg);
        float q0 = id, q1 = id, q2 = id, q3 = id;
        for (uint32_t i = 0; i < ecmax; i += 4) {
            if (i < ec) { const uint2 t = e[i]; q0 = agg_step(agg, q0, __uint_as_float(t.x), v[t.y]); }
            if (i + 1 < ec) { const uint2 t = e[i + 1]; q1 = agg_step(agg, q1, __uint_as_float(t.x), v[t.y]); }
            if (i + 2 < ec) { const uint2 t = e[i + 2]; q2 = agg_step(agg, q2, __uint_as_float(t.x), v[t.y]); }
            if (i + 3 < ec) { const uint2 t = e[i + 3]; q3 = agg_step(agg, q3, __uint_as_float(t.x), v[t.y]); }
        }
        const float a = agg_combine(agg, agg_combine(agg, q0, q1), agg_combine(agg, q2, q3));
        if (live)
            v[p] = FAST ? node_tanh(fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)))
                        : node_output(ne, agg, act, ec, a);
    }
}

template <bool PDL>
__global__ void __launch_bounds__(1024, 1) forward_serial_kernel(const ForwardArgs a)
{
    extern __shared__ __align__(16) uint4 smem[];
    const int gpb = blockDim.x;
    const int gi = threadIdx.x;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint4 *srec = smem + forward_header_words(gpb) + (size_t)gi * (a.rec_words + a.val_floats / 4);
    float *v = reinterpret_cast<float *>(srec + a.rec_words);
    // lanes of this warp that exist in the block (the last warp may be partial)
    const int wbase = threadIdx.x & ~31;
    const int wn = min(32, gpb - wbase);
    const unsigned mask = wn == 32 ? 0xffffffffu : ((1u << wn) - 1u);

    const long k = (long)blockIdx.x * gpb + gi;
    const bool valid = k < a.pop;
    const long g = valid && a.order ? (long)__ldg(a.order + k) : k;
    const uint8_t *grec = a.rec + (size_t)(valid ? g : 0) * a.stride;
    const uint32_t bar = smem_addr(bars + gi);
    if (valid) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, (uint32_t)a.rec_copy_bytes);
        bulk_g2s(smem_addr(srec), grec, (uint32_t)a.rec_copy_bytes, bar);
    }
    if constexpr (PDL) {
        pdl_wait();
        pdl_trigger();
    }
    const float *xb = a.x + (size_t)(valid ? g : 0) * a.B * a.I;
    float xr[kSerialInputs];
#pragma unroll
    for (int k = 0; k < kSerialInputs; ++k) xr[k] = (valid && k < a.I) ? __ldg(xb + k) : 0.0f;
    bool ok = valid && mbar_wait(bar, 0);
    if (valid && !ok) {
        atomicOr(&g_forward_error, kErrWaitExpired);
        mbar_wait(bar, 0);
    }
    int npos = 0, first = 0;
    uint4 h0 = make_uint4(0u, 0u, 0u, 0u), h1 = h0;
    if (ok) {
        h0 = srec[0];
        h1 = srec[1];
        ok = (h0.z & NEAT_G_ERROR_MASK) == 0;
    }
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
    if (ok) {
        first = (int)(h0.w >> 16);
        npos = (int)(h0.x & 0xffffu) - first;
#pragma unroll
        for (int k = 0; k < kSerialInputs; ++k)
            if (k < a.I) v[io[k]] = xr[k];
        for (int k = kSerialInputs; k < a.I; ++k) v[io[k]] = __ldg(xb + k);
    }
    // every lane of the warp takes part in the walk's warp-uniform loop counts
    if ((h0.w & 0xffffu) == kTraitsSumTanh) walk_serial<true>(srec, v, npos, first, mask);
    else walk_serial<false>(srec, v, npos, first, mask);
    if (valid) {
        float *yb = a.y + (size_t)g * a.B * a.O;
        for (int j = 0; j < a.O; ++j) yb[j] = ok ? v[io[a.I + j]] : __int_as_float(0x7fc00000);
    }
}

using KernelFn = void (*)(ForwardArgs);

KernelFn pick(bool pdl, bool t1)
{
    if (pdl) return t1 ? forward_kernel<true, true> : forward_kernel<true, false>;
    return t1 ? forward_kernel<false, true> : forward_kernel<false, false>;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int ensure_smem(KernelFn f, size_t bytes)
{
    return allow_dynamic_smem(reinterpret_cast<const void *>(f), bytes, "forward: shared memory per block");
}

}  // namespace

// Records up to this size are copied whole (reserved size) in one bulk copy;
// larger ones copy only their used bytes after reading the header.
constexpr int kOnePieceRecordBytes = 8192;

int check_launch(const neat_launch &L)
{
    if (!pow2(L.group) || L.group > 1024) return invalid("launch: group must be a power of two in 1..1024");
    if (!pow2(L.tile) || L.tile > L.group) return invalid("launch: tile must be a power of two <= group");
    if (L.groups_per_block < 1 || L.group * L.groups_per_block > 1024)
        return invalid("launch: group * groups_per_block must be in 1..1024");
    if (L.group > 32 && L.groups_per_block > 15) return invalid("launch: at most 15 multi-warp groups per block");
    if (L.split != 1 && L.split != 2 && L.split != 4) return invalid("launch: split must be 1, 2 or 4");
    if (L.tile == 1 && L.split > L.group) return invalid("launch: split must not exceed group");
    return NEAT_OK;
}

int make_forward_args(const void *transformed, int32_t pop, const neat_dims &d, const float *inputs,
                      int32_t batch, float *outputs, const neat_launch &L, ForwardArgs *out)
{
    if (!dims_ok(d)) return invalid("forward: invalid dims");
    if (pop < 0 || batch < 0) return invalid("forward: pop and batch must be >= 0");
    if ((size_t)pop * batch > 0 && (!transformed || !outputs || (d.num_inputs > 0 && !inputs)))
        return invalid("forward: null pointer");
    if (reinterpret_cast<uintptr_t>(transformed) & 15u) return invalid("forward: transformed must be 16-byte aligned");
    int rc = check_launch(L);
    if (rc) return rc;
    ForwardArgs a;
    a.rec = static_cast<const uint8_t *>(transformed);
    a.stride = record_stride(d);
    a.x = inputs;
    a.y = outputs;
    a.pop = pop;
    a.I = d.num_inputs;
    a.O = d.num_outputs;
    a.N = d.max_nodes;
    a.B = batch;
    a.tile = L.tile;
    a.group = L.group;
    a.lg_split = L.split == 4 ? 2 : (L.split == 2 ? 1 : 0);
    a.tiles = (batch + L.tile - 1) / L.tile;
    a.rec_words = (int)(record_max_bytes(a.I, a.O, a.N, d.max_conns) / 16);
    a.val_floats = (a.N * L.tile + 3) & ~3;
    a.rec_copy_bytes = (a.rec_words * 16 <= kOnePieceRecordBytes) ? a.rec_words * 16 : 0;
    a.order = L.order_dev;
    *out = a;
    return NEAT_OK;
}

int launch_forward(const ForwardArgs &a, const neat_launch &L, cudaStream_t s)
{
    const long items = (long)a.pop * a.tiles;
    if (items == 0) return NEAT_OK;
    const size_t per_group = (size_t)a.rec_words * 16 + (size_t)a.val_floats * 4;
    const size_t smem = per_group * L.groups_per_block + 16u * (size_t)forward_header_words(L.groups_per_block);
    if (smem > 227 * 1024) return invalid("forward: shared memory per block exceeds 227 KB; lower tile or groups_per_block");
    KernelFn f = pick(L.pdl != 0, a.tile == 1);
    if (L.group == 1 && a.tile == 1) {
        // one thread per genome; the whole record is copied in one piece
        if (a.rec_copy_bytes == 0) return invalid("forward: group 1 needs records of at most 8 KB");
        f = L.pdl ? forward_serial_kernel<true> : forward_serial_kernel<false>;
    }
    int rc = ensure_smem(f, smem);
    if (rc) return rc;
    const long grid = (items + L.groups_per_block - 1) / L.groups_per_block;
    if (grid > 0x7fffffffL) return invalid("forward: too many work items");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(L.group * L.groups_per_block));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (L.pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, f, a);
    if (e != cudaSuccess) return cuda_fail(e, "forward: launch");
    return NEAT_OK;
}

}  // namespace neat

using namespace neat;

namespace neat {
namespace {

struct DeviceCaps {
    int sms = 152;
    int smem_per_sm = 233472;
};

DeviceCaps device_caps()
{
    static std::mutex mu;
    static std::unordered_map<int, DeviceCaps> cache;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DeviceCaps();
    }
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceCaps c;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) c.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0)
        c.smem_per_sm = v;
    cudaGetLastError();
    cache[dev] = c;
    return c;
}

// Groups per block: all items resident in as few waves as possible, with the
// items spread evenly over the SMs (fewest groups on the busiest SM).
int choose_groups_per_block(long items, int group, size_t per_group, const DeviceCaps &caps)
{
    const int max_gpb = group > 32 ? std::min(15, 1024 / group) : 1024 / group;
    int best = 1;
    long best_waves = -1, best_load = -1;
    for (int gpb = 1; gpb <= max_gpb; ++gpb) {
        const size_t smem = per_group * gpb + 16u * (size_t)forward_header_words(gpb);
        if (smem > 227u * 1024u) break;
        const int threads = group * gpb;
        const int warps = (threads + 31) / 32;
        int resident = (int)(caps.smem_per_sm / (smem + 1024));
        resident = std::min(resident, 2048 / (warps * 32));
        resident = std::min(resident, 65536 / (warps * 32 * 64));
        resident = std::min(resident, 32);
        if (resident < 1) continue;
        const long blocks = (items + gpb - 1) / gpb;
        const long slots = (long)caps.sms * resident;
        const long waves = (blocks + slots - 1) / slots;
        const long load = ((blocks + caps.sms - 1) / caps.sms) * gpb;
        // ties: the smallest block of at least 128 threads, so that blocks of
        // the next launch can start (programmatic dependent launch) while the
        // slowest blocks of this one finish
        const bool smaller_ok = threads >= 128 || group * best < 128;
        if (best_waves < 0 || waves < best_waves || (waves == best_waves && load < best_load) ||
            (waves == best_waves && load == best_load && smaller_ok && group * best < 128)) {
            best = gpb;
            best_waves = waves;
            best_load = load;
        }
    }
    return best;
}

}  // namespace
}  // namespace neat

namespace neat {
int groups_per_block_for(long items, int group, size_t per_group)
{
    return choose_groups_per_block(items, group, per_group, device_caps());
}
}  // namespace neat

extern "C" int neat_default_launch(int32_t pop, neat_dims d, int32_t batch, neat_launch *out)
{
    if (!out) return invalid("neat_default_launch: null pointer");
    if (!dims_ok(d)) return invalid("neat_default_launch: invalid dims");
    if (pop < 0 || batch < 0) return invalid("neat_default_launch: pop and batch must be >= 0");
    neat_launch L;
    const int N = d.max_nodes;
    L.split = 1;
    L.reserved = 0;
    L.order_dev = nullptr;
    if (batch <= 1) {
        L.tile = 1;
        L.group = N <= 64 ? 8 : (N <= 256 ? 16 : 32);
    } else {
        int t = 1;
        while (t < batch && t < 32) t <<= 1;
        L.tile = t;
        L.group = t * tile_row_threads(N);
        // a group's record and value tile must fit one block's shared memory
        const size_t rec = record_max_bytes(d.num_inputs, d.num_outputs, N, d.max_conns);
        while (L.tile > 1 && rec + 4u * (size_t)N * L.tile > kMaxGroupSmem) {
            L.tile >>= 1;
            L.group >>= 1;
        }
    }
    const size_t per_group = record_max_bytes(d.num_inputs, d.num_outputs, N, d.max_conns) +
                             4u * (size_t)((N * L.tile + 3) & ~3);
    const long items = (long)std::max(pop, 1) * ((std::max(batch, 1) + L.tile - 1) / L.tile);
    L.groups_per_block = choose_groups_per_block(items, L.group, per_group, device_caps());
    L.pdl = 0;
    *out = L;
    return NEAT_OK;
}

extern "C" int neat_forward_ex(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                               int32_t batch, float *outputs_dev, const neat_launch *launch_host, void *stream)
{
    TraceRange trace_range("neat_forward");
    clear_error();
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch(pop, d, batch, &L);
        if (rc) return rc;
    }
    ForwardArgs a;
    int rc = make_forward_args(transformed_dev, pop, d, inputs_dev, batch, outputs_dev, L, &a);
    if (rc) return rc;
    return launch_forward(a, L, as_stream(stream));
}

extern "C" int neat_forward(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                            int32_t batch, float *outputs_dev, void *stream)
{
    return neat_forward_ex(transformed_dev, pop, d, inputs_dev, batch, outputs_dev, nullptr, stream);
}

// ------------------------------------------------------ CUDA-graph step loop

struct neat_steps_cache {
    const void *rec = nullptr;
    int32_t pop = -1;
    neat_dims d = {};
    const float *x = nullptr;
    int64_t xs = 0;
    int32_t batch = -1;
    float *y = nullptr;
    int64_t ys = 0;
    int32_t steps = -1;
    neat_launch L = {};
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static bool same_key(const neat_steps_cache &c, const void *rec, int32_t pop, const neat_dims &d, const float *x,
                     int64_t xs, int32_t batch, float *y, int64_t ys, int32_t steps, const neat_launch &L)
{
    return c.exec && c.rec == rec && c.pop == pop && c.d.num_inputs == d.num_inputs &&
           c.d.num_outputs == d.num_outputs && c.d.max_nodes == d.max_nodes && c.d.max_conns == d.max_conns &&
           c.x == x && c.xs == xs && c.batch == batch && c.y == y && c.ys == ys && c.steps == steps &&
           c.L.group == L.group && c.L.tile == L.tile && c.L.groups_per_block == L.groups_per_block &&
           c.L.pdl == L.pdl && c.L.split == L.split && c.L.order_dev == L.order_dev;
}

extern "C" int neat_forward_steps(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                  int64_t in_step_stride, int32_t batch, float *outputs_dev,
                                  int64_t out_step_stride, int32_t steps, const neat_launch *launch_host,
                                  neat_steps_cache **cache, void *stream)
{
    TraceRange trace_range("neat_forward_steps");
    clear_error();
    if (!cache) return invalid("neat_forward_steps: null cache pointer");
    if (steps < 0) return invalid("neat_forward_steps: steps < 0");
    if (steps == 0) return NEAT_OK;
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch(pop, d, batch, &L);
        if (rc) return rc;
        L.pdl = 1;
    }
    ForwardArgs a;
    int rc = make_forward_args(transformed_dev, pop, d, inputs_dev, batch, outputs_dev, L, &a);
    if (rc) return rc;
    if (!*cache) *cache = new neat_steps_cache();
    neat_steps_cache &c = **cache;
    if (!same_key(c, transformed_dev, pop, d, inputs_dev, in_step_stride, batch, outputs_dev, out_step_stride,
                  steps, L)) {
        if (c.exec) {
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
        }
        cudaError_t e;
        if (!c.cap) {
            e = cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "neat_forward_steps: stream create");
        }
        e = cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "neat_forward_steps: begin capture");
        for (int s = 0; s < steps && rc == NEAT_OK; ++s) {
            ForwardArgs as = a;
            as.x = inputs_dev ? inputs_dev + (size_t)s * in_step_stride : nullptr;
            as.y = outputs_dev + (size_t)s * out_step_stride;
            neat_launch Ls = L;
            Ls.pdl = (s > 0) ? L.pdl : 0;   // the first step fully waits for prior work
            rc = launch_forward(as, Ls, c.cap);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c.cap, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "neat_forward_steps: end capture");
        e = cudaGraphInstantiate(&c.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c.exec = nullptr;
            return cuda_fail(e, "neat_forward_steps: instantiate");
        }
        c.rec = transformed_dev;
        c.pop = pop;
        c.d = d;
        c.x = inputs_dev;
        c.xs = in_step_stride;
        c.batch = batch;
        c.y = outputs_dev;
        c.ys = out_step_stride;
        c.steps = steps;
        c.L = L;
    }
    cudaError_t e = cudaGraphLaunch(c.exec, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_steps: graph launch");
    return NEAT_OK;
}

extern "C" void neat_steps_cache_destroy(neat_steps_cache *c)
{
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

extern "C" int neat_device_error(int32_t clear, uint32_t *out_host)
{
    clear_error();
    if (!out_host) return invalid("neat_device_error: null pointer");
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_forward_error, sizeof(v));
    if (e != cudaSuccess) return cuda_fail(e, "neat_device_error: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_forward_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "neat_device_error: clear");
    }
    unsigned int vp = 0, vc = 0, vr = 0, vd = 0, vf = 0, vs = 0, vl = 0;
    int rc = read_plan_error(&vp, clear);
    if (rc == NEAT_OK) rc = read_cppn_error(&vc, clear);
    if (rc == NEAT_OK) rc = read_rnn_error(&vr, clear);
    if (rc == NEAT_OK) rc = read_distance_error(&vd, clear);
    if (rc == NEAT_OK) rc = read_fused_error(&vf, clear);
    if (rc == NEAT_OK) rc = read_substrate_error(&vs, clear);
    if (rc == NEAT_OK) rc = read_lanes_error(&vl, clear);
    if (rc) return rc;
    *out_host = v | vp | vc | vr | vd | vf | vs | vl;
    return NEAT_OK;
}

// ------------------------------------------------------------ genome order

namespace neat {
namespace {

// Sort key of a genome for the forward order: level count, deepest first
// (counts above 63 share the first bin), then non-input nodes (the nodes
// after the leading inputs, in units of 2^shift so that 64 bins span
// max_nodes), most first.  Bin 0 comes first.  Recurrent records have one
// level each, so only the node count orders them.
constexpr int kSchedBins = 64 * 64;
__device__ __forceinline__ int schedule_bin(const uint8_t *rec, int shift)
{
    const uint32_t w0 = __ldg(reinterpret_cast<const uint32_t *>(rec));
    const uint32_t w3 = __ldg(reinterpret_cast<const uint32_t *>(rec) + 3);
    const int n = (int)(w0 & 0xffffu), lv = min((int)(w0 >> 16), 63);
    const int nonin = max(0, n - (int)min(w3 >> 16, (uint32_t)n));
    return (63 - lv) * 64 + (63 - min(nonin >> shift, 63));
}

// Counting sort of genomes by schedule_bin (one block of 1024 threads): a
// histogram, a block-wide exclusive scan (four bins per thread), placement.
__global__ void __launch_bounds__(1024) schedule_kernel(const uint8_t *rec, size_t stride, int pop, int shift,
                                                        int32_t *order)
{
    __shared__ int hist[kSchedBins];
    __shared__ int warp_tot[32];
    static_assert(kSchedBins == 4 * 1024, "four bins per thread");
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < kSchedBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int g = tid; g < pop; g += blockDim.x) atomicAdd(&hist[schedule_bin(rec + (size_t)g * stride, shift)], 1);
    __syncthreads();
    // exclusive scan: each thread its four consecutive bins, then the warps
    const int h0 = hist[4 * tid], h1 = hist[4 * tid + 1], h2 = hist[4 * tid + 2], h3 = hist[4 * tid + 3];
    const int mine = h0 + h1 + h2 + h3;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int t = warp_tot[lane];
        int wi = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - t;           // exclusive: warps before this one
    }
    __syncthreads();
    const int base = warp_tot[wid] + incl - mine;
    hist[4 * tid] = base;
    hist[4 * tid + 1] = base + h0;
    hist[4 * tid + 2] = base + h0 + h1;
    hist[4 * tid + 3] = base + h0 + h1 + h2;
    __syncthreads();
    for (int g = tid; g < pop; g += blockDim.x)
        order[atomicAdd(&hist[schedule_bin(rec + (size_t)g * stride, shift)], 1)] = g;
}

}  // namespace
}  // namespace neat

extern "C" int neat_schedule(const void *transformed_dev, int32_t pop, neat_dims d, int32_t *order_dev, void *stream)
{
    TraceRange trace_range("neat_schedule");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_schedule: invalid dims");
    if (pop < 0) return invalid("neat_schedule: pop < 0");
    if (pop == 0) return NEAT_OK;
    if (!transformed_dev || !order_dev) return invalid("neat_schedule: null pointer");
    int shift = 0;
    while ((d.max_nodes >> shift) > 64) ++shift;     // 64 node-count bins span max_nodes
    schedule_kernel<<<1, 1024, 0, as_stream(stream)>>>(static_cast<const uint8_t *>(transformed_dev),
                                                       record_stride(d), pop, shift, order_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_schedule: launch");
    return NEAT_OK;
}

// ------------------------------------------------ bounded-wait self-test

namespace neat {
namespace {

// One thread waits on an mbarrier that expects two arrivals but gets one:
// the phase never completes, the bounded wait gives up after limit_ns, the
// error word gets kErrWaitExpired and the kernel returns normally.
__global__ void selftest_wait_kernel(uint64_t limit_ns, unsigned int *result)
{
    __shared__ uint64_t bar_mem;
    const uint32_t bar = smem_addr(&bar_mem);
    mbar_init(bar, 2);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    const bool ok = mbar_wait_for(bar, 0, limit_ns);
    if (!ok) atomicOr(&g_forward_error, kErrWaitExpired);
    *result = ok ? 1u : 2u;
    mbar_inval(bar);
}

}  // namespace
}  // namespace neat

extern "C" int neat_selftest_bounded_wait(uint32_t limit_us, uint32_t *result_host)
{
    clear_error();
    if (!result_host) return invalid("neat_selftest_bounded_wait: null pointer");
    if (limit_us == 0 || limit_us > 2000000u) return invalid("neat_selftest_bounded_wait: limit in 1..2000000 us");
    unsigned int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "neat_selftest_bounded_wait: cudaMalloc");
    selftest_wait_kernel<<<1, 1>>>((uint64_t)limit_us * 1000ull, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned int r = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&r, d, sizeof(r), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "neat_selftest_bounded_wait");
    *result_host = r;
    return NEAT_OK;
}
