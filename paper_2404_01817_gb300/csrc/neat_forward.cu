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
#include <mutex>
#include <unordered_map>

#include "neat_device.cuh"
#include "neat_internal.h"

namespace neat {
namespace {

template <int G>
__device__ __forceinline__ void group_sync(int gi)
{
    if constexpr (G < 32) {
        const unsigned base = (threadIdx.x & 31u) & ~(unsigned)(G - 1);
        __syncwarp(((1u << G) - 1u) << base);
    } else if constexpr (G == 32) {
        __syncwarp();
    } else {
        if (blockDim.x == G) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(gi + 1), "r"(G) : "memory");
    }
}

// One node of the node rule for column `col` of the tile.
__device__ __forceinline__ void eval_node(const uint4 ne, const uint2 *__restrict__ edges,
                                          float *__restrict__ v, int p, int T, int col)
{
    const uint32_t act = ne.w & 0xffu;
    if (act == kInputAct) return;
    const uint32_t agg = (ne.w >> 8) & 0xffu;
    const uint32_t eb = ne.z & 0xffffu, ec = ne.z >> 16;
    const uint2 *e = edges + eb;
    float acc = 0.0f;
    if (agg == 0u || agg == 3u) {
#pragma unroll 4
        for (uint32_t i = 0; i < ec; ++i) {
            const uint2 t = e[i];
            acc = fmaf(__uint_as_float(t.x), v[t.y * T + col], acc);
        }
        if (agg == 3u && ec) acc = acc / (float)ec;
    } else if (ec) {
        const uint2 t0 = e[0];
        acc = __uint_as_float(t0.x) * v[t0.y * T + col];
        if (agg == 1u) {
            for (uint32_t i = 1; i < ec; ++i) {
                const uint2 t = e[i];
                acc = acc * (__uint_as_float(t.x) * v[t.y * T + col]);
            }
        } else {
            for (uint32_t i = 1; i < ec; ++i) {
                const uint2 t = e[i];
                acc = fmaxf(acc, __uint_as_float(t.x) * v[t.y * T + col]);
            }
        }
    }
    const float z = fmaf(__uint_as_float(ne.y), acc, __uint_as_float(ne.x));
    v[p * T + col] = activate(act, z);
}

template <int G, bool PDL>
__global__ void __launch_bounds__(1024, 1) forward_kernel(const ForwardArgs a)
{
    extern __shared__ __align__(16) uint4 smem[];
    const int gpb = blockDim.x / G;
    const int gi = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    uint4 *srec = smem + (size_t)gi * (a.rec_words + a.val_floats / 4);
    float *v = reinterpret_cast<float *>(srec + a.rec_words);

    const long item = (long)blockIdx.x * gpb + gi;
    if (item >= (long)a.pop * a.tiles) return;
    const int g = (int)(item / a.tiles);
    const int b0 = (int)(item - (long)g * a.tiles) * a.tile;
    const int bt = min(a.tile, a.B - b0);

    // stage the record (independent of the previous kernel in the stream)
    const uint4 *grec = reinterpret_cast<const uint4 *>(a.rec + (size_t)g * a.stride);
    const uint4 h0 = ldg16(grec), h1 = ldg16(grec + 1);
    const int n_nodes = (int)h0.x, n_levels = (int)h0.y;
    const uint32_t status = h0.w;
    const int words = min((int)(h1.x >> 4), a.rec_words);
    for (int i = 2 + lane; i < words; i += G) srec[i] = ldg16(grec + i);

    if constexpr (PDL) {
        pdl_wait();
        pdl_trigger();
    }
    float *yb = a.y + ((size_t)g * a.B + b0) * a.O;
    if (status & NEAT_G_ERROR_MASK) {
        for (int i = lane; i < bt * a.O; i += G) yb[i] = __int_as_float(0x7fc00000);
        return;
    }
    group_sync<G>(gi);

    const int T = a.tile;
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
    const float *xb = a.x + ((size_t)g * a.B + b0) * a.I;
    for (int i = lane; i < bt * a.I; i += G) {
        const int b = i / a.I, j = i - b * a.I;
        v[io[j] * T + b] = __ldg(xb + i);
    }
    group_sync<G>(gi);

    const uint4 *nodes = srec + 2;
    const uint2 *edges = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(srec) + h1.y);
    const int col = lane % T;
    const int sub = lane / T;
    const int nsub = G / T;
    if (nsub == 1) {
        if (col < bt)
            for (int p = 0; p < n_nodes; ++p) eval_node(nodes[p], edges, v, p, T, col);
    } else {
        const uint16_t *lev = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.z);
        for (int l = 0; l < n_levels; ++l) {
            const int p1 = lev[l + 1];
            if (col < bt)
                for (int p = lev[l] + sub; p < p1; p += nsub) eval_node(nodes[p], edges, v, p, T, col);
            group_sync<G>(gi);
        }
    }
    group_sync<G>(gi);
    for (int i = lane; i < bt * a.O; i += G) {
        const int b = i / a.O, j = i - b * a.O;
        yb[i] = v[io[a.I + j] * T + b];
    }
}

using KernelFn = void (*)(ForwardArgs);

template <bool PDL>
KernelFn pick(int G)
{
    switch (G) {
    case 2: return forward_kernel<2, PDL>;
    case 4: return forward_kernel<4, PDL>;
    case 8: return forward_kernel<8, PDL>;
    case 16: return forward_kernel<16, PDL>;
    case 32: return forward_kernel<32, PDL>;
    case 64: return forward_kernel<64, PDL>;
    case 128: return forward_kernel<128, PDL>;
    case 256: return forward_kernel<256, PDL>;
    case 512: return forward_kernel<512, PDL>;
    }
    return nullptr;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

std::mutex g_attr_mu;
std::unordered_map<const void *, size_t> g_attr_bytes;   // dynamic smem already allowed per kernel

int ensure_smem(KernelFn f, size_t bytes)
{
    if (bytes <= 48 * 1024) return NEAT_OK;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &have = g_attr_bytes[reinterpret_cast<const void *>(f)];
    if (have >= bytes) return NEAT_OK;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "forward: cudaFuncSetAttribute");
    have = 227 * 1024;
    return NEAT_OK;
}

}  // namespace

int check_launch(const neat_launch &L)
{
    if (!pow2(L.group) || L.group < 2 || L.group > 512) return invalid("launch: group must be a power of two in 2..512");
    if (!pow2(L.tile) || L.tile > L.group) return invalid("launch: tile must be a power of two <= group");
    if (L.groups_per_block < 1 || L.group * L.groups_per_block > 1024)
        return invalid("launch: group * groups_per_block must be in 1..1024");
    if (L.group > 32 && L.groups_per_block > 15) return invalid("launch: at most 15 multi-warp groups per block");
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
    a.tiles = (batch + L.tile - 1) / L.tile;
    a.rec_words = (int)(record_max_bytes(a.I, a.O, a.N, d.max_conns) / 16);
    a.val_floats = (a.N * L.tile + 3) & ~3;
    *out = a;
    return NEAT_OK;
}

int launch_forward(const ForwardArgs &a, const neat_launch &L, cudaStream_t s)
{
    const long items = (long)a.pop * a.tiles;
    if (items == 0) return NEAT_OK;
    const size_t per_group = (size_t)a.rec_words * 16 + (size_t)a.val_floats * 4;
    const size_t smem = per_group * L.groups_per_block;
    if (smem > 227 * 1024) return invalid("forward: shared memory per block exceeds 227 KB; lower tile or groups_per_block");
    KernelFn f = L.pdl ? pick<true>(L.group) : pick<false>(L.group);
    if (!f) return invalid("forward: unsupported group size");
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

extern "C" int neat_default_launch(neat_dims d, int32_t batch, neat_launch *out)
{
    if (!out) return invalid("neat_default_launch: null pointer");
    if (!dims_ok(d)) return invalid("neat_default_launch: invalid dims");
    neat_launch L;
    const int N = d.max_nodes;
    if (batch <= 1) {
        L.tile = 1;
        L.group = N <= 64 ? 8 : (N <= 256 ? 16 : 32);
    } else {
        int t = 1;
        while (t < batch && t < 32) t <<= 1;
        L.tile = t;
        const int nsub = N <= 32 ? 1 : (N <= 128 ? 2 : (N <= 512 ? 4 : 8));
        L.group = t * nsub;
    }
    const size_t per_group = record_max_bytes(d.num_inputs, d.num_outputs, N, d.max_conns) +
                             4u * (size_t)((N * L.tile + 3) & ~3);
    int gpb = 256 / L.group;
    if (gpb < 1) gpb = 1;
    while (gpb > 1 && per_group * gpb > 96 * 1024) gpb >>= 1;
    if (L.group > 32 && gpb > 15) gpb = 8;
    L.groups_per_block = gpb;
    L.pdl = 0;
    *out = L;
    return NEAT_OK;
}

extern "C" int neat_forward_ex(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                               int32_t batch, float *outputs_dev, const neat_launch *launch_host, void *stream)
{
    clear_error();
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch(d, batch, &L);
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
           c.L.pdl == L.pdl;
}

extern "C" int neat_forward_steps(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                  int64_t in_step_stride, int32_t batch, float *outputs_dev,
                                  int64_t out_step_stride, int32_t steps, const neat_launch *launch_host,
                                  neat_steps_cache **cache, void *stream)
{
    clear_error();
    if (!cache) return invalid("neat_forward_steps: null cache pointer");
    if (steps < 0) return invalid("neat_forward_steps: steps < 0");
    if (steps == 0) return NEAT_OK;
    neat_launch L;
    if (launch_host) L = *launch_host;
    else {
        int rc = neat_default_launch(d, batch, &L);
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
