// Batched evaluation of several populations in one persistent launch per
// step (the data-parallel forward of Section 3.3 over uneven populations).
//
// Plan creation (host, once): every record header is read back, each
// population is split into size buckets by node count (powers of two from
// 16), and each bucket gets a launch shape: group size G, tile T and split
// (threads per node), chosen by a heuristic or timed on the plan's own data.
// A bucket's work is cut into block items of `gpc` work items each
// (gpc = threads per block / G); block items are numbered bucket by bucket,
// largest records first, so the most expensive items start first.
//
// Kernel (per step): persistent blocks pull block items from a per-step
// device counter.  For a block item every group of G threads bulk-copies its
// genome's record into its shared-memory region (TMA, completion on an
// mbarrier) and then runs the same item evaluation as the single-population
// kernel (run_item), so results match neat_forward bit for bit.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"
#include "neat_item.cuh"

namespace neat {
namespace {

__device__ unsigned int g_plan_error;

template <bool PDL>
__global__ void __launch_bounds__(1024, 1)
plan_kernel(const BucketDev *__restrict__ buckets, int nb, int item_lo, int item_hi, unsigned int *counter, int step)
{
    extern __shared__ __align__(16) uint4 smem[];
    __shared__ int s_ci;
    const int NT = blockDim.x;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int *flags = reinterpret_cast<int *>(bars + NT);
    uint4 *regions = smem + forward_header_words(NT);
    bool waited = !PDL;
    for (;;) {
        if (threadIdx.x == 0) s_ci = item_lo + (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int ci = s_ci;
        if (ci >= item_hi) break;
        int lo = 0, hi = nb - 1;                       // bucket holding block item ci
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (buckets[mid].cta_begin <= ci) lo = mid; else hi = mid - 1;
        }
        const BucketDev &d = buckets[lo];
        const int G = d.G, lgG = d.lgG;
        const int gi = threadIdx.x >> lgG;
        const int lane = threadIdx.x & (G - 1);
        const long item = (long)(ci - d.cta_begin) * d.gpc + gi;
        const bool active = gi < d.gpc && item < (long)d.n_genomes * d.tiles;
        uint4 *srec = regions + (size_t)gi * d.region_words;
        const uint32_t bar = smem_addr(bars + gi);
        int g = 0, b0 = 0;
        if (active) {
            const int k = (int)(item / d.tiles);
            g = __ldg(d.gidx + k);
            b0 = (int)(item - (long)k * d.tiles) * d.tile;
            if (lane == 0) {
                flags[gi] = 0;
                fence_proxy_async_smem();              // the region was read by the previous item
                mbar_init(bar, 1);
                mbar_arrive_expect_tx(bar, (uint32_t)d.rec_copy_bytes);
                bulk_g2s(smem_addr(srec), d.rec + (size_t)g * d.stride, (uint32_t)d.rec_copy_bytes, bar);
            }
        }
        if (PDL && !waited) {                          // inputs of this step may come from the previous kernel
            pdl_wait();
            pdl_trigger();
            waited = true;
        }
        if (active) {
            const int bt = min(d.tile, d.B - b0);
            const float *xb = d.x + d.x_step * step + ((size_t)g * d.B + b0) * d.I;
            float *yb = d.y + d.y_step * step + ((size_t)g * d.B + b0) * d.O;
            float *v = reinterpret_cast<float *>(srec + d.rec_words);
            if (d.tile == 1)
                run_item<true>(srec, v, bar, flags + gi, G, gi, lane, xb, yb, d.I, d.O, 1, 1, d.lg_split, &g_plan_error);
            else
                run_item<false>(srec, v, bar, flags + gi, G, gi, lane, xb, yb, d.I, d.O, bt, d.tile, 0, &g_plan_error);
        }
        __syncthreads();
        if (active && lane == 0) mbar_inval(bar);      // re-initialised by the next item using this slot
    }
}

struct Shape {
    int G = 0, tile = 0, split = 1;
};

struct HostBucket {
    int pop_index = 0;
    int n_class = 0;         // node-count bound of the bucket
    int max_used = 0;        // largest record (bytes) in the bucket
    std::vector<int32_t> gidx;
    Shape shape;
};

int lg(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// A shape the kernels can index: G and tile powers of two, tile <= G <= NT,
// split 1, 2 or 4 (a bad shape would mis-index shared memory, so it is
// refused on the host before any launch).
bool shape_ok(const Shape &s, int NT)
{
    const auto p2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    return p2(s.G) && s.G <= NT && p2(s.tile) && s.tile <= s.G && (s.split == 1 || s.split == 2 || s.split == 4);
}

// Launch shape without timing: as neat_default_launch, with groups of at
// most NT threads (the persistent block).
Shape heuristic_shape(int n_class, int batch, int NT)
{
    Shape s;
    s.split = 1;
    if (batch <= 1) {
        s.tile = 1;
        s.G = std::min(NT, n_class <= 64 ? 8 : (n_class <= 256 ? 16 : 32));
    } else {
        int t = 1;
        while (t < batch && t < 32 && t < NT) t <<= 1;
        s.tile = t;
        int nsub = tile_row_threads(n_class);
        while (nsub > 1 && t * nsub > NT) nsub >>= 1;
        s.G = t * nsub;
    }
    return s;
}

}  // namespace
}  // namespace neat

using namespace neat;

struct neat_plan {
    std::vector<neat_pop_desc> pops;
    neat_plan_options opt;
    std::vector<HostBucket> hb;
    std::vector<BucketDev> bd;
    BucketDev *d_buckets = nullptr;
    int32_t *d_gidx = nullptr;
    unsigned int *d_counters = nullptr;
    int n_counters = 0;
    int block_threads = 256;
    size_t smem = 0;
    int grid = 0;
    int total_items = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_first = -1, graph_steps = -1;
    std::string autotune_log;
    int max_footprint_bucket = -1;    // host bucket whose groups take the most shared memory
    size_t smem_override = 0;         // while timing one bucket: its own footprint
};

namespace neat {
namespace {

size_t region_bytes(const HostBucket &b, int I, int O)
{
    (void)I;
    (void)O;
    const size_t rec = (size_t)align16((uint32_t)b.max_used);
    const size_t vals = 4u * (size_t)((b.n_class * b.shape.tile + 3) & ~3);
    return (rec + vals + 15) & ~(size_t)15;
}

// Lay out the block items and the device bucket table for the current shapes.
int layout(neat_plan *P, cudaStream_t s)
{
    const int NT = P->block_threads;
    // largest records first
    std::vector<int> order(P->hb.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const size_t ca = (size_t)P->hb[a].max_used * P->hb[a].shape.tile;
        const size_t cb = (size_t)P->hb[b].max_used * P->hb[b].shape.tile;
        return ca > cb;
    });
    std::vector<BucketDev> bd;
    size_t smem_regions = 0;
    int cta = 0;
    size_t goff = 0;
    std::vector<size_t> goffs(P->hb.size());
    for (size_t i = 0; i < P->hb.size(); ++i) {
        goffs[i] = goff;
        goff += P->hb[i].gidx.size();
    }
    for (int bi : order) {
        const HostBucket &h = P->hb[bi];
        const neat_pop_desc &pd = P->pops[h.pop_index];
        BucketDev d;
        d.rec = static_cast<const uint8_t *>(pd.transformed_dev);
        d.gidx = P->d_gidx + goffs[bi];
        d.x = pd.inputs_dev;
        d.y = pd.outputs_dev;
        d.x_step = pd.in_step_stride;
        d.y_step = pd.out_step_stride;
        d.stride = record_stride(pd.dims);
        d.n_genomes = (int)h.gidx.size();
        d.I = pd.dims.num_inputs;
        d.O = pd.dims.num_outputs;
        d.B = pd.batch;
        d.tile = h.shape.tile;
        d.tiles = (pd.batch + d.tile - 1) / d.tile;
        d.lg_split = lg(h.shape.split);
        if (!shape_ok(h.shape, NT)) return invalid("plan: invalid bucket launch shape");
        d.G = h.shape.G;
        d.lgG = lg(d.G);
        const size_t reg = region_bytes(h, d.I, d.O);
        int gpc = NT / d.G;
        if (d.G > 32) gpc = std::min(gpc, 15);
        while (gpc > 1 && reg * gpc > 200u * 1024u) --gpc;
        if (reg * gpc + 16u * forward_header_words(NT) > 227u * 1024u)
            return invalid("plan: a bucket's region exceeds shared memory; use a smaller tile");
        d.gpc = gpc;
        d.region_words = (int)(reg / 16);
        d.rec_words = (int)(align16((uint32_t)h.max_used) / 16);
        d.rec_copy_bytes = (int)align16((uint32_t)h.max_used);
        const long items = (long)d.n_genomes * d.tiles;
        d.cta_begin = cta;
        d.cta_items = (int)((items + gpc - 1) / gpc);
        cta += d.cta_items;
        smem_regions = std::max(smem_regions, reg * gpc);
        bd.push_back(d);
    }
    P->bd = bd;
    P->total_items = cta;
    P->smem = smem_regions + 16u * forward_header_words(NT);
    P->max_footprint_bucket = -1;
    {
        size_t best = 0;
        for (size_t i = 0; i < bd.size(); ++i) {
            const size_t f = (size_t)bd[i].region_words * 16 * bd[i].gpc;
            if (f > best) {
                best = f;
                P->max_footprint_bucket = order[i];
            }
        }
    }
    if (P->d_buckets) cudaFree(P->d_buckets);
    cudaError_t e = cudaMalloc(&P->d_buckets, sizeof(BucketDev) * std::max<size_t>(bd.size(), 1));
    if (e != cudaSuccess) return cuda_fail(e, "plan: cudaMalloc buckets");
    e = cudaMemcpyAsync(P->d_buckets, bd.data(), sizeof(BucketDev) * bd.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "plan: copy buckets");
    // persistent grid: as many resident blocks as the shared memory allows
    int dev = 0, sms = 152, smem_sm = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per_sm = (int)(smem_sm / (P->smem + 1024));
    per_sm = std::max(1, std::min(per_sm, 2048 / NT));
    P->grid = std::max(1, std::min(sms * per_sm, P->total_items));
    for (auto f : {plan_kernel<true>, plan_kernel<false>}) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return cuda_fail(e, "plan: cudaFuncGetAttributes");
        if (P->smem + fa.sharedSizeBytes > 227u * 1024u)
            return invalid("plan: shared memory per block exceeds 227 KB; use a smaller tile");
        const int rc = allow_dynamic_smem(reinterpret_cast<const void *>(f), P->smem, "plan: shared memory per block");
        if (rc) return rc;
    }
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    return NEAT_OK;
}

int ensure_counters(neat_plan *P, int n)
{
    if (P->n_counters >= n) return NEAT_OK;
    if (P->d_counters) cudaFree(P->d_counters);
    P->d_counters = nullptr;
    cudaError_t e = cudaMalloc(&P->d_counters, sizeof(unsigned int) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "plan: cudaMalloc counters");
    P->n_counters = n;
    return NEAT_OK;
}

// One step of block items [lo, hi) using counter `ctr` (reset first).
int launch_step(neat_plan *P, int lo, int hi, unsigned int *ctr, int step, bool pdl, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(1, std::min(P->grid, hi - lo)));
    cfg.blockDim = dim3((unsigned)P->block_threads);
    cfg.dynamicSmemBytes = P->smem_override ? P->smem_override : P->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = pdl ? cudaLaunchKernelEx(&cfg, plan_kernel<true>, (const BucketDev *)P->d_buckets,
                                             (int)P->bd.size(), lo, hi, ctr, step)
                        : cudaLaunchKernelEx(&cfg, plan_kernel<false>, (const BucketDev *)P->d_buckets,
                                             (int)P->bd.size(), lo, hi, ctr, step);
    if (e != cudaSuccess) return cuda_fail(e, "plan: launch");
    return NEAT_OK;
}

// Time `reps` launches of bucket index `bi` (position in P->bd) alone.
float time_bucket(neat_plan *P, int bi, cudaStream_t s, int reps)
{
    const BucketDev &d = P->bd[bi];
    P->smem_override = (size_t)d.region_words * 16 * d.gpc + 16u * forward_header_words(P->block_threads);
    const int grid_saved = P->grid;
    {
        int dev = 0, sms = 152, smem_sm = 233472;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        int per_sm = (int)(smem_sm / (P->smem_override + 1024));
        per_sm = std::max(1, std::min(per_sm, 2048 / P->block_threads));
        P->grid = sms * per_sm;
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {
        cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned int), s);
        cudaEventRecord(a, s);
        if (launch_step(P, d.cta_begin, d.cta_begin + d.cta_items, P->d_counters, 0, false, s) != NEAT_OK) {
            best = 1e30f;
            break;
        }
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P->smem_override = 0;
    P->grid = grid_saved;
    return best;
}

// Time one whole step of the laid-out plan (best of reps).
float time_plan(neat_plan *P, cudaStream_t s, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {
        cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned int), s);
        cudaEventRecord(a, s);
        if (launch_step(P, 0, P->total_items, P->d_counters, 0, false, s) != NEAT_OK) break;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

std::vector<Shape> candidates(int n_class, int batch, int NT)
{
    std::vector<Shape> c;
    if (batch <= 1) {
        for (int G : {4, 8, 16, 32})
            for (int split : {1, 2})
                if (G <= NT) c.push_back(Shape{G, 1, split});
    } else {
        for (int t : {4, 8, 16, 32}) {
            if (t > 2 * batch && t > 4) continue;
            for (int nsub : {1, 2, 4, 8, 16, 32}) {
                if (t * nsub > NT || t * nsub < 8) continue;
                if (nsub > 1 && nsub * 4 > n_class) continue;       // more threads than a level can use
                c.push_back(Shape{t * nsub, t, 1});
            }
        }
    }
    return c;
}

// Footprint in shared memory of a bucket's groups in one block.
size_t footprint(const neat_plan *P, const HostBucket &h)
{
    int gpc = P->block_threads / h.shape.G;
    if (h.shape.G > 32) gpc = std::min(gpc, 15);
    return region_bytes(h, 0, 0) * gpc;
}

int autotune(neat_plan *P, cudaStream_t s, float *step_ms)
{
    char line[256];
    auto position_of = [&](size_t hbi) {
        size_t goff = 0;
        for (size_t i = 0; i < hbi; ++i) goff += P->hb[i].gidx.size();
        for (size_t i = 0; i < P->bd.size(); ++i)
            if (P->bd[i].gidx == P->d_gidx + goff) return (int)i;
        return -1;
    };
    // 1. each bucket alone, at its own shared-memory footprint
    std::vector<std::vector<std::pair<float, Shape>>> timed(P->hb.size());
    for (size_t hbi = 0; hbi < P->hb.size(); ++hbi) {
        HostBucket &h = P->hb[hbi];
        const neat_pop_desc &pd = P->pops[h.pop_index];
        const Shape keep = h.shape;
        for (const Shape &c : candidates(h.n_class, pd.batch, P->block_threads)) {
            h.shape = c;
            if (layout(P, s) != NEAT_OK) {
                cudaGetLastError();
                continue;
            }
            const int pos = position_of(hbi);
            if (pos < 0) continue;
            timed[hbi].push_back({time_bucket(P, pos, s, 2), c});
        }
        cudaGetLastError();
        std::sort(timed[hbi].begin(), timed[hbi].end(),
                  [](const std::pair<float, Shape> &a, const std::pair<float, Shape> &b) { return a.first < b.first; });
        h.shape = timed[hbi].empty() ? keep : timed[hbi][0].second;
    }
    // 2. the whole step: shrink the bucket that sets the block's shared
    //    memory (it limits every bucket's residency) while that pays
    int rc = layout(P, s);
    if (rc) return rc;
    float best_ms = time_plan(P, s, 2);
    for (int round = 0; round < 8; ++round) {
        const int hbi = P->max_footprint_bucket;
        if (hbi < 0) break;
        HostBucket &h = P->hb[hbi];
        const Shape cur = h.shape;
        const size_t cur_fp = footprint(P, h);
        bool improved = false;
        for (const auto &cand : timed[hbi]) {
            h.shape = cand.second;
            if (footprint(P, h) >= cur_fp) continue;
            if (layout(P, s) != NEAT_OK) {
                cudaGetLastError();
                continue;
            }
            const float ms = time_plan(P, s, 2);
            if (ms < best_ms) {
                best_ms = ms;
                improved = true;
                break;
            }
        }
        if (!improved) {
            h.shape = cur;
            break;
        }
    }
    for (size_t hbi = 0; hbi < P->hb.size(); ++hbi) {
        const HostBucket &h = P->hb[hbi];
        snprintf(line, sizeof(line), "%s{\"pop\":%d,\"n_class\":%d,\"G\":%d,\"tile\":%d,\"split\":%d}",
                 hbi ? "," : "", h.pop_index, h.n_class, h.shape.G, h.shape.tile, h.shape.split);
        P->autotune_log += line;
    }
    snprintf(line, sizeof(line), ",{\"block_threads\":%d,\"step_ms\":%.5f}", P->block_threads, best_ms);
    P->autotune_log += line;
    if (step_ms) *step_ms = best_ms;
    return layout(P, s);
}

// Autotune at each persistent block size and keep the fastest: large
// groups (a tile row of many threads for genomes of hundreds of nodes) need
// large blocks, many small groups share smaller ones well.
int autotune_block_threads(neat_plan *P, cudaStream_t s)
{
    struct Best {
        float ms = -1.0f;
        int NT = 0;
        std::vector<Shape> shapes;
        std::string log;
    } best;
    for (int NT : {256, 512, 1024}) {
        P->block_threads = NT;
        P->autotune_log.clear();
        for (HostBucket &b : P->hb) b.shape = heuristic_shape(b.n_class, P->pops[b.pop_index].batch, NT);
        int rc = layout(P, s);
        float ms = -1.0f;
        if (rc == NEAT_OK) rc = autotune(P, s, &ms);
        if (rc != NEAT_OK) {
            cudaGetLastError();
            clear_error();
            continue;
        }
        if (best.ms < 0.0f || ms < best.ms) {
            best.ms = ms;
            best.NT = NT;
            best.shapes.clear();
            for (const HostBucket &b : P->hb) best.shapes.push_back(b.shape);
            best.log = P->autotune_log;
        }
    }
    if (best.NT == 0) return invalid("neat_plan_create: no block size could be tuned");
    P->block_threads = best.NT;
    P->opt.block_threads = best.NT;
    for (size_t i = 0; i < P->hb.size(); ++i) P->hb[i].shape = best.shapes[i];
    P->autotune_log = best.log;
    return layout(P, s);
}

}  // namespace
}  // namespace neat

extern "C" int neat_plan_create(const neat_pop_desc *pops, int32_t npops, const neat_plan_options *opt,
                                void *stream, neat_plan **out)
{
    TraceRange trace_range("neat_plan_create");
    clear_error();
    if (!out) return invalid("neat_plan_create: null output pointer");
    *out = nullptr;
    if (!pops || npops < 1) return invalid("neat_plan_create: no populations");
    cudaStream_t s = as_stream(stream);
    neat_plan_options o = {0, 1, 0, 1};
    if (opt) o = *opt;
    const bool tune_block = o.autotune && o.block_threads == 0;
    if (o.block_threads == 0) o.block_threads = 256;
    if (o.block_threads < 32 || o.block_threads > 1024 || (o.block_threads & (o.block_threads - 1)))
        return invalid("neat_plan_create: block_threads must be a power of two in 32..1024");
    for (int p = 0; p < npops; ++p) {
        const neat_pop_desc &pd = pops[p];
        if (!dims_ok(pd.dims)) return invalid("neat_plan_create: invalid dims");
        if (pd.pop < 0 || pd.batch < 0) return invalid("neat_plan_create: pop and batch must be >= 0");
        if (pd.pop > 0 && pd.batch > 0 && (!pd.transformed_dev || !pd.outputs_dev ||
                                            (pd.dims.num_inputs > 0 && !pd.inputs_dev)))
            return invalid("neat_plan_create: null pointer");
        if (reinterpret_cast<uintptr_t>(pd.transformed_dev) & 15u)
            return invalid("neat_plan_create: transformed must be 16-byte aligned");
    }
    neat_plan *P = new neat_plan();
    P->pops.assign(pops, pops + npops);
    P->opt = o;
    P->block_threads = o.block_threads;
    // read every header once
    std::vector<std::vector<uint32_t>> hdrs(npops);
    for (int p = 0; p < npops; ++p) {
        const neat_pop_desc &pd = pops[p];
        if (pd.pop == 0 || pd.batch == 0) continue;
        hdrs[p].resize((size_t)pd.pop * 8);
        cudaError_t e = cudaMemcpy2DAsync(hdrs[p].data(), 32, pd.transformed_dev, record_stride(pd.dims), 32,
                                          (size_t)pd.pop, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            delete P;
            return cuda_fail(e, "neat_plan_create: header copy");
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "neat_plan_create: synchronize");
    }
    for (int p = 0; p < npops; ++p) {
        const neat_pop_desc &pd = pops[p];
        if (hdrs[p].empty()) continue;
        const int max_class = 1 << lg(pd.dims.max_nodes);
        std::vector<int> slot_of_class(12, -1);
        for (int g = 0; g < pd.pop; ++g) {
            const uint32_t *h = &hdrs[p][(size_t)g * 8];
            int n = (int)(h[0] & 0xffffu);
            int cls = o.size_buckets ? std::max(16, 1 << lg(std::max(n, 1))) : max_class;
            cls = std::min(cls, std::max(16, max_class));
            int key = lg(cls);
            if (slot_of_class[key] < 0) {
                slot_of_class[key] = (int)P->hb.size();
                HostBucket b;
                b.pop_index = p;
                b.n_class = std::min(cls, pd.dims.max_nodes);
                b.max_used = 32;
                P->hb.push_back(b);
            }
            HostBucket &b = P->hb[slot_of_class[key]];
            b.gidx.push_back(g);
            const uint32_t used = std::min<uint32_t>(h[4], record_max_bytes(pd.dims.num_inputs, pd.dims.num_outputs,
                                                                            pd.dims.max_nodes, pd.dims.max_conns));
            b.max_used = std::max<int>(b.max_used, (int)align16(used));
        }
    }
    // within a bucket, deepest and largest genomes first: groups that share
    // a warp then have similar level counts (a warp walks as many levels as
    // its deepest genome), and the longest items start first
    for (HostBucket &b : P->hb) {
        const std::vector<uint32_t> &h = hdrs[b.pop_index];
        std::stable_sort(b.gidx.begin(), b.gidx.end(), [&](int32_t x, int32_t y) {
            const uint32_t lx = h[(size_t)x * 8] >> 16, ly = h[(size_t)y * 8] >> 16;
            if (lx != ly) return lx > ly;
            return h[(size_t)x * 8 + 1] > h[(size_t)y * 8 + 1];
        });
        b.shape = heuristic_shape(b.n_class, P->pops[b.pop_index].batch, P->block_threads);
    }
    size_t total = 0;
    for (const HostBucket &b : P->hb) total += b.gidx.size();
    if (total > 0) {
        e = cudaMalloc(&P->d_gidx, sizeof(int32_t) * total);
        if (e != cudaSuccess) {
            delete P;
            return cuda_fail(e, "neat_plan_create: cudaMalloc indices");
        }
        size_t off = 0;
        for (const HostBucket &b : P->hb) {
            e = cudaMemcpyAsync(P->d_gidx + off, b.gidx.data(), sizeof(int32_t) * b.gidx.size(),
                                cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                neat_plan_destroy(P);
                return cuda_fail(e, "neat_plan_create: copy indices");
            }
            off += b.gidx.size();
        }
    }
    int rc = ensure_counters(P, 1);
    if (rc == NEAT_OK) rc = layout(P, s);
    if (rc == NEAT_OK && o.autotune && !P->hb.empty())
        rc = tune_block ? autotune_block_threads(P, s) : autotune(P, s, nullptr);
    if (rc == NEAT_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "neat_plan_create: synchronize");
    }
    if (rc != NEAT_OK) {
        neat_plan_destroy(P);
        return rc;
    }
    *out = P;
    return NEAT_OK;
}

extern "C" int neat_plan_forward(neat_plan *P, int32_t step, void *stream)
{
    TraceRange trace_range("neat_plan_forward");
    clear_error();
    if (!P) return invalid("neat_plan_forward: null plan");
    if (step < 0) return invalid("neat_plan_forward: step < 0");
    if (P->total_items == 0) return NEAT_OK;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "neat_plan_forward: counter reset");
    return launch_step(P, 0, P->total_items, P->d_counters, step, false, s);
}

extern "C" int neat_plan_forward_steps(neat_plan *P, int32_t first_step, int32_t steps, void *stream)
{
    TraceRange trace_range("neat_plan_forward_steps");
    clear_error();
    if (!P) return invalid("neat_plan_forward_steps: null plan");
    if (first_step < 0 || steps < 0) return invalid("neat_plan_forward_steps: negative step");
    if (steps == 0 || P->total_items == 0) return NEAT_OK;
    if (!P->exec || P->graph_first != first_step || P->graph_steps != steps) {
        if (P->exec) {
            cudaGraphExecDestroy(P->exec);
            P->exec = nullptr;
        }
        int rc = ensure_counters(P, steps);
        if (rc) return rc;
        cudaError_t e;
        if (!P->cap) {
            e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "neat_plan_forward_steps: stream");
        }
        e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "neat_plan_forward_steps: begin capture");
        e = cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned int) * (size_t)steps, P->cap);
        for (int k = 0; k < steps && rc == NEAT_OK && e == cudaSuccess; ++k)
            rc = launch_step(P, 0, P->total_items, P->d_counters + k, first_step + k, P->opt.pdl && k > 0, P->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(P->cap, &graph);
        if (rc != NEAT_OK || e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (rc) return rc;
            return cuda_fail(e != cudaSuccess ? e : e2, "neat_plan_forward_steps: capture");
        }
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->exec = nullptr;
            return cuda_fail(e, "neat_plan_forward_steps: instantiate");
        }
        P->graph_first = first_step;
        P->graph_steps = steps;
    }
    cudaError_t e = cudaGraphLaunch(P->exec, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "neat_plan_forward_steps: launch");
    return NEAT_OK;
}

extern "C" int neat_plan_describe(const neat_plan *P, char *buf, int32_t len)
{
    if (!P) return invalid("neat_plan_describe: null plan");
    std::string js = "{\"block_threads\":" + std::to_string(P->block_threads) +
                     ",\"grid\":" + std::to_string(P->grid) + ",\"smem\":" + std::to_string(P->smem) +
                     ",\"block_items\":" + std::to_string(P->total_items) + ",\"buckets\":[";
    for (size_t i = 0; i < P->bd.size(); ++i) {
        const BucketDev &d = P->bd[i];
        char tmp[320];
        snprintf(tmp, sizeof(tmp),
                 "%s{\"genomes\":%d,\"batch\":%d,\"G\":%d,\"tile\":%d,\"split\":%d,\"groups_per_block\":%d,"
                 "\"record_bytes\":%d,\"region_bytes\":%d,\"block_items\":%d}",
                 i ? "," : "", d.n_genomes, d.B, d.G, d.tile, 1 << d.lg_split, d.gpc, d.rec_copy_bytes,
                 d.region_words * 16, d.cta_items);
        js += tmp;
    }
    js += "],\"autotune\":[" + P->autotune_log + "]}";
    if (buf && len > 0) {
        const size_t n = std::min<size_t>(js.size(), (size_t)len - 1);
        memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return (int)js.size() + 1;
}

extern "C" void neat_plan_destroy(neat_plan *P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->cap) cudaStreamDestroy(P->cap);
    if (P->d_buckets) cudaFree(P->d_buckets);
    if (P->d_gidx) cudaFree(P->d_gidx);
    if (P->d_counters) cudaFree(P->d_counters);
    delete P;
}

namespace neat {
int read_plan_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_plan_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "plan error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_plan_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "plan error word: clear");
    }
    return NEAT_OK;
}
}  // namespace neat

// ------------------------------------------------------------------------
// Allocation-free batched forward: the persistent plan kernel, fed from a
// fixed scratch array in device memory instead of buffers the plan
// allocates.  For callers that cannot call cudaMalloc (see neat.h).
//
// Scratch layout (file-scope, 256-byte aligned, held by every GPU that loads
// the library until the process exits):
//   [0, 256)             the work counter, cleared by every call
//   [256, idx_off)       the bucket table, written by every call
//   [idx_off, end)       genome indices 0 .. kNoallocMaxGenomes-1, written once
// Host code only knows the array through a host-side stand-in, so its device
// address is fetched with cudaGetSymbolAddress once per device.
namespace neat {
namespace {

constexpr int kNoallocMaxPops = 64;
constexpr int kNoallocMaxGenomes = 32768;
constexpr size_t kNoallocTableOff = 256;
constexpr size_t kNoallocIdxOff = kNoallocTableOff + ((sizeof(BucketDev) * kNoallocMaxPops + 255) & ~(size_t)255);
constexpr size_t kNoallocScratchBytes = kNoallocIdxOff + sizeof(int32_t) * kNoallocMaxGenomes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

__global__ void noalloc_fill_indices(int32_t *idx, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

// The call's bucket table travels as a kernel argument (no host-to-device
// copy); one small kernel writes it into the scratch array and clears the
// work counter.
struct NoallocTable {
    BucketDev b[kNoallocMaxPops];
};

__global__ void noalloc_set_table(const NoallocTable t, int nb, BucketDev *dst, unsigned int *counter)
{
    const uint32_t *src = reinterpret_cast<const uint32_t *>(t.b);
    uint32_t *out = reinterpret_cast<uint32_t *>(dst);
    const int words = nb * (int)(sizeof(BucketDev) / sizeof(uint32_t));
    for (int i = threadIdx.x; i < words; i += blockDim.x) out[i] = src[i];
    if (threadIdx.x == 0) *counter = 0u;
}
static_assert(sizeof(BucketDev) % sizeof(uint32_t) == 0, "bucket entries copy as words");

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[256] = {};   // device address of the scratch array, per device id

// Per-device set-up, on the first call made with that device current: the
// array's device address (cudaGetSymbolAddress) and its index list.
int noalloc_setup(cudaStream_t s, unsigned char **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 256) return invalid("neat_forward_multi_noalloc: device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_base[dev]) {
        *base = g_noalloc_base[dev];
        return NEAT_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: cudaGetSymbolAddress");
    noalloc_fill_indices<<<64, 256, 0, s>>>(reinterpret_cast<int32_t *>(static_cast<unsigned char *>(p) + kNoallocIdxOff),
                                            kNoallocMaxGenomes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: index fill");
    // the index list is complete before any call (on any stream or thread)
    // can see the cached address
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: index fill");
    g_noalloc_base[dev] = static_cast<unsigned char *>(p);
    *base = g_noalloc_base[dev];
    return NEAT_OK;
}

}  // namespace
}  // namespace neat

extern "C" int neat_forward_multi_noalloc(const neat_pop_desc *pops, int32_t npops, int32_t step, void *stream)
{
    TraceRange trace_range("neat_forward_multi_noalloc");
    clear_error();
    if (!pops) return invalid("neat_forward_multi_noalloc: null populations");
    if (npops < 1 || npops > kNoallocMaxPops)
        return invalid("neat_forward_multi_noalloc: npops must be in 1..64 (the scratch table holds 64 populations)");
    if (step < 0) return invalid("neat_forward_multi_noalloc: step < 0");
    for (int p = 0; p < npops; ++p) {
        const neat_pop_desc &pd = pops[p];
        if (!dims_ok(pd.dims)) return invalid("neat_forward_multi_noalloc: invalid dims");
        if (pd.pop < 0 || pd.batch < 0) return invalid("neat_forward_multi_noalloc: pop and batch must be >= 0");
        if (pd.pop > kNoallocMaxGenomes)
            return invalid("neat_forward_multi_noalloc: at most 32768 genomes per population (scratch index list)");
        if (pd.pop > 0 && pd.batch > 0 &&
            (!pd.transformed_dev || !pd.outputs_dev || (pd.dims.num_inputs > 0 && !pd.inputs_dev)))
            return invalid("neat_forward_multi_noalloc: null pointer");
        if (reinterpret_cast<uintptr_t>(pd.transformed_dev) & 15u)
            return invalid("neat_forward_multi_noalloc: transformed must be 16-byte aligned");
    }
    cudaStream_t s = as_stream(stream);
    unsigned char *base = nullptr;
    int rc = noalloc_setup(s, &base);
    if (rc) return rc;

    // one bucket per population, shapes from the heuristic, reserved record size
    const int NT = 256;
    NoallocTable tab;
    BucketDev *table = tab.b;
    int order[kNoallocMaxPops];
    int nb = 0;
    for (int p = 0; p < npops; ++p)
        if (pops[p].pop > 0 && pops[p].batch > 0) order[nb++] = p;
    for (int i = 1; i < nb; ++i)                    // largest records first
        for (int j = i; j > 0; --j) {
            const neat_dims &a = pops[order[j]].dims, &b = pops[order[j - 1]].dims;
            if (record_max_bytes(a.num_inputs, a.num_outputs, a.max_nodes, a.max_conns) <=
                record_max_bytes(b.num_inputs, b.num_outputs, b.max_nodes, b.max_conns))
                break;
            std::swap(order[j], order[j - 1]);
        }
    size_t smem_regions = 0;
    int64_t cta = 0;
    for (int i = 0; i < nb; ++i) {
        const neat_pop_desc &pd = pops[order[i]];
        const Shape sh = heuristic_shape(pd.dims.max_nodes, pd.batch, NT);
        const uint32_t rec = record_max_bytes(pd.dims.num_inputs, pd.dims.num_outputs, pd.dims.max_nodes,
                                              pd.dims.max_conns);
        const size_t reg = ((size_t)rec + 4u * (size_t)((pd.dims.max_nodes * sh.tile + 3) & ~3) + 15) & ~(size_t)15;
        if (!shape_ok(sh, NT)) return invalid("neat_forward_multi_noalloc: invalid launch shape");
        int gpc = NT / sh.G;
        if (sh.G > 32) gpc = std::min(gpc, 15);
        while (gpc > 1 && reg * gpc > 200u * 1024u) --gpc;
        if (reg * gpc + 16u * forward_header_words(NT) > 227u * 1024u)
            return invalid("neat_forward_multi_noalloc: a population's genome is too large for one block");
        BucketDev &d = table[i];
        d.rec = static_cast<const uint8_t *>(pd.transformed_dev);
        d.gidx = reinterpret_cast<const int32_t *>(base + kNoallocIdxOff);
        d.x = pd.inputs_dev;
        d.y = pd.outputs_dev;
        d.x_step = pd.in_step_stride;
        d.y_step = pd.out_step_stride;
        d.stride = record_stride(pd.dims);
        d.n_genomes = pd.pop;
        d.I = pd.dims.num_inputs;
        d.O = pd.dims.num_outputs;
        d.B = pd.batch;
        d.tile = sh.tile;
        d.tiles = (pd.batch + sh.tile - 1) / sh.tile;
        d.lg_split = lg(sh.split);
        d.G = sh.G;
        d.lgG = lg(sh.G);
        d.gpc = gpc;
        d.region_words = (int)(reg / 16);
        d.rec_words = (int)(rec / 16);
        d.rec_copy_bytes = (int)rec;
        const int64_t items = ((int64_t)d.n_genomes * d.tiles + gpc - 1) / gpc;
        if (items > INT_MAX || cta + items > INT_MAX)
            return invalid("neat_forward_multi_noalloc: more than 2^31 - 1 block work items in one call");
        d.cta_begin = (int)cta;
        d.cta_items = (int)items;
        cta += items;
        smem_regions = std::max(smem_regions, reg * gpc);
    }
    if (nb == 0) return NEAT_OK;
    const size_t smem = smem_regions + 16u * forward_header_words(NT);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, plan_kernel<false>);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: cudaFuncGetAttributes");
    if (smem + fa.sharedSizeBytes > 227u * 1024u)
        return invalid("neat_forward_multi_noalloc: shared memory per block exceeds 227 KB");
    {
        const int rc = allow_dynamic_smem(reinterpret_cast<const void *>(plan_kernel<false>), smem,
                                          "neat_forward_multi_noalloc: shared memory per block");
        if (rc) return rc;
    }
    // the bucket table and a zero work counter, by one small kernel
    noalloc_set_table<<<1, 256, 0, s>>>(tab, nb, reinterpret_cast<BucketDev *>(base + kNoallocTableOff),
                                        reinterpret_cast<unsigned int *>(base));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: table");
    int dev = 0, sms = 152, smem_sm = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per_sm = std::max(1, std::min((int)(smem_sm / (smem + 1024)), 2048 / NT));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, cta));
    plan_kernel<false><<<grid, NT, smem, s>>>(reinterpret_cast<const BucketDev *>(base + kNoallocTableOff), nb, 0,
                                              (int)cta, reinterpret_cast<unsigned int *>(base), step);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_multi_noalloc: launch");
    return NEAT_OK;
}

// ------------------------------------------------------------------------
// Internal helpers for other translation units (the serving runtime).
namespace neat {

int fill_population_bucket(const neat_pop_desc &pd, const int32_t *gidx_dev, int block_threads, int cta_begin,
                           BucketDev *out, size_t *footprint)
{
    const Shape sh = heuristic_shape(pd.dims.max_nodes, pd.batch, block_threads);
    const uint32_t rec = record_max_bytes(pd.dims.num_inputs, pd.dims.num_outputs, pd.dims.max_nodes,
                                          pd.dims.max_conns);
    const size_t reg = ((size_t)rec + 4u * (size_t)((pd.dims.max_nodes * sh.tile + 3) & ~3) + 15) & ~(size_t)15;
    if (!shape_ok(sh, block_threads)) return invalid("invalid launch shape for a population bucket");
    int gpc = block_threads / sh.G;
    if (sh.G > 32) gpc = std::min(gpc, 15);
    while (gpc > 1 && reg * gpc > 200u * 1024u) --gpc;
    if (gpc < 1 || reg * gpc + 16u * forward_header_words(block_threads) > 227u * 1024u)
        return invalid("a genome of this size does not fit one block");
    BucketDev &d = *out;
    d.rec = static_cast<const uint8_t *>(pd.transformed_dev);
    d.gidx = gidx_dev;
    d.x = pd.inputs_dev;
    d.y = pd.outputs_dev;
    d.x_step = pd.in_step_stride;
    d.y_step = pd.out_step_stride;
    d.stride = record_stride(pd.dims);
    d.n_genomes = pd.pop;
    d.I = pd.dims.num_inputs;
    d.O = pd.dims.num_outputs;
    d.B = pd.batch;
    d.tile = sh.tile;
    d.tiles = (pd.batch + sh.tile - 1) / sh.tile;
    d.lg_split = lg(sh.split);
    d.G = sh.G;
    d.lgG = lg(sh.G);
    d.gpc = gpc;
    d.region_words = (int)(reg / 16);
    d.rec_words = (int)(rec / 16);
    d.rec_copy_bytes = (int)rec;
    d.cta_begin = cta_begin;
    d.cta_items = (int)(((long)d.n_genomes * d.tiles + gpc - 1) / gpc);
    *footprint = reg * gpc;
    return NEAT_OK;
}

int launch_plan_table(const BucketDev *table_dev, int nb, int total_items, unsigned int *counter_dev, int step,
                      size_t smem_regions, int block_threads, cudaStream_t s)
{
    if (nb == 0 || total_items == 0) return NEAT_OK;
    const size_t smem = smem_regions + 16u * forward_header_words(block_threads);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, plan_kernel<false>);
    if (e != cudaSuccess) return cuda_fail(e, "plan table: cudaFuncGetAttributes");
    if (smem + fa.sharedSizeBytes > 227u * 1024u) return invalid("plan table: shared memory exceeds 227 KB");
    {
        const int rc = allow_dynamic_smem(reinterpret_cast<const void *>(plan_kernel<false>), smem,
                                          "plan table: shared memory per block");
        if (rc) return rc;
    }
    int dev = 0, sms = 152, smem_sm = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int per_sm = std::max(1, std::min((int)(smem_sm / (smem + 1024)), 2048 / block_threads));
    const int grid = std::max(1, std::min(sms * per_sm, total_items));
    plan_kernel<false><<<grid, block_threads, smem, s>>>(table_dev, nb, 0, total_items, counter_dev, step);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "plan table: launch");
    return NEAT_OK;
}

}  // namespace neat
