// Transformation stage of tensorized NEAT inference (Section 3.3): one thread
// block per genome turns the padded node/connection tensors (Section 3.1)
// into a record holding the layered Kahn order and, in place of the dense
// expanded-connection tensor C_exp, the enabled incoming edges of every node
// packed by destination position (layout in include/neat.h).
//
// All per-genome work happens in shared memory, in time linear in the rows:
//   1. node rows: presence, key and attribute checks; keys go into an
//      open-addressing table key -> lowest row (a duplicated key shows up on
//      insertion);
//   2. connection rows: checks, endpoint lookup, duplicate (in,out) pairs
//      found by inserting them into a hash set;
//   3. layered Kahn: one pass over the active edges per level, removing the
//      edges of level L with shared-memory atomics; a node whose count hits
//      zero joins level L+1;
//   4. positions = rank of (level, row), and edges in (destination position,
//      connection row) order, each by a stable counting sort that one warp
//      runs over the rows in chunks of 32 (ranks inside a chunk from
//      __match_any_sync), which fixes each node's summation order.
#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_hash.cuh"
#include "neat_trace.h"

namespace neat {
namespace {

struct TransformArgs {
    const float *nodes;
    const float *conns;
    uint8_t *out;
    uint32_t *status;
    size_t stride;
    int pop, I, O, N, C;
    int Np2, Cp2;   // powers of two >= N and >= max(C, 1)
    int recurrent;  // cycles allowed: no Kahn order, every present node in level 0 (row order)
};

__device__ __forceinline__ bool is_enum(float v, int n)
{
    return !isnan(v) && floorf(v) == v && v >= 0.0f && v < (float)n;
}

// In-place exclusive prefix sum of a[0..n), by the 32 threads of warp 0.
__device__ void warp_exclusive_scan(int *a, int n)
{
    const int lane = threadIdx.x & 31;
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const int x = (i < n) ? a[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (i < n) a[i] = carry + incl - x;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Stable counting placement by warp 0: items 0..count-1 in index order, item
// i in bucket bucket_of(i) (negative: skipped), placed at start[b] + the
// number of earlier items of bucket b (run[b] counts them chunk by chunk;
// zero on entry).  place(i, slot) records the result.
template <typename BucketOf, typename Place>
__device__ void stable_place(int count, const int *start, int *run, BucketOf bucket_of, Place place)
{
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int base = 0; base < count; base += 32) {
        const int i = base + lane;
        const int b = (i < count) ? bucket_of(i) : -1;
        const unsigned m = __match_any_sync(0xffffffffu, b >= 0 ? b : -1 - lane);   // skipped items stay alone
        if (b >= 0) place(i, start[b] + run[b] + __popc(m & below));
        __syncwarp();
        if (b >= 0 && lane == 31 - __clz(m)) run[b] += __popc(m);              // last item of its bucket here
        __syncwarp();
    }
}

__host__ __device__ inline size_t transform_smem_bytes(int N, int C, int I, int O, int Np2, int Cp2)
{
    size_t b = 16u * (size_t)Np2 + 16u * (size_t)Cp2;        // key table, pair set
    b += 4u * (size_t)(9 * N + 1 + I + O);                    // level, indeg, cnt, pos, row, ebeg, lstart, lrun, erun, io
    b += 2u * 2u * (size_t)C;                                 // src_row, dst_row
    return (b + 15u) & ~(size_t)15u;
}

__global__ void __launch_bounds__(512) transform_kernel(TransformArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int g = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int N = a.N, C = a.C, I = a.I, O = a.O;
    const uint32_t kmask = 2u * (uint32_t)a.Np2 - 1u, pmask = 2u * (uint32_t)a.Cp2 - 1u;

    unsigned long long *ktab = reinterpret_cast<unsigned long long *>(sm);
    unsigned long long *ptab = ktab + 2 * a.Np2;
    int *level = reinterpret_cast<int *>(ptab + 2 * a.Cp2);   // -2 absent, -1 unplaced
    int *indeg = level + N;
    int *cnt = indeg + N;
    int *pos_of_row = cnt + N;
    int *row_of_pos = pos_of_row + N;
    int *ebeg = row_of_pos + N;
    int *lstart = ebeg + N;                                    // [N + 1]
    int *lrun = lstart + N + 1;
    int *erun = lrun + N;
    int *io_row = erun + N;
    short *src_row = reinterpret_cast<short *>(io_row + I + O);
    short *dst_row = src_row + C;

    __shared__ unsigned int st, acts_seen, aggs_seen;
    __shared__ int n_present, n_edges, max_level;
    if (tid == 0) {
        st = 0;
        acts_seen = 0;
        aggs_seen = 0;
        n_present = 0;
        n_edges = 0;
        max_level = -1;
        lstart[N] = 0;
    }
    const float *nd = a.nodes + (size_t)g * N * 5;
    const float4 *cn = reinterpret_cast<const float4 *>(a.conns + (size_t)g * C * 4);
    for (int i = tid; i < 2 * a.Np2; i += nt) ktab[i] = kFree;
    for (int i = tid; i < 2 * a.Cp2; i += nt) ptab[i] = kFree;
    for (int r = tid; r < N; r += nt) {
        lstart[r] = 0;
        lrun[r] = 0;
        erun[r] = 0;
    }
    __syncthreads();

    // 1. node rows (Section 3.1 encoding; an absent row is NaN); keys into
    //    the key -> lowest row table, duplicates found on insertion
    unsigned int lst = 0;
    for (int r = tid; r < N; r += nt) {
        const float k = __ldg(nd + r * 5);
        indeg[r] = 0;
        level[r] = -2;
        if (isnan(k)) continue;
        if (!is_key(k)) { lst |= NEAT_G_BADKEY; continue; }
        const float bias = __ldg(nd + r * 5 + 1), resp = __ldg(nd + r * 5 + 2);
        const float agg = __ldg(nd + r * 5 + 3), act = __ldg(nd + r * 5 + 4);
        if (!is_enum(agg, 4) || !is_enum(act, 7)) lst |= NEAT_G_BADENUM;
        else if (k >= (float)I) {
            atomicOr(&acts_seen, 1u << (int)act);
            atomicOr(&aggs_seen, 1u << (int)agg);
        }
        if (isnan(bias) || isnan(resp)) lst |= NEAT_G_BADATTR;
        level[r] = -1;
        if (key_insert(ktab, kmask, (uint32_t)k, (uint32_t)r)) lst |= NEAT_G_DUPKEY;
        atomicAdd(&n_present, 1);
    }
    if (lst) atomicOr(&st, lst);
    __syncthreads();
    const int n = n_present;

    lst = 0;
    for (int j = tid; j < I + O; j += nt) {
        const int r = key_row(ktab, kmask, (uint32_t)j);
        io_row[j] = r;
        if (r < 0) lst |= NEAT_G_MISSING_IO;
    }

    // 2. connection rows; disabled ones only count towards duplicate pairs
    for (int c = tid; c < C; c += nt) {
        src_row[c] = dst_row[c] = -1;
        const float4 row = __ldg(cn + c);
        if (isnan(row.x) || isnan(row.y) || isnan(row.z)) continue;
        if (!is_key(row.x) || !is_key(row.y)) { lst |= NEAT_G_BADKEY; continue; }
        const uint32_t ki = (uint32_t)row.x, ko = (uint32_t)row.y;
        if (pair_insert(ptab, pmask, ((unsigned long long)ki << 24) | ko)) lst |= NEAT_G_DUPCONN;
        if (row.z == 0.0f) continue;
        if (isnan(row.w)) lst |= NEAT_G_BADATTR;
        const int s = key_row(ktab, kmask, ki), d = key_row(ktab, kmask, ko);
        if (s < 0 || d < 0) { lst |= NEAT_W_DANGLING; continue; }
        if (ko < (uint32_t)I) { lst |= NEAT_W_INTO_INPUT; continue; }
        src_row[c] = (short)s;
        dst_row[c] = (short)d;
        atomicAdd(&indeg[d], 1);
        atomicAdd(&n_edges, 1);
    }
    if (lst) atomicOr(&st, lst);
    __syncthreads();

    // 3. layered Kahn: level 0 = present nodes without enabled incoming edges
    for (int r = tid; r < N; r += nt) {
        cnt[r] = indeg[r];
        if (level[r] == -1 && (indeg[r] == 0 || a.recurrent)) level[r] = 0;
    }
    // one barrier per level: it also tells every thread whether any node
    // joined the next level
    __syncthreads();
    for (int L = 0; !a.recurrent; ++L) {
        int joined = 0;
        for (int c = tid; c < C; c += nt) {
            const int d = dst_row[c];
            if (d >= 0 && level[src_row[c]] == L) {
                if (atomicSub(&indeg[d], 1) == 1) {
                    level[d] = L + 1;
                    joined = 1;
                }
            }
        }
        if (!__syncthreads_or(joined)) break;
    }
    lst = 0;
    int lmax = -1;
    for (int r = tid; r < N; r += nt) {
        if (level[r] == -1) lst |= NEAT_G_CYCLE;
        lmax = max(lmax, level[r]);
    }
    if (lst) atomicOr(&st, lst);
    atomicMax(&max_level, lmax);
    __syncthreads();

    const uint32_t status = st;
    uint8_t *rec = a.out + (size_t)g * a.stride;
    if (status & NEAT_G_ERROR_MASK) {
        if (tid == 0) {
            uint4 *h = reinterpret_cast<uint4 *>(rec);
            h[0] = make_uint4((unsigned)n, 0u, status, 0xffffu);
            h[1] = make_uint4(kHeaderBytes, kHeaderBytes, kHeaderBytes, kHeaderBytes);
            if (a.status) a.status[g] = status;
        }
        return;
    }

    // 4. positions = rank of (level, row): a stable counting sort by level
    const int nl = max_level + 1;
    const int E = n_edges;
    const uint32_t off_edge = kHeaderBytes + kNodeBytes * (uint32_t)n;
    const uint32_t off_level = align16(off_edge + kEdgeBytes * (uint32_t)E);
    const uint32_t off_io = align16(off_level + 2u * (uint32_t)(nl + 1));
    const uint32_t used = align16(off_io + 2u * (uint32_t)(I + O));
    for (int r = tid; r < N; r += nt)
        if (level[r] >= 0) atomicAdd(&lstart[level[r]], 1);
    __syncthreads();
    if (tid < 32) {
        warp_exclusive_scan(lstart, nl);
        __syncwarp();
        stable_place(N, lstart, lrun, [&](int r) { return level[r]; },
                     [&](int r, int p) {
                         pos_of_row[r] = p;
                         row_of_pos[p] = r;
                     });
    }
    __syncthreads();
    uint16_t *lev_out = reinterpret_cast<uint16_t *>(rec + off_level);
    for (int L = tid; L < nl; L += nt) lev_out[L] = (uint16_t)lstart[L];
    if (tid == 0) lev_out[nl] = (uint16_t)n;

    // 5. edges in (destination position, connection row) order: a stable
    //    counting sort by destination position
    for (int p = tid; p < n; p += nt) ebeg[p] = cnt[row_of_pos[p]];
    __syncthreads();
    uint2 *edges = reinterpret_cast<uint2 *>(rec + off_edge);
    if (tid < 32) {
        warp_exclusive_scan(ebeg, n);
        __syncwarp();
        stable_place(C, ebeg, erun, [&](int c) { return dst_row[c] >= 0 ? pos_of_row[dst_row[c]] : -1; },
                     [&](int c, int k) {
                         const float w = __ldg(a.conns + ((size_t)g * C + c) * 4 + 3);
                         edges[k] = make_uint2(__float_as_uint(w), (uint32_t)pos_of_row[src_row[c]]);
                     });
    }
    __syncthreads();

    // 6. node entries by position, io positions, header
    uint4 *nodes_out = reinterpret_cast<uint4 *>(rec + kHeaderBytes);
    for (int p = tid; p < n; p += nt) {
        const int r = row_of_pos[p];
        const float key = __ldg(nd + r * 5);
        const float bias = __ldg(nd + r * 5 + 1), resp = __ldg(nd + r * 5 + 2);
        const uint32_t agg = (uint32_t)__ldg(nd + r * 5 + 3);
        const uint32_t act = key < (float)I ? (uint32_t)kInputAct : (uint32_t)__ldg(nd + r * 5 + 4);
        nodes_out[p] = make_uint4(__float_as_uint(bias), __float_as_uint(resp),
                                  (uint32_t)ebeg[p] | ((uint32_t)cnt[r] << 16),
                                  act | (agg << 8) | ((uint32_t)r << 16));
    }
    // leading positions that are input nodes (a prefix of level 0)
    __shared__ int lead_inputs;
    if (tid == 0) lead_inputs = n;
    __syncthreads();
    for (int p = tid; p < n; p += nt)
        if (__ldg(nd + row_of_pos[p] * 5) >= (float)I) atomicMin(&lead_inputs, p);
    __syncthreads();
    uint16_t *io_out = reinterpret_cast<uint16_t *>(rec + off_io);
    for (int j = tid; j < I + O; j += nt) io_out[j] = (uint16_t)pos_of_row[io_row[j]];
    if (tid == 0) {
        uint4 *h = reinterpret_cast<uint4 *>(rec);
        const uint32_t ua = __popc(acts_seen) == 1 ? (uint32_t)(__ffs(acts_seen) - 1) : 0xffu;
        const uint32_t ug = __popc(aggs_seen) == 1 ? (uint32_t)(__ffs(aggs_seen) - 1) : 0xffu;
        h[0] = make_uint4((unsigned)n | ((unsigned)nl << 16), (unsigned)E, status,
                          ua | (ug << 8) | ((uint32_t)lead_inputs << 16));
        h[1] = make_uint4(used, off_edge, off_level, off_io);
        if (a.status) a.status[g] = status;
    }
}

int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

}  // namespace neat

using namespace neat;

extern "C" size_t neat_record_stride(neat_dims d)
{
    return dims_ok(d) ? record_stride(d) : 0;
}

extern "C" size_t neat_transformed_bytes(int32_t pop, neat_dims d)
{
    if (!dims_ok(d) || pop < 0) return 0;
    return record_stride(d) * (size_t)pop;
}

static int transform_impl(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                          void *transformed_dev, size_t transformed_bytes, uint32_t *status_dev, void *stream,
                          int recurrent)
{
    TraceRange trace_range(recurrent ? "neat_transform_recurrent" : "neat_transform");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_transform: invalid dims");
    if (pop < 0) return invalid("neat_transform: pop < 0");
    if (pop == 0) return NEAT_OK;
    if (!nodes_dev || (!conns_dev && d.max_conns > 0) || !transformed_dev)
        return invalid("neat_transform: null pointer");
    if ((reinterpret_cast<uintptr_t>(conns_dev) & 15u) || (reinterpret_cast<uintptr_t>(transformed_dev) & 15u))
        return invalid("neat_transform: conns and transformed must be 16-byte aligned");
    const size_t stride = record_stride(d);
    if (transformed_bytes < stride * (size_t)pop) {
        set_error("neat_transform: transformed buffer too small");
        return NEAT_ENOMEM;
    }
    TransformArgs a;
    a.nodes = nodes_dev;
    a.conns = conns_dev;
    a.out = static_cast<uint8_t *>(transformed_dev);
    a.status = status_dev;
    a.stride = stride;
    a.pop = pop;
    a.I = d.num_inputs;
    a.O = d.num_outputs;
    a.N = d.max_nodes;
    a.C = d.max_conns;
    a.Np2 = next_pow2(a.N);
    a.Cp2 = next_pow2(a.C > 0 ? a.C : 1);
    a.recurrent = recurrent;
    const size_t smem = transform_smem_bytes(a.N, a.C, a.I, a.O, a.Np2, a.Cp2);
    const int threads = (a.N <= 64 && a.C <= 512) ? 128 : (a.N <= 256 && a.C <= 2048 ? 256 : 512);
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(transform_kernel), smem,
                                "neat_transform: shared memory per block");
    if (rc) return rc;
    transform_kernel<<<pop, threads, smem, as_stream(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_transform: launch");
    return NEAT_OK;
}

extern "C" int neat_transform(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                              void *transformed_dev, size_t transformed_bytes, uint32_t *status_dev,
                              void *stream)
{
    return transform_impl(nodes_dev, conns_dev, pop, d, transformed_dev, transformed_bytes, status_dev, stream, 0);
}

extern "C" int neat_transform_recurrent(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                                        void *transformed_dev, size_t transformed_bytes, uint32_t *status_dev,
                                        void *stream)
{
    return transform_impl(nodes_dev, conns_dev, pop, d, transformed_dev, transformed_bytes, status_dev, stream, 1);
}
