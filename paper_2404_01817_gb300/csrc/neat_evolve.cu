// Tensorized mutation and crossover (Section 3.2): node addition writes the
// first NaN row, removal writes NaN over a row, attribute modification
// overwrites one column, and the NEAT operators are built from these, for a
// whole population at once.  The operator hyperparameters are the
// appendix's list; the rules (declared with neat_mutate in neat.h) take
// every random number from caller-supplied inputs: uint32 words decide
// (u < T(p), T(p) = min(floor(p 2^32), 2^32)) and choose (floor(u k / 2^32)),
// float normals give the perturbations.
//
// GB300 mapping: one block per genome, working in place on the population
// tensors.  The node keys and the connections' (in, out, enabled) columns
// are kept in shared memory while the four structural steps run one after
// another (block-wide counts, rank selection by a block scan, first-free-row
// searches, and for feedforward networks a key -> row hash table and a
// breadth-first reachability sweep over the connections); the attribute step then updates every present row
// in parallel.  Crossover: one block per child, the second parent's node
// keys and (in, out) pairs in shared-memory hash tables (lowest row per key
// or pair) looked up for every row of the first parent.
#include <algorithm>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_hash.cuh"
#include "neat_trace.h"

namespace neat {
namespace {

constexpr int kEvoThreads = 256;
constexpr int kStructWords = 16;
constexpr int kStructNormals = 4;

struct MutArgs {
    float *nodes;
    float *conns;
    const uint32_t *words;
    const float *normals;
    const int32_t *new_keys;
    int N, C, I, O, Np2;
    size_t W, Z;                               // words / normals per genome
    unsigned long long t_node_add, t_node_delete, t_conn_add, t_conn_delete;
    unsigned long long t_bias_m, t_bias_mr, t_resp_m, t_resp_mr, t_w_m, t_w_mr, t_act, t_agg, t_en;
    float bias_mean, bias_std, bias_power, resp_mean, resp_std, resp_power, w_mean, w_std, w_power;
    int act_default, agg_default, n_act, n_agg;
    int act_opt[8], agg_opt[4];
    int feedforward;
};

__device__ __forceinline__ bool below(uint32_t u, unsigned long long t) { return (unsigned long long)u < t; }
__device__ __forceinline__ int choose(uint32_t u, int k)
{
    return (int)(((unsigned long long)u * (unsigned long long)k) >> 32);
}

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// Block-wide rank selection: rows [0, R) in order, `pred(row)` the
// candidates.  One block scan counts them; then, with the count known to
// every thread, the rows of ranks rank_of(total) (and rank2_of(total), when
// asked for) among the candidates are found (-1 where there are not that
// many).  Returns the first row, the second through *row2, the count
// through *total_out.
template <typename Pred, typename RankOf, typename Rank2Of>
__device__ int select_ranks(int R, Pred pred, RankOf rank_of, Rank2Of rank2_of, int *s_cnt, int *s_row,
                            int *total_out, int *row2)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (R + nt - 1) / nt;
    const int r0 = min(R, tid * chunk), r1 = min(R, r0 + chunk);
    int c = 0;
    for (int r = r0; r < r1; ++r) c += pred(r) ? 1 : 0;
    // exclusive scan of the per-thread counts: warp scan, then warp totals
    const int lane = tid & 31, warp = tid >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_cnt[warp] = incl;
    if (tid == 0) s_row[0] = s_row[1] = -1;
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < nt / 32; ++w) {
        if (w < warp) base += s_cnt[w];
        total += s_cnt[w];
    }
    const int excl = base + incl - c;
    auto find = [&](int rank, int *out) {
        if (rank >= 0 && rank >= excl && rank < excl + c) {
            int k = rank - excl;
            for (int r = r0; r < r1; ++r)
                if (pred(r) && k-- == 0) {
                    *out = r;
                    break;
                }
        }
    };
    find(rank_of(total), s_row);
    find(rank2_of(total), s_row + 1);
    __syncthreads();
    const int row = s_row[0];
    if (row2) *row2 = s_row[1];
    *total_out = total;
    __syncthreads();
    return row;
}

// The candidate of rank `rank` (-1 if there are not that many).
template <typename Pred>
__device__ int select_rank(int R, Pred pred, int rank, int *s_cnt, int *s_row, int *total_out)
{
    return select_ranks(
        R, pred, [=](int) { return rank; }, [](int) { return -1; }, s_cnt, s_row, total_out, nullptr);
}

// The candidate chosen by the random word u among all of them (-1 if none).
template <typename Pred>
__device__ int select_choose(int R, Pred pred, uint32_t u, int *s_cnt, int *s_row, int *total_out)
{
    return select_ranks(
        R, pred, [=](int total) { return total > 0 ? choose(u, total) : -1; }, [](int) { return -1; }, s_cnt,
        s_row, total_out, nullptr);
}

__global__ void __launch_bounds__(kEvoThreads) mutate_kernel(const MutArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *map = reinterpret_cast<unsigned long long *>(sm);   // [2 Np2] key -> lowest row table
    float *nk = reinterpret_cast<float *>(map + 2 * a.Np2);                  // [N] node keys
    float *ci = nk + a.N;                                                     // [C] in keys
    float *co = ci + a.C;                                                     // [C] out keys
    float *ce = co + a.C;                                                     // [C] enabled
    short *inr = reinterpret_cast<short *>(ce + a.C);                        // [C] rows of the endpoints
    short *outr = inr + a.C;
    unsigned char *seen = reinterpret_cast<unsigned char *>(outr + a.C);     // [N]
    __shared__ int s_cnt[kEvoThreads / 32], s_row[2];
    const int g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int N = a.N, C = a.C;
    float *nodes = a.nodes + (size_t)g * N * 5;
    float *conns = a.conns + (size_t)g * C * 4;
    const uint32_t *u = a.words + (size_t)g * a.W;
    const float *z = a.normals + (size_t)g * a.Z;

    for (int r = tid; r < N; r += nt) nk[r] = nodes[(size_t)r * 5];
    for (int c = tid; c < C; c += nt) {
        const float4 x = *reinterpret_cast<const float4 *>(conns + (size_t)c * 4);
        ci[c] = x.x;
        co[c] = x.y;
        ce[c] = x.z;
    }
    __syncthreads();
    auto node_present = [&](int r) { return !isnan(nk[r]); };
    auto conn_present = [&](int c) { return !(isnan(ci[c]) || isnan(co[c]) || isnan(ce[c])); };
    auto conn_free = [&](int c) { return !conn_present(c); };
    auto node_free = [&](int r) { return !node_present(r); };
    int total = 0;

    // 1. node addition: split a present enabled connection
    if (below(u[0], a.t_node_add)) {
        const float nkey = (float)__ldg(a.new_keys + g);
        auto enabled = [&](int c) { return conn_present(c) && ce[c] != 0.0f; };
        const int pick = select_choose(C, enabled, u[1], s_cnt, s_row, &total);
        const int rn = select_rank(N, node_free, 0, s_cnt, s_row, &total);
        int rb = -1;
        const int ra = select_ranks(
            C, conn_free, [](int) { return 0; }, [](int) { return 1; }, s_cnt, s_row, &total, &rb);
        bool used = false;
        for (int r = tid; r < N; r += nt) used |= node_present(r) && nk[r] == nkey;
        used = __syncthreads_or(used);
        if (pick >= 0 && rn >= 0 && ra >= 0 && rb >= 0 && !used) {
            if (tid == 0) {
                const float in = ci[pick], out = co[pick], w = conns[(size_t)pick * 4 + 3];
                ce[pick] = 0.0f;
                conns[(size_t)pick * 4 + 2] = 0.0f;
                nk[rn] = nkey;
                float *n = nodes + (size_t)rn * 5;
                n[0] = nkey;
                n[1] = a.bias_mean;
                n[2] = a.resp_mean;
                n[3] = (float)a.agg_default;
                n[4] = (float)a.act_default;
                *reinterpret_cast<float4 *>(conns + (size_t)ra * 4) = make_float4(in, nkey, 1.0f, 1.0f);
                *reinterpret_cast<float4 *>(conns + (size_t)rb * 4) = make_float4(nkey, out, 1.0f, w);
                ci[ra] = in; co[ra] = nkey; ce[ra] = 1.0f;
                ci[rb] = nkey; co[rb] = out; ce[rb] = 1.0f;
            }
        }
        __syncthreads();
    }

    // 2. node deletion: a hidden node and every connection touching it
    if (below(u[2], a.t_node_delete)) {
        const float io_end = (float)(a.I + a.O);
        auto hidden = [&](int r) { return node_present(r) && nk[r] >= io_end; };
        const int rd = select_choose(N, hidden, u[3], s_cnt, s_row, &total);
        if (total > 0) {
            const float q = nk[rd];
            for (int c = tid; c < C; c += nt)
                if (conn_present(c) && (ci[c] == q || co[c] == q)) {
                    *reinterpret_cast<float4 *>(conns + (size_t)c * 4) = make_float4(qnan(), qnan(), qnan(), qnan());
                    ci[c] = co[c] = ce[c] = qnan();
                }
            __syncthreads();
            if (tid == 0) {
                for (int j = 0; j < 5; ++j) nodes[(size_t)rd * 5 + j] = qnan();
                nk[rd] = qnan();
            }
            __syncthreads();
        }
    }

    // 3. connection addition
    if (below(u[4], a.t_conn_add)) {
        const float in_end = (float)a.I;
        auto target = [&](int r) { return node_present(r) && nk[r] >= in_end; };
        int ks = 0, kt = 0;
        const int rs = select_choose(N, node_present, u[5], s_cnt, s_row, &ks);
        const int rt = select_choose(N, target, u[6], s_cnt, s_row, &kt);
        if (ks > 0 && kt > 0) {
            const float s = nk[rs], t = nk[rt];
            const int existing =
                select_rank(C, [&](int c) { return conn_present(c) && ci[c] == s && co[c] == t; }, 0, s_cnt, s_row,
                            &total);
            if (existing >= 0) {
                if (tid == 0) {
                    ce[existing] = 1.0f;
                    conns[(size_t)existing * 4 + 2] = 1.0f;
                }
                __syncthreads();
            } else {
                bool reject = false;
                if (a.feedforward) {
                    if (s == t) {
                        reject = true;
                    } else {
                        // key -> lowest row table of the present nodes, endpoint
                        // rows of the connections, then a sweep from t until s is seen
                        const uint32_t kmask = 2u * (uint32_t)a.Np2 - 1u;
                        for (int i = tid; i < 2 * a.Np2; i += nt) map[i] = kFree;
                        __syncthreads();
                        for (int r = tid; r < N; r += nt)
                            if (node_present(r)) key_insert(map, kmask, (uint32_t)nk[r], (uint32_t)r);
                        __syncthreads();
                        for (int c = tid; c < C; c += nt) {
                            inr[c] = outr[c] = -1;
                            if (conn_present(c)) {
                                inr[c] = (short)key_row(map, kmask, (uint32_t)ci[c]);
                                outr[c] = (short)key_row(map, kmask, (uint32_t)co[c]);
                            }
                        }
                        for (int r = tid; r < N; r += nt) seen[r] = 0;
                        __syncthreads();
                        const int row_s = key_row(map, kmask, (uint32_t)s);
                        const int row_t = key_row(map, kmask, (uint32_t)t);
                        if (tid == 0) seen[row_t] = 1;
                        __syncthreads();
                        for (int it = 0; it <= N; ++it) {
                            bool changed = false;
                            for (int c = tid; c < C; c += nt) {
                                const int x = inr[c], y = outr[c];
                                if (x >= 0 && y >= 0 && seen[x] && !seen[y]) {
                                    seen[y] = 1;
                                    changed = true;
                                }
                            }
                            changed = __syncthreads_or(changed);
                            // read by one thread between two barriers, so the next
                            // pass's writes cannot race with the exit decision
                            const bool hit = __syncthreads_or(tid == 0 && seen[row_s]);
                            if (hit || !changed) break;
                        }
                        reject = seen[row_s] != 0;
                        __syncthreads();
                    }
                }
                if (!reject) {
                    const int rf = select_rank(C, conn_free, 0, s_cnt, s_row, &total);
                    if (rf >= 0 && tid == 0) {
                        const float w = fmaf(a.w_std, z[0], a.w_mean);
                        *reinterpret_cast<float4 *>(conns + (size_t)rf * 4) = make_float4(s, t, 1.0f, w);
                        ci[rf] = s; co[rf] = t; ce[rf] = 1.0f;
                    }
                    __syncthreads();
                }
            }
        }
    }

    // 4. connection deletion
    if (below(u[7], a.t_conn_delete)) {
        const int rc = select_choose(C, conn_present, u[8], s_cnt, s_row, &total);
        if (total > 0) {
            if (tid == 0) {
                *reinterpret_cast<float4 *>(conns + (size_t)rc * 4) = make_float4(qnan(), qnan(), qnan(), qnan());
                ci[rc] = co[rc] = ce[rc] = qnan();
            }
            __syncthreads();
        }
    }

    // attributes of every present row
    const float in_end = (float)a.I;
    for (int r = tid; r < N; r += nt) {
        if (!node_present(r) || nk[r] < in_end) continue;
        float *n = nodes + (size_t)r * 5;
        const uint32_t *w = u + kStructWords + 6 * (size_t)r;
        const float *zz = z + kStructNormals + 2 * (size_t)r;
        if (below(w[0], a.t_bias_m)) n[1] = fmaf(a.bias_power, zz[0], n[1]);
        else if (below(w[0], a.t_bias_mr)) n[1] = fmaf(a.bias_std, zz[0], a.bias_mean);
        if (below(w[1], a.t_resp_m)) n[2] = fmaf(a.resp_power, zz[1], n[2]);
        else if (below(w[1], a.t_resp_mr)) n[2] = fmaf(a.resp_std, zz[1], a.resp_mean);
        if (a.n_act > 0 && below(w[2], a.t_act)) n[4] = (float)a.act_opt[choose(w[3], a.n_act)];
        if (a.n_agg > 0 && below(w[4], a.t_agg)) n[3] = (float)a.agg_opt[choose(w[5], a.n_agg)];
    }
    for (int c = tid; c < C; c += nt) {
        if (!conn_present(c)) continue;
        float *x = conns + (size_t)c * 4;
        const uint32_t *w = u + kStructWords + 6 * (size_t)N + 2 * (size_t)c;
        const float zz = z[kStructNormals + 2 * (size_t)N + c];
        if (below(w[0], a.t_w_m)) x[3] = fmaf(a.w_power, zz, x[3]);
        else if (below(w[0], a.t_w_mr)) x[3] = fmaf(a.w_std, zz, a.w_mean);
        if (below(w[1], a.t_en)) x[2] = (ce[c] != 0.0f) ? 0.0f : 1.0f;
    }
}

struct CrossArgs {
    const float *nodes;
    const float *conns;
    const int32_t *parents;
    const uint32_t *words;
    float *nodes_out;
    float *conns_out;
    int pop, K, N, C, Np2, Cp2;
};

// A child whose parent index lies outside [0, pop) is written empty (every
// row NaN) by threads i, i + step, ...
__device__ __forceinline__ void write_empty_child(float *no, float4 *co, int N, int C, int lane, int step)
{
    for (int e = lane; e < N * 5; e += step) no[e] = __int_as_float(0x7fc00000);
    const float q = __int_as_float(0x7fc00000);
    for (int c = lane; c < C; c += step) co[c] = make_float4(q, q, q, q);
}

__global__ void __launch_bounds__(kEvoThreads) crossover_kernel(const CrossArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *ntab = reinterpret_cast<unsigned long long *>(sm);   // key -> lowest row of p2
    unsigned long long *ctab = ntab + 2 * a.Np2;                              // (in, out) -> lowest row of p2
    const uint32_t nmask = 2u * (uint32_t)a.Np2 - 1u, cmask = 2u * (uint32_t)a.Cp2 - 1u;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int N = a.N, C = a.C;
    const int p1 = __ldg(a.parents + 2 * k), p2 = __ldg(a.parents + 2 * k + 1);
    if (p1 < 0 || p1 >= a.pop || p2 < 0 || p2 >= a.pop) {
        write_empty_child(a.nodes_out + (size_t)k * N * 5, reinterpret_cast<float4 *>(a.conns_out + (size_t)k * C * 4),
                          N, C, tid, nt);
        return;
    }
    const float *n1 = a.nodes + (size_t)p1 * N * 5, *n2 = a.nodes + (size_t)p2 * N * 5;
    const float *c1 = a.conns + (size_t)p1 * C * 4, *c2 = a.conns + (size_t)p2 * C * 4;
    float *no = a.nodes_out + (size_t)k * N * 5;
    float *co = a.conns_out + (size_t)k * C * 4;
    const uint32_t *w = a.words + (size_t)k * (N + C);
    for (int i = tid; i < 2 * a.Np2; i += nt) ntab[i] = kFree;
    for (int i = tid; i < 2 * a.Cp2; i += nt) ctab[i] = kFree;
    __syncthreads();
    for (int r = tid; r < N; r += nt) {
        const float key = __ldg(n2 + (size_t)r * 5);
        if (is_key(key)) key_insert(ntab, nmask, (uint32_t)key, (uint32_t)r);
    }
    for (int c = tid; c < C; c += nt) {
        const float4 y = __ldg(reinterpret_cast<const float4 *>(c2) + c);
        if (is_key(y.x) && is_key(y.y) && !isnan(y.z))
            pair_row_insert(ctab, cmask, ((unsigned long long)(uint32_t)y.x << 24) | (uint32_t)y.y, (uint32_t)c);
    }
    __syncthreads();
    for (int r = tid; r < N; r += nt) {
        const float *x = n1 + (size_t)r * 5;
        float v[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = __ldg(x + j);
        if (is_key(v[0]) && w[r] >= 0x80000000u) {
            const int q = key_row(ntab, nmask, (uint32_t)v[0]);     // p2's lowest row with the key
            if (q >= 0) {
                const float *y = n2 + (size_t)q * 5;
#pragma unroll
                for (int j = 1; j < 5; ++j) v[j] = __ldg(y + j);
            }
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) no[(size_t)r * 5 + j] = v[j];
    }
    for (int c = tid; c < C; c += nt) {
        float4 x = __ldg(reinterpret_cast<const float4 *>(c1) + c);
        if (is_key(x.x) && is_key(x.y) && !isnan(x.z) && w[N + c] >= 0x80000000u) {
            const int q = pair_row(ctab, cmask, ((unsigned long long)(uint32_t)x.x << 24) | (uint32_t)x.y);
            if (q >= 0) {
                const float4 y = __ldg(reinterpret_cast<const float4 *>(c2) + q);
                x.z = y.z;
                x.w = y.w;
            }
        }
        reinterpret_cast<float4 *>(co)[c] = x;
    }
}

unsigned long long threshold(double p)
{
    if (!(p > 0.0)) return 0ull;
    const double t = std::floor(p * 4294967296.0);
    return t >= 4294967296.0 ? 4294967296ull : (unsigned long long)t;
}

int pow2_at_least(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace
}  // namespace neat

using namespace neat;

extern "C" int neat_mutation_sizes(neat_dims d, int64_t *words, int64_t *normals)
{
    if (!dims_ok(d) || !words || !normals) return invalid("neat_mutation_sizes: invalid argument");
    *words = kStructWords + 6 * (int64_t)d.max_nodes + 2 * (int64_t)d.max_conns;
    *normals = kStructNormals + 2 * (int64_t)d.max_nodes + (int64_t)d.max_conns;
    return NEAT_OK;
}

extern "C" int neat_mutate(float *nodes_dev, float *conns_dev, int32_t pop, neat_dims d, const neat_mutation *m,
                           const uint32_t *words_dev, const float *normals_dev, const int32_t *new_keys_dev,
                           void *stream)
{
    TraceRange trace_range("neat_mutate");
    clear_error();
    if (!dims_ok(d) || !m) return invalid("neat_mutate: invalid dims or config");
    if (pop < 0) return invalid("neat_mutate: pop < 0");
    if (pop == 0) return NEAT_OK;
    if (!nodes_dev || (!conns_dev && d.max_conns > 0) || !words_dev || !normals_dev || !new_keys_dev)
        return invalid("neat_mutate: null pointer");
    if (reinterpret_cast<uintptr_t>(conns_dev) & 15u) return invalid("neat_mutate: conns must be 16-byte aligned");
    if (m->n_activation_options < 0 || m->n_activation_options > 8 || m->n_aggregation_options < 0 ||
        m->n_aggregation_options > 4)
        return invalid("neat_mutate: option counts out of range");
    MutArgs a;
    a.nodes = nodes_dev;
    a.conns = conns_dev;
    a.words = words_dev;
    a.normals = normals_dev;
    a.new_keys = new_keys_dev;
    a.N = d.max_nodes;
    a.C = d.max_conns;
    a.I = d.num_inputs;
    a.O = d.num_outputs;
    a.Np2 = pow2_at_least(a.N);
    a.W = kStructWords + 6 * (size_t)a.N + 2 * (size_t)a.C;
    a.Z = kStructNormals + 2 * (size_t)a.N + (size_t)a.C;
    a.t_node_add = threshold(m->node_add);
    a.t_node_delete = threshold(m->node_delete);
    a.t_conn_add = threshold(m->conn_add);
    a.t_conn_delete = threshold(m->conn_delete);
    a.t_bias_m = threshold(m->bias_mutate_rate);
    a.t_bias_mr = threshold((double)m->bias_mutate_rate + (double)m->bias_replace_rate);
    a.t_resp_m = threshold(m->response_mutate_rate);
    a.t_resp_mr = threshold((double)m->response_mutate_rate + (double)m->response_replace_rate);
    a.t_w_m = threshold(m->weight_mutate_rate);
    a.t_w_mr = threshold((double)m->weight_mutate_rate + (double)m->weight_replace_rate);
    a.t_act = threshold(m->activation_replace_rate);
    a.t_agg = threshold(m->aggregation_replace_rate);
    a.t_en = threshold(m->enabled_mutate_rate);
    a.bias_mean = m->bias_init_mean;
    a.bias_std = m->bias_init_std;
    a.bias_power = m->bias_mutate_power;
    a.resp_mean = m->response_init_mean;
    a.resp_std = m->response_init_std;
    a.resp_power = m->response_mutate_power;
    a.w_mean = m->weight_init_mean;
    a.w_std = m->weight_init_std;
    a.w_power = m->weight_mutate_power;
    a.act_default = m->activation_default;
    a.agg_default = m->aggregation_default;
    a.n_act = m->n_activation_options;
    a.n_agg = m->n_aggregation_options;
    for (int i = 0; i < 8; ++i) a.act_opt[i] = m->activation_options[i];
    for (int i = 0; i < 4; ++i) a.agg_opt[i] = m->aggregation_options[i];
    a.feedforward = m->feedforward != 0;
    const size_t smem = 16u * (size_t)a.Np2 + 4u * (size_t)a.N + 12u * (size_t)a.C + 4u * (size_t)a.C +
                        (size_t)a.N + 16u;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(mutate_kernel), smem, "neat_mutate: shared memory");
    if (rc) return rc;
    // small genomes: two warps (its block-wide steps are barrier-bound, and
    // more genomes share an SM; 10 000 Ant-sized genomes: 0.094 -> 0.089 ms
    // against four warps)
    const int threads = (a.N <= 64 && a.C <= 256) ? 64 : kEvoThreads;
    mutate_kernel<<<pop, threads, smem, as_stream(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_mutate: launch");
    return NEAT_OK;
}

extern "C" int neat_crossover(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                              const int32_t *parents_dev, int32_t n_children, const uint32_t *words_dev,
                              float *nodes_out_dev, float *conns_out_dev, void *stream)
{
    TraceRange trace_range("neat_crossover");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_crossover: invalid dims");
    if (pop < 0 || n_children < 0) return invalid("neat_crossover: sizes must be >= 0");
    if (n_children == 0) return NEAT_OK;
    if (!nodes_dev || (!conns_dev && d.max_conns > 0) || !parents_dev || !words_dev || !nodes_out_dev ||
        (!conns_out_dev && d.max_conns > 0))
        return invalid("neat_crossover: null pointer");
    if ((reinterpret_cast<uintptr_t>(conns_dev) & 15u) || (reinterpret_cast<uintptr_t>(conns_out_dev) & 15u))
        return invalid("neat_crossover: connection tensors must be 16-byte aligned");
    CrossArgs a;
    a.nodes = nodes_dev;
    a.conns = conns_dev;
    a.parents = parents_dev;
    a.words = words_dev;
    a.nodes_out = nodes_out_dev;
    a.conns_out = conns_out_dev;
    a.pop = pop;
    a.K = n_children;
    a.N = d.max_nodes;
    a.C = d.max_conns;
    a.Np2 = pow2_at_least(a.N);
    a.Cp2 = pow2_at_least(a.C > 0 ? a.C : 1);
    const size_t smem = 16u * ((size_t)a.Np2 + (size_t)a.Cp2);
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(crossover_kernel), smem, "neat_crossover: shared memory");
    if (rc) return rc;
    const int threads = (a.N <= 64 && a.C <= 256) ? 128 : kEvoThreads;
    crossover_kernel<<<n_children, threads, smem, as_stream(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_crossover: launch");
    return NEAT_OK;
}
