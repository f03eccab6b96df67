// Evaluation of one work item from a genome record staged in shared memory:
// the node rule of Section 3.3 applied level by level.  Shared by the
// single-population forward kernel, the multi-population persistent kernel
// and the CPPN query kernel.
#pragma once

#include "neat_device.cuh"
#include "neat_internal.h"

namespace neat {

// Barrier among the G threads of group `gi` (G a power of two).  Groups of
// at most a warp use a warp-level barrier on their lanes; larger groups use
// a named barrier (id 1 + gi) unless the group is the whole block.
__device__ __forceinline__ void group_sync(int G, int gi)
{
    if (G < 32) {
        const unsigned base = (threadIdx.x & 31u) & ~(unsigned)(G - 1);
        __syncwarp(((1u << G) - 1u) << base);
    } else if (G == 32) {
        __syncwarp();
    } else if (G == (int)blockDim.x) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gi + 1), "r"(G) : "memory");
    }
}

// Value slot of position p, column col.  T1: one column (tile 1).
template <bool T1>
__device__ __forceinline__ int vslot(uint32_t p, int lgT, int col)
{
    return T1 ? (int)p : (int)(p << lgT) + col;
}

// Aggregation order.  A node's incoming edges i = 0..ec-1 (record order) are
// dealt round-robin into four partials, partial k = edges k, k+4, k+8, ...,
// each accumulated in increasing i (sum and mean with fused multiply-add);
// the aggregate is ((p0 . p1) . (p2 . p3)) with . the aggregation's binary
// operation, divided by ec for the mean, and 0 when ec = 0.  The order is a
// function of the genome alone: one thread, two or four threads per node
// (combined through warp shuffles along the same tree) give identical bits.
enum : uint32_t { kAggSum = 0, kAggProduct = 1, kAggMax = 2, kAggMean = 3 };

__device__ __forceinline__ float agg_identity(uint32_t agg)
{
    // max starts from NaN: fmaxf(NaN, x) = x, and an all-NaN set stays NaN
    return agg == kAggProduct ? 1.0f : (agg == kAggMax ? __int_as_float(0x7fc00000) : 0.0f);
}

__device__ __forceinline__ float agg_combine(uint32_t agg, float a, float b)
{
    return agg == kAggProduct ? a * b : (agg == kAggMax ? fmaxf(a, b) : a + b);
}

__device__ __forceinline__ float agg_step(uint32_t agg, float acc, float w, float x)
{
    return agg == kAggProduct ? acc * (w * x) : (agg == kAggMax ? fmaxf(acc, w * x) : fmaf(w, x, acc));
}

// Partials k0 .. k0+nk-1 of one node for one column, combined along the tree.
template <bool T1, bool SUM>
__device__ __forceinline__ float partials(uint32_t agg, const uint2 *__restrict__ e, uint32_t ec,
                                          const float *__restrict__ v, int lgT, int col, int k0, int nk)
{
    if (SUM) agg = kAggSum;
    const float id = SUM ? 0.0f : agg_identity(agg);
    if (nk == 4) {
        float q0 = id, q1 = id, q2 = id, q3 = id;
        uint32_t i = 0;
        // not unrolled further: nodes have few edges (about 8 in the Ant
        // workload), where a second copy of the body costs more issue than
        // it saves (measured 8.27 -> 8.09 us per Ant step without it)
#pragma unroll 1
        for (; i + 4 <= ec; i += 4) {
            const uint2 t0 = e[i], t1 = e[i + 1], t2 = e[i + 2], t3 = e[i + 3];
            q0 = agg_step(agg, q0, __uint_as_float(t0.x), v[vslot<T1>(t0.y, lgT, col)]);
            q1 = agg_step(agg, q1, __uint_as_float(t1.x), v[vslot<T1>(t1.y, lgT, col)]);
            q2 = agg_step(agg, q2, __uint_as_float(t2.x), v[vslot<T1>(t2.y, lgT, col)]);
            q3 = agg_step(agg, q3, __uint_as_float(t3.x), v[vslot<T1>(t3.y, lgT, col)]);
        }
        if (i < ec) { const uint2 t = e[i]; q0 = agg_step(agg, q0, __uint_as_float(t.x), v[vslot<T1>(t.y, lgT, col)]); }
        if (i + 1 < ec) { const uint2 t = e[i + 1]; q1 = agg_step(agg, q1, __uint_as_float(t.x), v[vslot<T1>(t.y, lgT, col)]); }
        if (i + 2 < ec) { const uint2 t = e[i + 2]; q2 = agg_step(agg, q2, __uint_as_float(t.x), v[vslot<T1>(t.y, lgT, col)]); }
        return agg_combine(agg, agg_combine(agg, q0, q1), agg_combine(agg, q2, q3));
    }
    if (nk == 2) {
        float q0 = id, q1 = id;
        for (uint32_t i = (uint32_t)k0; i < ec; i += 4) {
            const uint2 t0 = e[i];
            q0 = agg_step(agg, q0, __uint_as_float(t0.x), v[vslot<T1>(t0.y, lgT, col)]);
            if (i + 1 < ec) {
                const uint2 t1 = e[i + 1];
                q1 = agg_step(agg, q1, __uint_as_float(t1.x), v[vslot<T1>(t1.y, lgT, col)]);
            }
        }
        return agg_combine(agg, q0, q1);
    }
    float q = id;
    for (uint32_t i = (uint32_t)k0; i < ec; i += 4) {
        const uint2 t = e[i];
        q = agg_step(agg, q, __uint_as_float(t.x), v[vslot<T1>(t.y, lgT, col)]);
    }
    return q;
}

// Finish a node from its combined aggregate: mean division, empty set, node rule.
__device__ __forceinline__ float node_output(const uint4 ne, uint32_t agg, uint32_t act, uint32_t ec, float a)
{
    if (agg == kAggMean) a = a / (float)ec;
    if (ec == 0) a = 0.0f;
    return activate(act, fmaf(__uint_as_float(ne.y), a, __uint_as_float(ne.x)));
}

// The four partials of one node for one column of a tile, combined along
// the tree, for a compile-time aggregation AGG (sum also serves mean): the
// operations of `partials` with all four partials, in the same order, so the
// bits are those of every other shape.  One loop per aggregation instead of
// a select among the three per edge.
template <uint32_t AGG>
__device__ __forceinline__ float partials_agg(const uint2 *__restrict__ e, uint32_t ec,
                                              const float *__restrict__ v, int lgT, int col)
{
    const float id = agg_identity(AGG);
    float q0 = id, q1 = id, q2 = id, q3 = id;
    uint32_t i = 0;
#pragma unroll 2
    for (; i + 4 <= ec; i += 4) {
        const uint2 t0 = e[i], t1 = e[i + 1], t2 = e[i + 2], t3 = e[i + 3];
        q0 = agg_step(AGG, q0, __uint_as_float(t0.x), v[vslot<false>(t0.y, lgT, col)]);
        q1 = agg_step(AGG, q1, __uint_as_float(t1.x), v[vslot<false>(t1.y, lgT, col)]);
        q2 = agg_step(AGG, q2, __uint_as_float(t2.x), v[vslot<false>(t2.y, lgT, col)]);
        q3 = agg_step(AGG, q3, __uint_as_float(t3.x), v[vslot<false>(t3.y, lgT, col)]);
    }
    if (i < ec) { const uint2 t = e[i]; q0 = agg_step(AGG, q0, __uint_as_float(t.x), v[vslot<false>(t.y, lgT, col)]); }
    if (i + 1 < ec) { const uint2 t = e[i + 1]; q1 = agg_step(AGG, q1, __uint_as_float(t.x), v[vslot<false>(t.y, lgT, col)]); }
    if (i + 2 < ec) { const uint2 t = e[i + 2]; q2 = agg_step(AGG, q2, __uint_as_float(t.x), v[vslot<false>(t.y, lgT, col)]); }
    return agg_combine(AGG, agg_combine(AGG, q0, q1), agg_combine(AGG, q2, q3));
}

// The four partials of an aggregation AGG over exactly EC edges (EC known
// at compile time), for one column, combined along the tree: straight-line
// code with the operations of `partials` in the same order (partial i mod 4,
// edges in increasing i, from the aggregation's identity), so the same bits.
template <bool T1, uint32_t AGG, int EC>
__device__ __forceinline__ float agg_edges_fixed(const uint2 *__restrict__ e, const float *__restrict__ v, int lgT,
                                                 int col)
{
    const float id = agg_identity(AGG);
    float q[4] = {id, id, id, id};
#pragma unroll
    for (int i = 0; i < EC; ++i) {
        const uint2 t = e[i];
        q[i & 3] = agg_step(AGG, q[i & 3], __uint_as_float(t.x), v[vslot<T1>(t.y, lgT, col)]);
    }
    return agg_combine(AGG, agg_combine(AGG, q[0], q[1]), agg_combine(AGG, q[2], q[3]));
}

// The aggregate of a node's ec edges for one column: one dispatch on ec
// into straight-line code for up to 8 edges (instead of a loop test per
// four edges and three remainder tests), the loop of `partials` beyond.
// For callers whose warp is on one node (a tile row of 32 or more columns,
// a CPPN's queries): lanes on different nodes would run the cases one after
// another.
template <bool T1, uint32_t AGG>
__device__ __forceinline__ float agg_edges(const uint2 *__restrict__ e, uint32_t ec, const float *__restrict__ v,
                                           int lgT, int col)
{
    switch (ec) {
    case 0: return agg_edges_fixed<T1, AGG, 0>(e, v, lgT, col);
    case 1: return agg_edges_fixed<T1, AGG, 1>(e, v, lgT, col);
    case 2: return agg_edges_fixed<T1, AGG, 2>(e, v, lgT, col);
    case 3: return agg_edges_fixed<T1, AGG, 3>(e, v, lgT, col);
    case 4: return agg_edges_fixed<T1, AGG, 4>(e, v, lgT, col);
    case 5: return agg_edges_fixed<T1, AGG, 5>(e, v, lgT, col);
    case 6: return agg_edges_fixed<T1, AGG, 6>(e, v, lgT, col);
    case 7: return agg_edges_fixed<T1, AGG, 7>(e, v, lgT, col);
    case 8: return agg_edges_fixed<T1, AGG, 8>(e, v, lgT, col);
    default:
        if (T1) return partials<T1, AGG == kAggSum>(AGG, e, ec, v, lgT, col, 0, 4);
        return partials_agg<AGG>(e, ec, v, lgT, col);
    }
}

// One whole node for one column of a tile (one thread), the aggregation
// dispatched once per node: the threads of a node row take the same branch.
template <bool FAST>
__device__ __forceinline__ void eval_node_tile(const uint4 ne, const uint2 *__restrict__ edges,
                                               float *__restrict__ v, int p, int lgT, int col)
{
    const uint32_t act = ne.w & 0xffu;
    if (act == kInputAct) return;
    const uint32_t agg = FAST ? kAggSum : ((ne.w >> 8) & 0xffu);
    const uint32_t ec = ne.z >> 16;
    const uint2 *e = edges + (ne.z & 0xffffu);
    float a;
    if (lgT >= 5) {
        // a tile row fills whole warps: every lane of a warp is on this node,
        // so the dispatch on its edge count does not diverge
        if (FAST || agg == kAggSum || agg == kAggMean) a = agg_edges<false, kAggSum>(e, ec, v, lgT, col);
        else if (agg == kAggProduct) a = agg_edges<false, kAggProduct>(e, ec, v, lgT, col);
        else a = agg_edges<false, kAggMax>(e, ec, v, lgT, col);
    } else {
        if (FAST || agg == kAggSum || agg == kAggMean) a = partials_agg<kAggSum>(e, ec, v, lgT, col);
        else if (agg == kAggProduct) a = partials_agg<kAggProduct>(e, ec, v, lgT, col);
        else a = partials_agg<kAggMax>(e, ec, v, lgT, col);
    }
    v[vslot<false>(p, lgT, col)] = FAST ? node_tanh(fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)))
                                        : node_output(ne, agg, act, ec, a);
}

// eval_node_sum with the edge sum dispatched on the edge count (the same
// bits; with no edges the sum of the four +0 partials is already the +0 of
// the empty set).  For callers whose warp is on one node.
template <bool T1>
__device__ __forceinline__ void eval_node_sum_by_count(const uint4 ne, const uint2 *__restrict__ edges,
                                                       float *__restrict__ v, int p, int lgT, int col)
{
    const uint32_t act = ne.w & 0xffu;
    if (act == kInputAct) return;
    const float a = agg_edges<T1, kAggSum>(edges + (ne.z & 0xffffu), ne.z >> 16, v, lgT, col);
    v[vslot<T1>(p, lgT, col)] = activate(act, fmaf(__uint_as_float(ne.y), a, __uint_as_float(ne.x)));
}

// The sums of a node's EC edges (EC known at compile time) for two columns
// col and col + off of the same node row: each column's operations are
// those of agg_edges_fixed<false, kAggSum, EC> in the same order (the same
// bits); the edge entries are loaded once for both.
template <int EC>
__device__ __forceinline__ float2 sum_edges_fixed2(const uint2 *__restrict__ e, const float *__restrict__ v, int lgT,
                                                   int col, int off)
{
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < EC; ++i) {
        const uint2 t = e[i];
        const int s = vslot<false>(t.y, lgT, col);
        a[i & 3] = fmaf(__uint_as_float(t.x), v[s], a[i & 3]);
        b[i & 3] = fmaf(__uint_as_float(t.x), v[s + off], b[i & 3]);
    }
    return make_float2((a[0] + a[1]) + (a[2] + a[3]), (b[0] + b[1]) + (b[2] + b[3]));
}

// Two columns of eval_node_sum_by_count: the node entry, the dispatch on the
// edge count and the edge entries shared; each column's value bit-equal to
// a one-column evaluation.  For callers whose warp is on one node.
__device__ __forceinline__ void eval_node_sum_by_count2(const uint4 ne, const uint2 *__restrict__ edges,
                                                        float *__restrict__ v, int p, int lgT, int col, int off)
{
    const uint32_t act = ne.w & 0xffu;
    if (act == kInputAct) return;
    const uint32_t ec = ne.z >> 16;
    const uint2 *e = edges + (ne.z & 0xffffu);
    float2 a;
    switch (ec) {
    case 0: a = sum_edges_fixed2<0>(e, v, lgT, col, off); break;
    case 1: a = sum_edges_fixed2<1>(e, v, lgT, col, off); break;
    case 2: a = sum_edges_fixed2<2>(e, v, lgT, col, off); break;
    case 3: a = sum_edges_fixed2<3>(e, v, lgT, col, off); break;
    case 4: a = sum_edges_fixed2<4>(e, v, lgT, col, off); break;
    case 5: a = sum_edges_fixed2<5>(e, v, lgT, col, off); break;
    case 6: a = sum_edges_fixed2<6>(e, v, lgT, col, off); break;
    case 7: a = sum_edges_fixed2<7>(e, v, lgT, col, off); break;
    case 8: a = sum_edges_fixed2<8>(e, v, lgT, col, off); break;
    default:
        a = make_float2(partials<false, true>(kAggSum, e, ec, v, lgT, col, 0, 4),
                        partials<false, true>(kAggSum, e, ec, v, lgT, col + off, 0, 4));
    }
    const int s = vslot<false>((uint32_t)p, lgT, col);
    v[s] = activate(act, fmaf(__uint_as_float(ne.y), a.x, __uint_as_float(ne.x)));
    v[s + off] = activate(act, fmaf(__uint_as_float(ne.y), a.y, __uint_as_float(ne.x)));
}

// One whole node for one column when every non-input node of the genome
// aggregates by sum (any activation): no aggregation dispatch.
template <bool T1>
__device__ __forceinline__ void eval_node_sum(const uint4 ne, const uint2 *__restrict__ edges,
                                              float *__restrict__ v, int p, int lgT, int col)
{
    const uint32_t act = ne.w & 0xffu;
    if (act == kInputAct) return;
    const uint32_t ec = ne.z >> 16;
    const float a = partials<T1, true>(kAggSum, edges + (ne.z & 0xffffu), ec, v, lgT, col, 0, 4);
    v[vslot<T1>(p, lgT, col)] = activate(act, fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)));
}

// All non-input nodes of a staged record, for the columns this thread owns.
//  Columns (T > 1): thread `lane` = (sub, col) computes column col of nodes
//  sub, sub + nsub, ... of every level, nsub = G / T.
//  One column (T1): per level, `split` threads (1, 2 or 4, at most
//  2^lg_split_max) share each node, lane = (slot, part); slots = G / split
//  nodes of the level are in flight at once.
// A group barrier separates levels.  Every thread of the group must call it.
// FAST: every non-input node uses sum aggregation and tanh activation (the
// setting of the paper's experiments), decoded once per genome.
template <bool T1, bool FAST>
__device__ __forceinline__ void walk_levels(const uint4 *srec, float *v, int G, int gi, int lane, int lgT,
                                            int lg_split_max, bool col_ok)
{
    const uint4 h0 = srec[0], h1 = srec[1];
    const int n_nodes = (int)(h0.x & 0xffffu), n_levels = (int)(h0.x >> 16);
    const uint4 *nodes = srec + 2;
    const uint2 *edges = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(srec) + h1.y);
    const uint16_t *lev = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.z);
    if (T1) {
        // the leading input positions of level 0 are skipped
        int p0 = (int)(h0.w >> 16);
        if (lg_split_max == 0) {                 // one thread per node, no shuffles
            // the node entry of a thread's first node in the next level is
            // read before the level barrier (entries do not depend on values)
            int p1 = lev[1];
            uint4 ne = (p0 + lane < n_nodes) ? nodes[p0 + lane] : make_uint4(0u, 0u, 0u, (uint32_t)kInputAct);
            for (int l = 0; l < n_levels; ++l) {
                const int p2 = lev[l + 2 <= n_levels ? l + 2 : n_levels];
                for (int p = p0 + lane; p < p1; p += G) {
                    if (p != p0 + lane) ne = nodes[p];
                    const uint32_t act = ne.w & 0xffu;
                    if (act == kInputAct) continue;
                    const uint32_t agg = FAST ? kAggSum : ((ne.w >> 8) & 0xffu);
                    const uint32_t ec = ne.z >> 16;
                    const float a = partials<true, FAST>(agg, edges + (ne.z & 0xffffu), ec, v, 0, 0, 0, 4);
                    v[p] = FAST ? node_tanh(fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)))
                                : node_output(ne, agg, act, ec, a);
                }
                const int pn = p1 + lane;
                if (pn < n_nodes) ne = nodes[pn];
                p0 = p1;
                p1 = p2;
                group_sync(G, gi);
            }
            group_sync(G, gi);
            return;
        }
        // threads per node chosen per level: 4 when the level has at most
        // G/4 nodes, 2 when at most G/2, else 1 (capped by lg_split_max)
        for (int l = 0; l < n_levels; ++l) {
            const int p1 = lev[l + 1];
            const int cnt = p1 - p0;
            const int lg_split = min(lg_split_max, (cnt * 4 <= G) ? 2 : ((cnt * 2 <= G) ? 1 : 0));
            const int split = 1 << lg_split;
            const int slot = lane >> lg_split, part = lane & (split - 1);
            const int slots = G >> lg_split;
            const int nk = 4 >> lg_split;
            const unsigned mask = ((1u << split) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(split - 1));
            for (int p = p0 + slot; p < p1; p += slots) {
                const uint4 ne = nodes[p];
                const uint32_t act = ne.w & 0xffu;
                if (act == kInputAct) continue;              // same for every part of the slot
                const uint32_t agg = FAST ? kAggSum : ((ne.w >> 8) & 0xffu);
                const uint32_t ec = ne.z >> 16;
                float a = partials<true, FAST>(agg, edges + (ne.z & 0xffffu), ec, v, 0, 0, part * nk, nk);
                for (int m = 1; m < split; m <<= 1) a = agg_combine(agg, a, __shfl_xor_sync(mask, a, m));
                if (part == 0)
                    v[p] = FAST ? node_tanh(fmaf(__uint_as_float(ne.y), ec ? a : 0.0f, __uint_as_float(ne.x)))
                                : node_output(ne, agg, act, ec, a);
            }
            p0 = p1;
            group_sync(G, gi);
        }
    } else {
        const int col = lane & ((1 << lgT) - 1);
        const int sub = lane >> lgT;
        const int nsub = G >> lgT;
        if (nsub == 1) {
            if (col_ok)
                for (int p = 0; p < n_nodes; ++p) eval_node_tile<FAST>(nodes[p], edges, v, p, lgT, col);
        } else {
            int p0 = lev[0];
            for (int l = 0; l < n_levels; ++l) {
                const int p1 = lev[l + 1];
                if (col_ok)
                    for (int p = p0 + sub; p < p1; p += nsub) eval_node_tile<FAST>(nodes[p], edges, v, p, lgT, col);
                p0 = p1;
                group_sync(G, gi);
            }
        }
    }
    group_sync(G, gi);
}

// Record traits word (header word 3): uniform activation | uniform aggregation << 8.
constexpr uint32_t kTraitsSumTanh = 1u | (0u << 8);

__device__ __forceinline__ int ilog2(int x) { return 31 - __clz(x); }

constexpr int kInputRegs = 8;   // inputs prefetched into registers per thread

// Everything of one work item after its record copy was issued by lane 0
// (mbarrier `bar` initialised and armed, `flag` set to 0, both before the
// call): inputs are read into registers while the copy is in flight, the
// group waits for the record (a bounded wait; on expiry the device error
// word gets kErrWaitExpired and the outputs NaN), scatters the inputs into
// the value tile, walks the levels and writes the outputs.
//   xb: inputs of the item [bt][I]; yb: its outputs [bt][O].
template <bool T1>
__device__ __forceinline__ void run_item(const uint4 *srec, float *v, uint32_t bar, volatile int *flag, int G,
                                         int gi, int lane, const float *__restrict__ xb, float *__restrict__ yb,
                                         int I, int O, int bt, int tile, int lg_split, unsigned int *err)
{
    const int lgT = T1 ? 0 : ilog2(tile);
    const int nx = bt * I;
    float xr[kInputRegs];
#pragma unroll
    for (int k = 0; k < kInputRegs; ++k) {
        const int i = lane + k * G;
        xr[k] = (i < nx) ? __ldg(xb + i) : 0.0f;
    }
    group_sync(G, gi);                    // barrier initialised before anyone waits on it
    if (!mbar_wait(bar, 0)) *flag = 1;
    group_sync(G, gi);
    if (*flag) {                          // uniform over the group
        if (lane == 0) atomicOr(err, kErrWaitExpired);
        mbar_wait(bar, 0);                // let the copy land before the region is reused
        for (int i = lane; i < bt * O; i += G) yb[i] = __int_as_float(0x7fc00000);
        return;
    }
    const uint4 h0 = srec[0], h1 = srec[1];
    if (h0.z & NEAT_G_ERROR_MASK) {
        for (int i = lane; i < bt * O; i += G) yb[i] = __int_as_float(0x7fc00000);
        return;
    }
    const uint16_t *io = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(srec) + h1.w);
#pragma unroll
    for (int k = 0; k < kInputRegs; ++k) {
        const int i = lane + k * G;
        if (i < nx) {
            if (T1) v[io[i]] = xr[k];
            else {
                const int b = i / I, j = i - b * I;
                v[((int)io[j] << lgT) + b] = xr[k];
            }
        }
    }
    for (int i = lane + kInputRegs * G; i < nx; i += G) {
        if (T1) v[io[i]] = __ldg(xb + i);
        else {
            const int b = i / I, j = i - b * I;
            v[((int)io[j] << lgT) + b] = __ldg(xb + i);
        }
    }
    group_sync(G, gi);
    const bool col_ok = T1 || (lane & (tile - 1)) < bt;
    if ((h0.w & 0xffffu) == kTraitsSumTanh) walk_levels<T1, true>(srec, v, G, gi, lane, lgT, lg_split, col_ok);
    else walk_levels<T1, false>(srec, v, G, gi, lane, lgT, lg_split, col_ok);
    for (int i = lane; i < bt * O; i += G) {
        if (T1) yb[i] = v[io[I + i]];
        else {
            const int b = i / O, j = i - b * O;
            yb[i] = v[((int)io[I + j] << lgT) + b];
        }
    }
}

}  // namespace neat
