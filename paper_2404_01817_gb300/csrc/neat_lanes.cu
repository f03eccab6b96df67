// Calculation stage of tensorized NEAT inference (Section 3.3) for one input
// vector per genome, run from "lane programs".
//
// Why: with one vector per genome (a control loop stepping every genome
// once per environment step) a genome is a few dozen nodes in a dependent
// chain a handful of levels deep.  A group of threads per genome that walks
// the levels leaves most of its threads idle at every level; here each
// genome gets kLaneG = 2 threads of a warp ("lanes"), each evaluating one
// node per "beat", and the 16 genomes of a warp follow one instruction
// stream compiled for them in advance.
//
// A lane program is compiled once per transform (neat_lanes_pack) from the
// records of neat_transform:
//   1. per genome (one warp each): a list schedule of width kLaneG -- beats
//      of up to kLaneG nodes whose sources are all inputs or computed in
//      earlier beats, the nodes with the longest remaining path first, each
//      beat's nodes dealt to the genome's lanes so that their edge counts
//      stay balanced;
//   2. genomes sorted by (beats, edge quads), deepest first (two stable
//      counting passes), and dealt 16 to a warp;
//   3. per warp: each beat's node entry for every lane, and each lane's
//      nodes' incoming edges in quads (4 x (weight, value offset)),
//      interleaved by lane so that every shared-memory access of the warp is
//      conflict-free.  A lane whose node has fewer quads than the beat's
//      longest reads a padding quad whose edges leave every partial
//      unchanged bit for bit (sum / mean: weight -0 on a slot holding +0,
//      so fma adds -0; product: 1 x 1; max: a NaN product, which fmaxf
//      ignores).
// Values live in a per-warp tile v[slot][32 columns] in shared memory: input
// key j in slot j, output key I + j in slot I + j, hidden nodes after them,
// then a +0 slot, a 1 slot and a slot that absorbs unused node slots.  Each
// lane reads only its own column (bank = lane); a genome's value is written
// into the columns of all its lanes (a rotation that keeps the writes
// conflict-free), and the lanes of a warp meet once per beat.
//
// Arithmetic is that of every other forward of this library: a node's edges
// (ascending connection row) dealt round-robin into four partials, partial k
// = edges k, k+4, ..., combined as ((p0 . p1) . (p2 . p3)), then the node
// rule; outputs are bit-identical to neat_forward's.
//
// Per step: lane 0 bulk-copies the warp's program (TMA) into shared memory
// and the lanes prefetch the genome's inputs into L2 before the programmatic-
// dependence wait (the loads after it then take about 0.7 us at Ant size
// instead of 1.0); after it the inputs are loaded in one round trip, the
// beats run, and the outputs are written.
#include <algorithm>
#include <cstring>
#include <vector>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_item.cuh"
#include "neat_trace.h"

namespace neat {
namespace {

// Dynamic shared memory of every kernel in this file.
extern __shared__ __align__(128) unsigned char lane_sm[];

constexpr int kLaneG = 2;                              // lanes (threads) per genome
constexpr int kLaneJ = 32 / kLaneG;                    // genomes per warp
constexpr int kLaneMaxNodes = 128;                     // positions and value slots fit a byte
constexpr uint32_t kLaneMaxRecord = 12288;             // a warp stages kLaneJ records in shared memory
constexpr uint32_t kLanesHeaderBytes = 256;
constexpr uint32_t kLanesMagic = 0x3250414eu;          // "NAP2"
constexpr uint32_t kWarpSbOff = 16u + 32u * 8u;        // warp header, lane table
constexpr uint32_t kRowBytes = 32u * 24u;              // one quad per lane: 4 weights, 4 u16 offsets
constexpr uint32_t kPadRows = 3;                       // padding quads: sum/mean, product, max
constexpr uint32_t kLaneBar = 16;                      // forward's shared memory: mbarrier, then the value tile
constexpr uint32_t kLaneError = 1u;                    // genome has an error bit: outputs NaN
constexpr uint32_t kLaneUnordered = 2u;                // no feedforward schedule (cyclic record): outputs NaN
constexpr uint32_t kWarpFast = 1u;                     // every genome of the warp is sum + tanh
constexpr uint32_t kWarpRecurrent = 2u;                // a recurrent program (neat_lanes_pack_recurrent)
constexpr uint32_t kMeasError = 1u, kMeasUnordered = 2u;

// Device header of a packed buffer.
struct LanesHeader {
    uint32_t magic;
    int32_t pop, warps;
    uint32_t max_warp_bytes;
    uint64_t warp_base, warp_stride;
    int32_t I, O, N, C;
    uint32_t unordered;      // genomes without a feedforward schedule
    uint32_t recurrent;      // 1: packed by neat_lanes_pack_recurrent
    uint32_t pad[50];
};
static_assert(sizeof(LanesHeader) == kLanesHeaderBytes, "lanes header size");

// Per-genome schedule (scratch of the pack): 16-byte head (beats, flags,
// quads per lane), then sched[beat][kLaneG] positions (0xff none), then
// vslot[position].
struct LanesGeom {
    size_t meas_off, ord_a_off, ord_b_off, scr_off, scr_stride, warp_base, warp_stride, total;
    int warps, max_sb, max_rows;
    uint32_t rec_bytes;      // reserved bytes of one record in shared memory
};

LanesGeom lanes_geom(int pop, const neat_dims &d)
{
    LanesGeom g;
    const int N = d.max_nodes;
    g.warps = (pop + kLaneJ - 1) / kLaneJ;
    g.meas_off = kLanesHeaderBytes;
    g.ord_a_off = g.meas_off + 4u * (size_t)pop;
    g.ord_b_off = g.ord_a_off + 4u * (size_t)pop;
    g.scr_off = (g.ord_b_off + 4u * (size_t)pop + 15) & ~(size_t)15;
    g.scr_stride = align16(16u + (uint32_t)(N * kLaneG + N));
    g.warp_base = (g.scr_off + g.scr_stride * (size_t)pop + 127) & ~(size_t)127;
    // beats <= non-input nodes; a lane's quads <= sum over nodes of ceil(edges / 4) <= (E + 3 n) / 4
    g.max_sb = std::max(1, N - d.num_inputs);
    g.max_rows = (int)kPadRows + (d.max_conns + 3 * g.max_sb) / 4;
    size_t s = kWarpSbOff + align16(4u * (uint32_t)g.max_sb) + 512u * (size_t)g.max_sb + (size_t)kRowBytes * g.max_rows;
    g.warp_stride = (s + 127) & ~(size_t)127;
    g.total = g.warp_base + g.warp_stride * (size_t)g.warps;
    g.rec_bytes = record_max_bytes(d.num_inputs, d.num_outputs, N, d.max_conns);
    return g;
}

bool lanes_dims_ok(const neat_dims &d)
{
    return dims_ok(d) && d.max_nodes <= kLaneMaxNodes &&
           record_max_bytes(d.num_inputs, d.num_outputs, d.max_nodes, d.max_conns) <= kLaneMaxRecord;
}

// Library error word of the lane-program kernels: a bounded wait expired.
__device__ unsigned int g_lanes_error;

// ------------------------------------------------------------- scheduling

// One warp per genome: the genome's record staged in shared memory, then
//   heights: longest path to a sink, levels in decreasing order;
//   the width-kLaneG list schedule (warp-wide arg-max per pick);
//   value slots of the positions.
// Writes the genome's schedule into the scratch and its sort key into
// meas[g] = beats | max lane quads << 8 | flags << 24.  Thread 0 of block 0
// also writes the buffer header (its reductions zero).
constexpr int kSchedWarps = 4;

// Shared memory of the schedule kernel per warp: the record, heights,
// schedule positions and the genome's scratch image; mbarriers first.
__host__ __device__ inline uint32_t sched_warp_bytes(uint32_t rec_bytes, int N, uint32_t scr_stride)
{
    return rec_bytes + align16(4u * (uint32_t)kLaneMaxNodes + (uint32_t)N) + scr_stride;
}

__global__ void __launch_bounds__(32 * kSchedWarps) lanes_sched_kernel(const uint8_t *rec, size_t stride, int pop,
                                                                      int I, int O, int N, uint32_t rec_bytes,
                                                                      uint8_t *lanes, LanesGeom geo,
                                                                      const LanesHeader hv, int recurrent)
{
    uint8_t *sm = lane_sm;
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t per_warp = sched_warp_bytes(rec_bytes, N, (uint32_t)geo.scr_stride);
    uint8_t *srec = sm + 128 + (size_t)wi * per_warp;
    uint32_t *hgt = reinterpret_cast<uint32_t *>(srec + rec_bytes);            // kLaneMaxNodes words
    uint8_t *sbv = reinterpret_cast<uint8_t *>(hgt + kLaneMaxNodes);
    uint8_t *scr = srec + rec_bytes + align16(4u * (uint32_t)kLaneMaxNodes + (uint32_t)N);   // the scratch image
    const uint32_t bar = smem_addr(sm) + 8u * (uint32_t)wi;
    if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<LanesHeader *>(lanes) = hv;
    const int g = blockIdx.x * kSchedWarps + wi;
    if (g >= pop) return;
    const uint8_t *grec = rec + (size_t)g * stride;
    uint8_t *gscr = lanes + geo.scr_off + (size_t)g * geo.scr_stride;
    uint8_t *sched = scr + 16;
    uint8_t *vslot = sched + N * kLaneG;
    uint32_t *meas = reinterpret_cast<uint32_t *>(lanes + geo.meas_off);
    const uint4 h0 = __ldg(reinterpret_cast<const uint4 *>(grec));
    if (h0.z & NEAT_G_ERROR_MASK) {
        if (lane == 0) {
            meas[g] = kMeasError << 24;
            reinterpret_cast<uint4 *>(gscr)[0] = make_uint4(0u, kMeasError, 0u, 0u);
        }
        return;
    }
    // the record into shared memory: one bulk copy, bounded wait
    const uint32_t used = min(align16(__ldg(reinterpret_cast<const uint32_t *>(grec) + 4)), rec_bytes);
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, used);
        bulk_g2s(smem_addr(srec), grec, used, bar);
    }
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait(bar, 0))) {
        if (lane == 0) {
            atomicOr(&g_lanes_error, kErrWaitExpired);
            meas[g] = kMeasUnordered << 24;          // never scheduled: NaN outputs
            reinterpret_cast<uint4 *>(gscr)[0] = make_uint4(0u, kMeasUnordered, 0u, 0u);
        }
        mbar_wait(bar, 0);                           // the copy lands before the block's memory is reused
        return;
    }
    const uint4 h1 = reinterpret_cast<const uint4 *>(srec)[1];
    const int n = (int)(h0.x & 0xffffu), nl = (int)(h0.x >> 16);
    const uint4 *nodes = reinterpret_cast<const uint4 *>(srec + kHeaderBytes);
    const uint2 *edges = reinterpret_cast<const uint2 *>(srec + h1.y);
    const uint16_t *lev = reinterpret_cast<const uint16_t *>(srec + h1.z);
    const uint16_t *io = reinterpret_cast<const uint16_t *>(srec + h1.w);

    // value slots: input key j -> j, output key I + j -> I + j, hidden positions after them in order
    for (int p = lane; p < n; p += 32) vslot[p] = 0xffu;
    __syncwarp();
    for (int j = lane; j < I + O; j += 32) vslot[io[j]] = (uint8_t)j;
    __syncwarp();
    int hidden_before = 0;
    for (int base = 0; base < n; base += 32) {
        const int p = base + lane;
        const bool hid = p < n && vslot[p] == 0xffu;
        const unsigned m = __ballot_sync(0xffffffffu, hid);
        if (hid) vslot[p] = (uint8_t)(I + O + hidden_before + __popc(m & ((1u << lane) - 1u)));
        hidden_before += __popc(m);
    }

    for (int p = lane; p < n; p += 32) sbv[p] = (nodes[p].w & 0xffu) == kInputAct ? 0xfeu : 0xffu;
    __syncwarp();
    uint32_t lane_quads[kLaneG];
    for (int k = 0; k < kLaneG; ++k) lane_quads[k] = 0;
    int b = 0;
    bool stuck = false;
    if (recurrent) {
        // every non-input node is evaluated once per iteration from the
        // previous iteration's values, so beats carry no dependences: the
        // nodes by quad count, most first (then position), dealt in turn to
        // the genome's lanes in a snake (0 1 1 0 0 1 ...), beat i / kLaneG
        // holding nodes i .. i + kLaneG - 1 of that order
        uint32_t *keys = hgt;                                  // kLaneMaxNodes sort keys
        const unsigned FULLM = 0xffffffffu, below = (1u << lane) - 1u;
        int m = 0;
        for (int base = 0; base < n; base += 32) {
            const int p = base + lane;
            const bool ev = p < n && sbv[p] == 0xffu;
            const unsigned msk = __ballot_sync(FULLM, ev);
            if (ev) keys[m + __popc(msk & below)] = ((nodes[p].z >> 16) + 3u) >> 2 << 16 | (0xffffu - (uint32_t)p);
            m += __popc(msk);
        }
        int m2 = 1;
        while (m2 < m) m2 <<= 1;
        for (int i = m + lane; i < m2; i += 32) keys[i] = 0;
        __syncwarp();
        for (int kk = 2; kk <= m2; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < m2; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t x = keys[i], y = keys[ixj];
                        if ((x < y) == ((i & kk) == 0)) {
                            keys[i] = y;
                            keys[ixj] = x;
                        }
                    }
                }
                __syncwarp();
            }
        b = (m + kLaneG - 1) / kLaneG;
        for (int i = lane; i < b * kLaneG; i += 32) sched[i] = 0xffu;
        __syncwarp();
        uint32_t q_of[kLaneG];
        for (int k = 0; k < kLaneG; ++k) q_of[k] = 0;
        for (int i = lane; i < m; i += 32) {
            const int beat = i / kLaneG, r = i % kLaneG;
            const int k = (beat & 1) ? kLaneG - 1 - r : r;
            const uint32_t key = keys[i];
            sched[beat * kLaneG + k] = (uint8_t)(0xffffu - (key & 0xffffu));
            q_of[k] += key >> 16;
        }
        for (int k = 0; k < kLaneG; ++k) lane_quads[k] = __reduce_add_sync(FULLM, q_of[k]);
        __syncwarp();
    } else {
        // heights (longest path to a sink): a node's successors lie in higher levels
        for (int p = lane; p < n; p += 32) hgt[p] = 0;
        __syncwarp();
        for (int L = nl - 1; L >= 1; --L) {
            for (int p = lev[L] + lane; p < lev[L + 1]; p += 32) {
                const uint4 ne = nodes[p];
                if ((ne.w & 0xffu) == kInputAct) continue;
                const uint32_t h = hgt[p] + 1u;
                const int eb = (int)(ne.z & 0xffffu), ec = (int)(ne.z >> 16);
                for (int e = 0; e < ec; ++e) atomicMax(&hgt[edges[eb + e].y], h);
            }
            __syncwarp();
        }

        // list schedule: each beat the kLaneG ready nodes of largest (height, -position)
        int remaining = 0;
        for (int p = lane; p < n; p += 32) remaining += sbv[p] == 0xffu;
        remaining = __reduce_add_sync(0xffffffffu, remaining);
        for (; remaining > 0; ++b) {
            uint32_t cand[kLaneMaxNodes / 32];
    #pragma unroll
            for (int c = 0; c < kLaneMaxNodes / 32; ++c) {
                const int p = lane + 32 * c;
                cand[c] = 0;
                if (p < n && sbv[p] == 0xffu) {
                    const uint32_t z = nodes[p].z;
                    const int eb = (int)(z & 0xffffu), ec = (int)(z >> 16);
                    bool ready = true;
                    for (int e = 0; e < ec && ready; ++e) {
                        const uint8_t s = sbv[edges[eb + e].y];
                        ready = s == 0xfeu || s < (uint8_t)b;
                    }
                    if (ready) cand[c] = (min(hgt[p], 0x7fffu) + 1u) << 16 | (0xffffu - (uint32_t)p);
                }
            }
            int pick[kLaneG], q[kLaneG], np = 0;
            for (int k = 0; k < kLaneG; ++k) {
                uint32_t best = 0;
    #pragma unroll
                for (int c = 0; c < kLaneMaxNodes / 32; ++c) best = max(best, cand[c]);
                best = __reduce_max_sync(0xffffffffu, best);
                if (best == 0) break;
                const int p = (int)(0xffffu - (best & 0xffffu));
    #pragma unroll
                for (int c = 0; c < kLaneMaxNodes / 32; ++c)
                    if (cand[c] == best) cand[c] = 0;
                pick[np] = p;
                q[np] = (int)((nodes[p].z >> 16) + 3u) >> 2;
                ++np;
            }
            if (np == 0 || b >= 0xfe || b >= N) {
                stuck = true;
                break;
            }
            // deal the picks to the lanes: largest first, each to the lane with
            // the fewest quads so far (every lane computes the same assignment)
            int slot_of[kLaneG];
            bool used_lane[kLaneG];
            for (int k = 0; k < kLaneG; ++k) used_lane[k] = false;
            for (int i = 0; i < np; ++i) {
                int bi = -1;
                for (int k = 0; k < np; ++k)
                    if (!used_lane[k] && (bi < 0 || q[k] > q[bi])) bi = k;
                used_lane[bi] = true;
                int lk = -1;
                for (int k = 0; k < kLaneG; ++k) {
                    bool taken = false;
                    for (int t = 0; t < i; ++t) taken |= slot_of[t] == k;
                    if (!taken && (lk < 0 || lane_quads[k] < lane_quads[lk])) lk = k;
                }
                slot_of[i] = lk;
                lane_quads[lk] += (uint32_t)q[bi];
                if (lane == 0) sched[b * kLaneG + lk] = (uint8_t)pick[bi];
                if (lane == (pick[bi] & 31)) sbv[pick[bi]] = (uint8_t)b;
            }
            if (lane == 0)
                for (int k = 0; k < kLaneG; ++k) {
                    bool taken = false;
                    for (int t = 0; t < np; ++t) taken |= slot_of[t] == k;
                    if (!taken) sched[b * kLaneG + k] = 0xffu;
                }
            remaining -= np;
            __syncwarp();
        }
    }
    if (lane == 0) {
        uint32_t mq = 0;
        for (int k = 0; k < kLaneG; ++k) mq = max(mq, lane_quads[k]);
        const uint32_t flags = stuck ? kMeasUnordered : 0u;
        const uint32_t nb = stuck ? 0u : (uint32_t)b;
        meas[g] = nb | (min(mq, 0xffffu) << 8) | (flags << 24);
        uint4 head = make_uint4(nb, flags, lane_quads[0], kLaneG > 1 ? lane_quads[1] : 0u);
        reinterpret_cast<uint4 *>(scr)[0] = head;
    }
    __syncwarp();
    for (uint32_t i = (uint32_t)lane; i < (uint32_t)geo.scr_stride / 16u; i += 32u)
        reinterpret_cast<uint4 *>(gscr)[i] = reinterpret_cast<const uint4 *>(scr)[i];
}

// One stable counting pass over 128 buckets by one block of 1024 threads:
// warp k owns a contiguous range of the input order; out = in sorted by
// bucket, ties in input order (the result is deterministic).
template <typename BucketOf>
__device__ void stable_pass(const int32_t *in, int32_t *out, int pop, BucketOf bucket_of, int (*cnt)[128],
                            int *tot)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = (pop + 31) / 32;
    const int lo = min(pop, w * R), hi = min(pop, lo + R);
    for (int i = threadIdx.x; i < 32 * 128; i += blockDim.x) cnt[i >> 7][i & 127] = 0;
    __syncthreads();
    for (int i = lo + lane; i < hi; i += 32) atomicAdd(&cnt[w][bucket_of(in[i])], 1);
    __syncthreads();
    if (threadIdx.x < 128) {               // per bucket total
        const int b = threadIdx.x;
        int s = 0;
        for (int k = 0; k < 32; ++k) s += cnt[k][b];
        tot[b] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {                // exclusive scan of the 128 totals by warp 0
        int carry = 0;
        for (int base = 0; base < 128; base += 32) {
            const int x = tot[base + lane];
            int incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            tot[base + lane] = carry + incl - x;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    if (threadIdx.x < 128) {               // start of each (warp, bucket) run
        const int b = threadIdx.x;
        int s = tot[b];
        for (int k = 0; k < 32; ++k) {
            const int c = cnt[k][b];
            cnt[k][b] = s;
            s += c;
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    for (int base = lo; base < hi; base += 32) {
        const int i = base + lane;
        const int b = i < hi ? bucket_of(in[i]) : -1 - lane;
        const unsigned m = __match_any_sync(0xffffffffu, b);
        if (i < hi) out[cnt[w][b] + __popc(m & below)] = in[i];
        __syncwarp();
        if (i < hi && lane == 31 - __clz(m)) cnt[w][b] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
}

// Genome order: most beats first, then most quads in a lane (two stable
// passes, least significant key first).  One block.
__global__ void __launch_bounds__(1024) lanes_sort_kernel(uint8_t *lanes, LanesGeom geo, int pop)
{
    __shared__ int cnt[32][128];
    __shared__ int tot[128];
    const uint32_t *meas = reinterpret_cast<const uint32_t *>(lanes + geo.meas_off);
    int32_t *oa = reinterpret_cast<int32_t *>(lanes + geo.ord_a_off);
    int32_t *ob = reinterpret_cast<int32_t *>(lanes + geo.ord_b_off);
    for (int i = threadIdx.x; i < pop; i += blockDim.x) oa[i] = i;
    __syncthreads();
    stable_pass(oa, ob, pop, [&](int g) { return 127 - (int)min((meas[g] >> 8) & 0xffffu, 127u); }, cnt, tot);
    stable_pass(ob, oa, pop, [&](int g) { return 127 - (int)min(meas[g] & 0xffu, 127u); }, cnt, tot);
}

// One warp per warp program: lane (j, k) = (lane % kLaneJ, lane / kLaneJ)
// writes the stream of slot k of genome order[kLaneJ w + j].  The warp's
// records and schedules are staged in shared memory first.  Value slots are
// slot_bytes apart in the forward's tile (128: one tile; 256: the recurrent
// forward's two tiles, interleaved by slot); warp_flags go into every warp
// header.
__global__ void __launch_bounds__(32) lanes_pack_kernel(const uint8_t *rec, size_t stride, int pop, int I, int O,
                                                        int N, uint32_t rec_bytes, uint8_t *lanes, LanesGeom geo,
                                                        uint32_t slot_bytes, uint32_t warp_flags)
{
    uint8_t *sm = lane_sm;
    const int lane = threadIdx.x;
    const int w = blockIdx.x;
    const int j = lane % kLaneJ, k = lane / kLaneJ;
    const uint32_t per = rec_bytes + (uint32_t)geo.scr_stride;
    LanesHeader *hdr = reinterpret_cast<LanesHeader *>(lanes);
    const int32_t *order = reinterpret_cast<const int32_t *>(lanes + geo.ord_a_off);
    // stage the kLaneJ genomes' schedules and records: lane jj issues the two
    // bulk copies of genome jj, all on one mbarrier (bounded wait)
    const uint32_t bar = smem_addr(lane_sm);
    uint8_t *stage = sm + 128;
    if (lane == 0) mbar_init(bar, 32);
    __syncwarp();
    {
        const int kk = w * kLaneJ + lane;
        if (lane < kLaneJ && kk < pop) {
            const int gg = order[kk];
            uint8_t *dst = stage + (size_t)lane * per;
            const uint8_t *gscr = lanes + geo.scr_off + (size_t)gg * geo.scr_stride;
            const uint8_t *grec = rec + (size_t)gg * stride;
            const uint32_t used = min(align16(__ldg(reinterpret_cast<const uint32_t *>(grec) + 4)), rec_bytes);
            mbar_arrive_expect_tx(bar, used + (uint32_t)geo.scr_stride);
            bulk_g2s(smem_addr(dst), grec, used, bar);
            bulk_g2s(smem_addr(dst + rec_bytes), gscr, (uint32_t)geo.scr_stride, bar);
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        }
    }
    const bool staged_ok = __all_sync(0xffffffffu, mbar_wait(bar, 0));
    if (!staged_ok) {
        if (lane == 0) atomicOr(&g_lanes_error, kErrWaitExpired);
        mbar_wait(bar, 0);                 // the copies land before shared memory is read or released
    }
    const int kg = w * kLaneJ + j;
    const int g = kg < pop ? order[kg] : -1;
    const uint8_t *srec = stage + (size_t)j * per;
    const uint8_t *scr = srec + rec_bytes;
    const uint4 sh = reinterpret_cast<const uint4 *>(scr)[0];
    uint32_t flags = 0;
    if (g >= 0) flags = (sh.y & kMeasError) ? kLaneError : ((sh.y & kMeasUnordered) ? kLaneUnordered : 0u);
    if (g >= 0 && !staged_ok) flags = kLaneError;     // nothing staged can be trusted: NaN outputs
    const bool ok = g >= 0 && flags == 0;
    const int nb = ok ? (int)sh.x : 0;
    const int my_quads = ok ? (int)(k == 0 ? sh.z : sh.w) : 0;
    const uint8_t *sched = scr + 16;
    const uint8_t *vslot = sched + N * kLaneG;
    const uint4 h0 = reinterpret_cast<const uint4 *>(srec)[0];
    const uint4 h1 = reinterpret_cast<const uint4 *>(srec)[1];
    const bool fast = !ok || (h0.w & 0xffffu) == kTraitsSumTanh;
    if (flags == kLaneUnordered && k == 0) atomicAdd(&hdr->unordered, 1u);
    const unsigned FULL = 0xffffffffu;
    const int nbw = (int)__reduce_max_sync(FULL, (unsigned)nb);
    const bool fast_w = __all_sync(FULL, fast);
    // a warp whose nodes all sum needs only the sum padding quad
    const uint32_t pad_rows = fast_w ? 1u : kPadRows;
    const int rows_w = (int)pad_rows + (int)__reduce_max_sync(FULL, (unsigned)my_quads);
    const uint4 *nodes = reinterpret_cast<const uint4 *>(srec + kHeaderBytes);
    const uint2 *edges = reinterpret_cast<const uint2 *>(srec + h1.y);

    uint8_t *wp = lanes + geo.warp_base + (size_t)w * geo.warp_stride;
    const uint32_t off_node = kWarpSbOff + align16(4u * (uint32_t)nbw);
    const uint32_t off_rows = off_node + 512u * (uint32_t)nbw;
    const uint32_t bytes = off_rows + kRowBytes * (uint32_t)rows_w;
    if (lane == 0) {
        reinterpret_cast<uint4 *>(wp)[0] = make_uint4((uint32_t)nbw | ((uint32_t)rows_w << 16), bytes,
                                                      (fast_w ? kWarpFast : 0u) | warp_flags, 0u);
        atomicMax(&hdr->max_warp_bytes, bytes);
    }
    reinterpret_cast<int2 *>(wp + 16)[lane] = make_int2(g, (int)flags);
    const uint32_t col4 = 4u * (uint32_t)lane;
    const uint32_t zero_off = (uint32_t)N * slot_bytes + col4, one_off = (uint32_t)(N + 1) * slot_bytes + col4;
    const uint32_t junk_off = (uint32_t)(N + 2) * slot_bytes + col4;
    uint8_t *rows = wp + off_rows + 24u * (uint32_t)lane;
    // padding quads: rows 0 (sum, mean), 1 (product), 2 (max); row 0 alone in a fast warp
    {
        const float pw[3] = {-0.0f, 1.0f, __int_as_float(0x7fc00000)};
        const uint32_t ps[3] = {zero_off, one_off, zero_off};
        for (int r = 0; r < (int)pad_rows; ++r) {
            uint2 *q = reinterpret_cast<uint2 *>(rows + (size_t)r * kRowBytes);
            q[0] = make_uint2(__float_as_uint(pw[r]), __float_as_uint(pw[r]));
            q[1] = q[0];
            q[2] = make_uint2(ps[r] | (ps[r] << 16), ps[r] | (ps[r] << 16));
        }
    }
    uint32_t *sbt = reinterpret_cast<uint32_t *>(wp + kWarpSbOff);
    uint4 *nrow = reinterpret_cast<uint4 *>(wp + off_node) + lane;
    uint32_t row = pad_rows;
    for (int b = 0; b < nbw; ++b) {
        const int p = b < nb ? sched[b * kLaneG + k] : 0xff;
        uint4 ent = make_uint4(0u, 0u, junk_off, 0u);   // unused slot: no edges, identity, sum
        uint32_t q = 0;
        if (p != 0xff) {
            const uint4 ne = nodes[p];
            const uint32_t ec = ne.z >> 16, eb = ne.z & 0xffffu;
            const uint32_t act = ne.w & 0xffu, agg = (ne.w >> 8) & 0xffu;
            const uint32_t pad = agg == kAggProduct ? 1u : (agg == kAggMax ? 2u : 0u);
            q = (ec + 3u) >> 2;
            ent = make_uint4(ne.x, ne.y, ((uint32_t)vslot[p] * slot_bytes + col4) | (row << 16),
                             ec | (act << 16) | (agg << 24) | (pad << 28));
            const float pad_w = agg == kAggProduct ? 1.0f : (agg == kAggMax ? __int_as_float(0x7fc00000) : -0.0f);
            const uint32_t pad_s = agg == kAggProduct ? one_off : zero_off;
            for (uint32_t t = 0; t < q; ++t) {
                float wv[4];
                uint32_t so[4];
                for (uint32_t e4 = 0; e4 < 4; ++e4) {
                    const uint32_t e = 4u * t + e4;
                    if (e < ec) {
                        const uint2 ed = edges[eb + e];
                        wv[e4] = __uint_as_float(ed.x);
                        so[e4] = (uint32_t)vslot[ed.y] * slot_bytes + col4;
                    } else {
                        wv[e4] = pad_w;
                        so[e4] = pad_s;
                    }
                }
                uint2 *qd = reinterpret_cast<uint2 *>(rows + (size_t)(row + t) * kRowBytes);
                qd[0] = make_uint2(__float_as_uint(wv[0]), __float_as_uint(wv[1]));
                qd[1] = make_uint2(__float_as_uint(wv[2]), __float_as_uint(wv[3]));
                qd[2] = make_uint2(so[0] | (so[1] << 16), so[2] | (so[3] << 16));
            }
            row += q;
        }
        nrow[(size_t)b * 32] = ent;
        // the beat's trips: the largest quad count, rounded up to even (the
        // forward runs trips in pairs; extra trips read padding quads)
        const uint32_t tw = __reduce_max_sync(FULL, q);
        if (lane == 0) sbt[b] = (tw + 1u) & ~1u;
    }
    // runs of beats with equal trips: the first beat of a run carries the
    // run's length in its high half (the forward dispatches once per run)
    if (lane == 0) {
        uint32_t len = 0, prev = 0xffffffffu;
        for (int b = nbw - 1; b >= 0; --b) {
            const uint32_t t = sbt[b] & 0xffffu;
            len = t == prev ? len + 1u : 1u;
            prev = t;
            sbt[b] = t | (len << 16);
        }
    }
}

// ---------------------------------------------------------------- forward

struct LanesArgs {
    const uint8_t *lanes;
    uint64_t warp_base, warp_stride;
    const float *x;          // [pop][I]
    float *y;                // [pop][O]
    int pop, I, O, N;
    uint32_t cap;            // shared-memory bytes reserved for a warp's program
};

__device__ __forceinline__ float ldv(const char *V, uint32_t off) { return *reinterpret_cast<const float *>(V + off); }

// A node's value offset in every column of its genome: kLaneG stores, the
// m-th into column (lane + m * kLaneJ) mod 32, so that the 32 lanes' m-th
// stores hit 32 different banks.
__device__ __forceinline__ void store_value(char *V, uint32_t dst, int lane, float v, uint32_t wr = 0)
{
#pragma unroll
    for (int m = 0; m < kLaneG; ++m)
        *reinterpret_cast<float *>(V + (((dst & ~127u) + wr) | ((uint32_t)((lane + m * kLaneJ) & 31) << 2))) = v;
}

// The beats of a warp program at P (shared or device memory).  FAST: every
// node sums and applies tanh.  Each beat: the lane's node entry, then T
// trips (the beat's largest quad count), trip t reading the lane's quad t or
// its padding quad; partials, node rule, the value into every column of the
// genome, and a warp barrier.
// RD / WR: byte offsets added to every value read / write (0 / 0 for the
// feedforward tile; the recurrent forward reads one of its two interleaved
// tiles and writes the other); SYNC: a warp barrier after every beat (the
// feedforward walk reads values written in earlier beats; the recurrent
// walk reads only the previous iteration's tile).
template <bool FAST, uint32_t RD = 0, uint32_t WR = 0, bool SYNC = true>
__device__ __forceinline__ void walk(const unsigned char *__restrict__ P, int nb, float *V, int lane)
{
    const uint32_t off_node = kWarpSbOff + align16(4u * (uint32_t)nb);
    const uint32_t *sbt = reinterpret_cast<const uint32_t *>(P + kWarpSbOff);
    const uint4 *nodes = reinterpret_cast<const uint4 *>(P + off_node) + lane;
    const unsigned char *R = P + off_node + 512u * (uint32_t)nb + 24u * (uint32_t)lane;
    const char *Vc = reinterpret_cast<const char *>(V);
    char *Vw = reinterpret_cast<char *>(V);
    for (int b = 0; b < nb; ++b) {
        const int T = (int)(sbt[b] & 0xffffu);
        const uint4 ne = nodes[32 * b];
        const uint32_t ec = ne.w & 0xffffu;
        const uint32_t mt = (ec + 3u) >> 2;
        const uint32_t first = ne.z >> 16;
        const uint32_t agg = FAST ? kAggSum : (ne.w >> 24) & 0xfu;
        const uint32_t pad = FAST ? 0u : ne.w >> 28;
        const float id = FAST ? 0.0f : agg_identity(agg);
        float p0 = id, p1 = id, p2 = id, p3 = id;
#pragma unroll 2
        for (int t = 0; t < T; ++t) {
            const uint32_t r = (uint32_t)t < mt ? first + (uint32_t)t : pad;
            const unsigned char *q = R + (size_t)r * kRowBytes;
            const uint2 w01 = *reinterpret_cast<const uint2 *>(q);
            const uint2 w23 = *reinterpret_cast<const uint2 *>(q + 8);
            const uint2 s = *reinterpret_cast<const uint2 *>(q + 16);
            const float v0 = ldv(Vc, (s.x & 0xffffu) + RD), v1 = ldv(Vc, (s.x >> 16) + RD);
            const float v2 = ldv(Vc, (s.y & 0xffffu) + RD), v3 = ldv(Vc, (s.y >> 16) + RD);
            if (FAST) {
                p0 = fmaf(__uint_as_float(w01.x), v0, p0);
                p1 = fmaf(__uint_as_float(w01.y), v1, p1);
                p2 = fmaf(__uint_as_float(w23.x), v2, p2);
                p3 = fmaf(__uint_as_float(w23.y), v3, p3);
            } else {
                p0 = agg_step(agg, p0, __uint_as_float(w01.x), v0);
                p1 = agg_step(agg, p1, __uint_as_float(w01.y), v1);
                p2 = agg_step(agg, p2, __uint_as_float(w23.x), v2);
                p3 = agg_step(agg, p3, __uint_as_float(w23.y), v3);
            }
        }
        float v;
        if (FAST) {
            v = node_tanh(fmaf(__uint_as_float(ne.y), (p0 + p1) + (p2 + p3), __uint_as_float(ne.x)));
        } else {
            const float a = agg_combine(agg, agg_combine(agg, p0, p1), agg_combine(agg, p2, p3));
            v = node_output(ne, agg, (ne.w >> 16) & 0xffu, ec, a);
        }
        store_value(Vw, ne.z & 0xffffu, lane, v, WR);
        if (SYNC) __syncwarp();
    }
}

// Shared-memory loads of program data (read-only once the copy has landed).
__device__ __forceinline__ uint4 lds_u4(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
// One quad (4 weights, 4 value offsets) of a lane at shared address a.
struct Quad {
    uint2 w01, w23, s;
};
__device__ __forceinline__ Quad lds_quad(uint32_t a)
{
    Quad q;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%6];\n\t"
                 "ld.shared.v2.u32 {%2, %3}, [%6+8];\n\t"
                 "ld.shared.v2.u32 {%4, %5}, [%6+16];"
                 : "=r"(q.w01.x), "=r"(q.w01.y), "=r"(q.w23.x), "=r"(q.w23.y), "=r"(q.s.x), "=r"(q.s.y)
                 : "r"(a));
    return q;
}
// Value at byte offset `off` of the tile (the tile sits kLaneBar bytes into
// the block's dynamic shared memory).
__device__ __forceinline__ float tile_ld(uint32_t off) { return *reinterpret_cast<const float *>(lane_sm + kLaneBar + off); }
__device__ __forceinline__ void tile_st(uint32_t off, float v) { *reinterpret_cast<float *>(lane_sm + kLaneBar + off) = v; }

template <uint32_t RD = 0>
__device__ __forceinline__ void fma_quad(const Quad &q, float &p0, float &p1, float &p2, float &p3)
{
    const float v0 = tile_ld((q.s.x & 0xffffu) + RD), v1 = tile_ld((q.s.x >> 16) + RD);
    const float v2 = tile_ld((q.s.y & 0xffffu) + RD), v3 = tile_ld((q.s.y >> 16) + RD);
    p0 = fmaf(__uint_as_float(q.w01.x), v0, p0);
    p1 = fmaf(__uint_as_float(q.w01.y), v1, p1);
    p2 = fmaf(__uint_as_float(q.w23.x), v2, p2);
    p3 = fmaf(__uint_as_float(q.w23.y), v3, p3);
}

// State carried from one beat to the next in the fast walk: the beat's node
// entry, its quad count and first row address, and its first kHeadRows rows
// (loaded during the previous beat, so that after the warp barrier only the
// value loads stand between a beat and its multiply-adds).
constexpr int kHeadRows = 4;
struct BeatState {
    uint4 ne;
    uint32_t mt, base;
    Quad q[kHeadRows];
};

__device__ __forceinline__ void load_beat_head(BeatState &st, uint4 ne, uint32_t ra)
{
    st.ne = ne;
    st.mt = ((ne.w & 0xffffu) + 3u) >> 2;
    st.base = ra + (ne.z >> 16) * kRowBytes;
#pragma unroll
    for (int t = 0; t < kHeadRows; ++t) st.q[t] = lds_quad((uint32_t)t < st.mt ? st.base + (uint32_t)t * kRowBytes : ra);
}

// `len` beats from beat b on, every one with T trips (T even, known at
// compile time; T = 0: nodes without edges).  Per beat: rows kHeadRows..T-1
// loaded (the first rows are in the state), then the values and the fused
// multiply-adds in trip order per partial; the next beat's head (entry and
// first rows) is loaded before the node rule, the store of the value into
// every column of the genome and the warp barrier.  A lane past its own
// quads reads the padding quad at `ra`.
template <int T, uint32_t RD = 0, uint32_t WR = 0, bool SYNC = true>
__device__ __forceinline__ void run_beats(BeatState &st, int b, int len, int nb, uint32_t na, uint32_t ra, int lane)
{
    for (int i = 0; i < len; ++i, ++b) {
        const uint4 nn = b + 1 < nb ? lds_u4(na + 512u * (uint32_t)(b + 1)) : st.ne;
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
        if (T > 0) {
            Quad q[T > 0 ? T : 1];
#pragma unroll
            for (int t = 0; t < T; ++t)
                q[t] = t < kHeadRows ? st.q[t < kHeadRows ? t : 0]
                                     : lds_quad((uint32_t)t < st.mt ? st.base + (uint32_t)t * kRowBytes : ra);
#pragma unroll
            for (int t = 0; t < T; ++t) fma_quad<RD>(q[t], p0, p1, p2, p3);
        }
        const uint4 ne = st.ne;
        load_beat_head(st, nn, ra);
        const float v = node_tanh(fmaf(__uint_as_float(ne.y), (p0 + p1) + (p2 + p3), __uint_as_float(ne.x)));
        const uint32_t dst = ne.z & 0xffffu;
#pragma unroll
        for (int m = 0; m < kLaneG; ++m)
            tile_st(((dst & ~127u) + WR) | ((uint32_t)((lane + m * kLaneJ) & 31) << 2), v);
        if (SYNC) __syncwarp();
    }
}

// The same for any even T above 8 (trip pairs in a loop after the head rows).
template <uint32_t RD = 0, uint32_t WR = 0, bool SYNC = true>
__device__ __forceinline__ void run_beats_any(BeatState &st, int T, int b, int len, int nb, uint32_t na, uint32_t ra,
                                           int lane)
{
    for (int i = 0; i < len; ++i, ++b) {
        const uint4 nn = b + 1 < nb ? lds_u4(na + 512u * (uint32_t)(b + 1)) : st.ne;
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
#pragma unroll
        for (int t = 0; t < kHeadRows; ++t)
            if (t < T) fma_quad<RD>(st.q[t], p0, p1, p2, p3);
        for (int t = kHeadRows; t < T; t += 2) {
            const Quad qa = lds_quad((uint32_t)t < st.mt ? st.base + (uint32_t)t * kRowBytes : ra);
            const Quad qb = lds_quad((uint32_t)t + 1u < st.mt ? st.base + (uint32_t)(t + 1) * kRowBytes : ra);
            fma_quad<RD>(qa, p0, p1, p2, p3);
            fma_quad<RD>(qb, p0, p1, p2, p3);
        }
        const uint4 ne = st.ne;
        load_beat_head(st, nn, ra);
        const float v = node_tanh(fmaf(__uint_as_float(ne.y), (p0 + p1) + (p2 + p3), __uint_as_float(ne.x)));
        const uint32_t dst = ne.z & 0xffffu;
#pragma unroll
        for (int m = 0; m < kLaneG; ++m)
            tile_st(((dst & ~127u) + WR) | ((uint32_t)((lane + m * kLaneJ) & 31) << 2), v);
        if (SYNC) __syncwarp();
    }
}

// The fast form (every node sums and applies tanh) of a warp program staged
// at shared address P: the beats in runs of equal trip count, one dispatch
// per run to a loop compiled for that count (one code path per loop keeps
// the hot loop compact; dispatching per beat measured ~120 cycles slower
// per beat).
template <uint32_t RD = 0, uint32_t WR = 0, bool SYNC = true>
__device__ __forceinline__ void walk_fast_staged(uint32_t P, int nb, int lane)
{
    const uint32_t off_node = kWarpSbOff + align16(4u * (uint32_t)nb);
    const uint32_t sa = P + kWarpSbOff;
    const uint32_t na = P + off_node + 16u * (uint32_t)lane;
    const uint32_t ra = P + off_node + 512u * (uint32_t)nb + 24u * (uint32_t)lane;   // row 0: padding quad
    if (nb <= 0) return;
    BeatState st;
    load_beat_head(st, lds_u4(na), ra);
    for (int b = 0; b < nb;) {
        const uint32_t e = lds_u32(sa + 4u * (uint32_t)b);
        const int T = (int)(e & 0xffffu), len = max(1, (int)(e >> 16));
        switch (T) {
        case 0: run_beats<0, RD, WR, SYNC>(st, b, len, nb, na, ra, lane); break;
        case 2: run_beats<2, RD, WR, SYNC>(st, b, len, nb, na, ra, lane); break;
        case 4: run_beats<4, RD, WR, SYNC>(st, b, len, nb, na, ra, lane); break;
        case 6: run_beats<6, RD, WR, SYNC>(st, b, len, nb, na, ra, lane); break;
        case 8: run_beats<8, RD, WR, SYNC>(st, b, len, nb, na, ra, lane); break;
        default: run_beats_any<RD, WR, SYNC>(st, T, b, len, nb, na, ra, lane);
        }
        b += len;
    }
}

// Chunks of 16 bytes a lane holds in registers while it loads inputs.
constexpr int kLaneInputChunks = 4;

// The genome's inputs into both of its columns of the value tile.  The row
// of I floats is read as the 16-byte-aligned chunks that cover it, the
// genome's two lanes taking alternate chunks (adjacent chunks of one row in
// one instruction, so that a load touches about one L1 line per genome
// instead of one per genome and float); each lane stores the words of its
// chunks into its own column and its partner's.  A chunk that reaches
// outside the input array [x, x_end) is read word by word, the row's words
// only.  Lanes without a genome store zeros.  SS: floats between value
// slots (32; 64 for the recurrent forward's two interleaved tiles, TWO: the
// inputs go into both).
template <int SS = 32, bool TWO = false>
__device__ __forceinline__ void load_inputs(const float *__restrict__ x, const float *x_end, int g, int I, int lane,
                                            float *V)
{
    if (I <= 0) return;
    const int half = lane / kLaneJ;
    const int mate = (lane + kLaneJ) & 31;
    const uintptr_t ra = reinterpret_cast<uintptr_t>(x + (size_t)(g >= 0 ? g : 0) * I);
    const float4 *w = reinterpret_cast<const float4 *>(ra & ~(uintptr_t)15);
    const int mis = g >= 0 ? (int)((ra & 15u) >> 2) : 0;
    const int nch = (mis + I + 3) >> 2;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(x), hi = reinterpret_cast<uintptr_t>(x_end);
    for (int c0 = 0; c0 < nch; c0 += 2 * kLaneInputChunks) {
        float4 r[kLaneInputChunks];
#pragma unroll
        for (int k = 0; k < kLaneInputChunks; ++k) {
            const int c = c0 + 2 * k + half;
            r[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (g >= 0 && c < nch) {
                const float4 *p = w + c;
                const uintptr_t pa = reinterpret_cast<uintptr_t>(p);
                if (pa >= lo && pa + 16u <= hi) {
                    r[k] = __ldg(p);
                } else {
                    const float *pf = reinterpret_cast<const float *>(p);
                    const int j = 4 * c - mis;
                    if (j >= 0 && j < I) r[k].x = __ldg(pf);
                    if (j + 1 >= 0 && j + 1 < I) r[k].y = __ldg(pf + 1);
                    if (j + 2 >= 0 && j + 2 < I) r[k].z = __ldg(pf + 2);
                    if (j + 3 >= 0 && j + 3 < I) r[k].w = __ldg(pf + 3);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kLaneInputChunks; ++k) {
            const int j = 4 * (c0 + 2 * k + half) - mis;
            const float e[4] = {r[k].x, r[k].y, r[k].z, r[k].w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j + q >= 0 && j + q < I) {
                    V[(j + q) * SS + lane] = e[q];
                    V[(j + q) * SS + mate] = e[q];
                    if (TWO) {
                        V[(j + q) * SS + 32 + lane] = e[q];
                        V[(j + q) * SS + 32 + mate] = e[q];
                    }
                }
        }
    }
}

// Shared memory of the forward: [0, 16) mbarrier | value tile (N + 3) x 32
// floats | program (cap bytes).  (At Ant size a block takes 36.3 KB with the
// 1 KB the runtime reserves per block: six blocks per SM.)
__host__ __device__ inline uint32_t lanes_tile_bytes(int N) { return (uint32_t)(N + 3) * 128u; }

template <bool PDL>
__global__ void __launch_bounds__(32) lanes_kernel(const LanesArgs a)
{
    unsigned char *sm = lane_sm;
    float *V = reinterpret_cast<float *>(sm + kLaneBar);
    unsigned char *sprog = sm + kLaneBar + lanes_tile_bytes(a.N);
    const int lane = threadIdx.x;
    const unsigned char *gw = a.lanes + a.warp_base + (size_t)blockIdx.x * a.warp_stride;
    const uint4 wh = __ldg(reinterpret_cast<const uint4 *>(gw));
    const int2 li = __ldg(reinterpret_cast<const int2 *>(gw + 16) + lane);
    const uint32_t bytes = wh.y;
    const bool staged = bytes <= a.cap;
    const uint32_t bar = smem_addr(sm);
    if (staged && lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(sprog), gw, bytes, bar);
    }
    const int g = li.x;
    if constexpr (PDL) {
        // the genome's inputs into L2 while the previous kernel finishes (a
        // hint: L2 is the point of coherence, no L1 line is filled)
        if (g >= 0 && a.I > 0 && lane < kLaneJ) {
            const char *p0 = reinterpret_cast<const char *>(a.x + (size_t)g * a.I);
            const char *p1 = p0 + 4u * (uint32_t)a.I - 1;
            for (const char *p = p0; p <= p1; p += 128) prefetch_l2(p);
            prefetch_l2(p1);
        }
        pdl_wait();
        pdl_trigger();
    }
    load_inputs(a.x, a.x + (size_t)a.pop * a.I, g, a.I, lane, V);
    V[a.N * 32 + lane] = 0.0f;
    V[(a.N + 1) * 32 + lane] = 1.0f;
    bool ok = true;
    if (staged) {
        __syncwarp();                    // the barrier is initialised before any lane waits on it
        ok = __all_sync(0xffffffffu, mbar_wait(bar, 0));
        if (!ok) {
            if (lane == 0) atomicOr(&g_lanes_error, kErrWaitExpired);
            mbar_wait(bar, 0);   // let the copy land before the block's memory is released
        }
    }
    const int nb = (int)(wh.x & 0xffffu);
    if (wh.z & kWarpRecurrent) ok = false;   // packed for the recurrent forward: its offsets index two tiles
    if (ok) {
        const bool fast = (wh.z & kWarpFast) != 0;
        if (staged) {
            if (fast) walk_fast_staged(smem_addr(sprog), nb, lane);
            else walk<false>(sprog, nb, V, lane);
        } else {
            if (fast) walk<true>(gw, nb, V, lane);
            else walk<false>(gw, nb, V, lane);
        }
    }
    if (g >= 0) {
        float *yg = a.y + (size_t)g * a.O;
        const bool nan_out = !ok || (li.y & (int)(kLaneError | kLaneUnordered));
        const float qnan = __int_as_float(0x7fc00000);
        if ((a.O & 3) == 0 && (reinterpret_cast<uintptr_t>(a.y) & 15u) == 0) {
            // 16-byte stores, the genome's two lanes alternating
            for (int j = 4 * (lane / kLaneJ); j < a.O; j += 4 * kLaneG) {
                const float *v = V + (a.I + j) * 32 + lane;
                *reinterpret_cast<float4 *>(yg + j) = nan_out ? make_float4(qnan, qnan, qnan, qnan)
                                                              : make_float4(v[0], v[32], v[64], v[96]);
            }
        } else {
            for (int j = lane / kLaneJ; j < a.O; j += kLaneG) yg[j] = nan_out ? qnan : V[(a.I + j) * 32 + lane];
        }
    }
}

// ------------------------------------------------------ recurrent forward

// Shared memory of the recurrent forward: [0, 16) mbarrier | two value
// tiles interleaved by slot, (N + 3) x 256 bytes (slot s of tile 0 at
// 256 s, of tile 1 at 256 s + 128) | program (cap bytes).
__host__ __device__ inline uint32_t lanes_rnn_tile_bytes(int N) { return (uint32_t)(N + 3) * 256u; }

// One iteration of a recurrent warp program: every beat reads tile RD and
// writes tile WR (byte offsets 0 / 128), no barrier between beats.
template <uint32_t RD, uint32_t WR>
__device__ __forceinline__ void rnn_iteration(const unsigned char *sprog, const unsigned char *gw, bool staged,
                                              bool fast, int nb, float *V, int lane)
{
    if (staged) {
        if (fast) walk_fast_staged<RD, WR, false>(smem_addr(sprog), nb, lane);
        else walk<false, RD, WR, false>(sprog, nb, V, lane);
    } else {
        if (fast) walk<true, RD, WR, false>(gw, nb, V, lane);
        else walk<false, RD, WR, false>(gw, nb, V, lane);
    }
    __syncwarp();      // the iteration's writes before the next one reads them
}

// K synchronous iterations of recurrent lane programs (records of
// neat_transform_recurrent packed by neat_lanes_pack_recurrent), one input
// vector per genome: non-input nodes start at 0; iteration k computes every
// non-input node from iteration k-1's values (tile k mod 2 -> tile (k+1)
// mod 2); the outputs are read from tile K mod 2.  Staging, inputs and
// error handling as in lanes_kernel.
template <bool PDL>
__global__ void __launch_bounds__(32) lanes_rnn_kernel(const LanesArgs a, int K)
{
    unsigned char *sm = lane_sm;
    float *V = reinterpret_cast<float *>(sm + kLaneBar);
    unsigned char *sprog = sm + kLaneBar + lanes_rnn_tile_bytes(a.N);
    const int lane = threadIdx.x;
    const unsigned char *gw = a.lanes + a.warp_base + (size_t)blockIdx.x * a.warp_stride;
    const uint4 wh = __ldg(reinterpret_cast<const uint4 *>(gw));
    const int2 li = __ldg(reinterpret_cast<const int2 *>(gw + 16) + lane);
    const uint32_t bytes = wh.y;
    const bool staged = bytes <= a.cap;
    const uint32_t bar = smem_addr(sm);
    if (staged && lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(sprog), gw, bytes, bar);
    }
    const int g = li.x;
    // both tiles zero (non-input nodes start at 0; the zero slots), the one
    // slots 1; tiles are block-private, so this overlaps the previous kernel
    for (int i = lane; i < (a.N + 3) * 64; i += 32) V[i] = 0.0f;
    V[(a.N + 1) * 64 + lane] = 1.0f;
    V[(a.N + 1) * 64 + 32 + lane] = 1.0f;
    if constexpr (PDL) {
        if (g >= 0 && a.I > 0 && lane < kLaneJ) {
            const char *p0 = reinterpret_cast<const char *>(a.x + (size_t)g * a.I);
            const char *p1 = p0 + 4u * (uint32_t)a.I - 1;
            for (const char *p = p0; p <= p1; p += 128) prefetch_l2(p);
            prefetch_l2(p1);
        }
        pdl_wait();
        pdl_trigger();
    }
    __syncwarp();
    load_inputs<64, true>(a.x, a.x + (size_t)a.pop * a.I, g, a.I, lane, V);
    bool ok = true;
    if (staged) {
        __syncwarp();
        ok = __all_sync(0xffffffffu, mbar_wait(bar, 0));
        if (!ok) {
            if (lane == 0) atomicOr(&g_lanes_error, kErrWaitExpired);
            mbar_wait(bar, 0);
        }
    }
    __syncwarp();
    const int nb = (int)(wh.x & 0xffffu);
    if (!(wh.z & kWarpRecurrent)) ok = false;   // a feedforward program: its offsets index one tile
    if (ok) {
        const bool fast = (wh.z & kWarpFast) != 0;
        for (int k = 0; k + 1 < K; k += 2) {
            rnn_iteration<0u, 128u>(sprog, gw, staged, fast, nb, V, lane);
            rnn_iteration<128u, 0u>(sprog, gw, staged, fast, nb, V, lane);
        }
        if (K & 1) rnn_iteration<0u, 128u>(sprog, gw, staged, fast, nb, V, lane);
    }
    if (g >= 0) {
        float *yg = a.y + (size_t)g * a.O;
        const bool nan_out = !ok || (li.y & (int)(kLaneError | kLaneUnordered));
        const float qnan = __int_as_float(0x7fc00000);
        const int fin = (K & 1) ? 32 : 0;
        for (int j = lane / kLaneJ; j < a.O; j += kLaneG) yg[j] = nan_out ? qnan : V[(a.I + j) * 64 + fin + lane];
    }
}

uint32_t default_cap(const LanesGeom &g)
{
    return (uint32_t)std::min<size_t>(g.warp_stride, 48u * 1024u);
}

int launch_lanes(const LanesArgs &a, int warps, bool pdl, cudaStream_t s)
{
    if (warps == 0) return NEAT_OK;
    const size_t smem = kLaneBar + lanes_tile_bytes(a.N) + a.cap;
    auto f = pdl ? lanes_kernel<true> : lanes_kernel<false>;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(f), smem, "neat_forward_lanes: shared memory per block");
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)warps);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, f, a);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes: launch");
    return NEAT_OK;
}

int make_lanes_args(const void *lanes, int32_t pop, const neat_dims &d, const float *x, float *y, uint32_t cap,
                    LanesArgs *out, int *warps, bool recurrent = false)
{
    if (!lanes_dims_ok(d))
        return invalid("neat_forward_lanes: invalid dims (lane programs need max_nodes <= 128 and records <= 12 KB)");
    if (pop < 0) return invalid("neat_forward_lanes: pop < 0");
    if (pop > 0 && (!lanes || !y || (d.num_inputs > 0 && !x))) return invalid("neat_forward_lanes: null pointer");
    if (reinterpret_cast<uintptr_t>(lanes) & 127u) return invalid("neat_forward_lanes: lanes must be 128-byte aligned");
    const LanesGeom g = lanes_geom(pop, d);
    LanesArgs a;
    a.lanes = static_cast<const uint8_t *>(lanes);
    a.warp_base = g.warp_base;
    a.warp_stride = g.warp_stride;
    a.x = x;
    a.y = y;
    a.pop = pop;
    a.I = d.num_inputs;
    a.O = d.num_outputs;
    a.N = d.max_nodes;
    a.cap = cap ? align16(std::min<uint32_t>(cap, (uint32_t)g.warp_stride)) : default_cap(g);
    const uint32_t tile = recurrent ? lanes_rnn_tile_bytes(a.N) : lanes_tile_bytes(a.N);
    if (kLaneBar + tile + a.cap > kMaxSmemPerBlock) return invalid("neat_forward_lanes: stage_bytes too large");
    *out = a;
    *warps = g.warps;
    return NEAT_OK;
}

int launch_lanes_rnn(const LanesArgs &a, int warps, int K, bool pdl, cudaStream_t s)
{
    if (warps == 0) return NEAT_OK;
    const size_t smem = kLaneBar + lanes_rnn_tile_bytes(a.N) + a.cap;
    auto f = pdl ? lanes_rnn_kernel<true> : lanes_rnn_kernel<false>;
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(f), smem,
                                "neat_forward_lanes_recurrent: shared memory per block");
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)warps);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, f, a, K);
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes_recurrent: launch");
    return NEAT_OK;
}

int lanes_pack_impl(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev, size_t lanes_bytes,
                    void *stream, int recurrent);

}  // namespace
}  // namespace neat

using namespace neat;

extern "C" size_t neat_lanes_bytes(int32_t pop, neat_dims d)
{
    if (!lanes_dims_ok(d) || pop < 0) return 0;
    return lanes_geom(pop, d).total;
}

extern "C" int neat_lanes_pack(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev,
                               size_t lanes_bytes, void *stream)
{
    TraceRange trace_range("neat_lanes_pack");
    return lanes_pack_impl(transformed_dev, pop, d, lanes_dev, lanes_bytes, stream, 0);
}

extern "C" int neat_lanes_pack_recurrent(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev,
                                         size_t lanes_bytes, void *stream)
{
    TraceRange trace_range("neat_lanes_pack_recurrent");
    return lanes_pack_impl(transformed_dev, pop, d, lanes_dev, lanes_bytes, stream, 1);
}

namespace neat {
namespace {
int lanes_pack_impl(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev, size_t lanes_bytes,
                    void *stream, int recurrent)
{
    clear_error();
    if (!lanes_dims_ok(d))
        return invalid("neat_lanes_pack: invalid dims (lane programs need max_nodes <= 128 and records <= 12 KB)");
    if (pop < 0) return invalid("neat_lanes_pack: pop < 0");
    if (!lanes_dev || (pop > 0 && !transformed_dev)) return invalid("neat_lanes_pack: null pointer");
    if (reinterpret_cast<uintptr_t>(lanes_dev) & 127u) return invalid("neat_lanes_pack: lanes must be 128-byte aligned");
    const LanesGeom g = lanes_geom(pop, d);
    if (lanes_bytes < g.total) {
        set_error("neat_lanes_pack: lanes buffer too small (see neat_lanes_bytes)");
        return NEAT_ENOMEM;
    }
    cudaStream_t s = as_stream(stream);
    uint8_t *L = static_cast<uint8_t *>(lanes_dev);
    LanesHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kLanesMagic;
    h.pop = pop;
    h.warps = g.warps;
    h.warp_base = g.warp_base;
    h.warp_stride = g.warp_stride;
    h.I = d.num_inputs;
    h.O = d.num_outputs;
    h.N = d.max_nodes;
    h.C = d.max_conns;
    h.recurrent = recurrent ? 1u : 0u;
    const uint8_t *rec = static_cast<const uint8_t *>(transformed_dev);
    const size_t stride = record_stride(d);
    const int N = d.max_nodes;
    const size_t sched_smem = 128u + (size_t)kSchedWarps * sched_warp_bytes(g.rec_bytes, N, (uint32_t)g.scr_stride);
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(lanes_sched_kernel), sched_smem,
                                "neat_lanes_pack: shared memory");
    if (rc) return rc;
    const size_t pack_smem = 128u + (size_t)kLaneJ * (g.rec_bytes + g.scr_stride);
    rc = allow_dynamic_smem(reinterpret_cast<const void *>(lanes_pack_kernel), pack_smem,
                            "neat_lanes_pack: shared memory");
    if (rc) return rc;
    // the header goes in as a kernel argument (also when pop is 0)
    lanes_sched_kernel<<<std::max(1, (pop + kSchedWarps - 1) / kSchedWarps), 32 * kSchedWarps, sched_smem, s>>>(
        rec, stride, pop, d.num_inputs, d.num_outputs, N, g.rec_bytes, L, g, h, recurrent);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_pack: schedule");
    if (pop == 0) return NEAT_OK;
    lanes_sort_kernel<<<1, 1024, 0, s>>>(L, g, pop);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_pack: sort");
    lanes_pack_kernel<<<g.warps, 32, pack_smem, s>>>(rec, stride, pop, d.num_inputs, d.num_outputs, N, g.rec_bytes, L,
                                                     g, recurrent ? 256u : 128u, recurrent ? kWarpRecurrent : 0u);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_pack: pack");
    return NEAT_OK;
}
}  // namespace
}  // namespace neat

extern "C" int neat_forward_lanes_recurrent(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                            int32_t iterations, float *outputs_dev, uint32_t stage_bytes, int32_t pdl,
                                            void *stream)
{
    TraceRange trace_range("neat_forward_lanes_recurrent");
    clear_error();
    if (iterations < 0) return invalid("neat_forward_lanes_recurrent: iterations < 0");
    LanesArgs a;
    int warps = 0;
    int rc = make_lanes_args(lanes_dev, pop, d, inputs_dev, outputs_dev, stage_bytes, &a, &warps, true);
    if (rc) return rc;
    return launch_lanes_rnn(a, warps, iterations, pdl != 0, as_stream(stream));
}

extern "C" int neat_lanes_query(const void *lanes_dev, neat_lanes_info *out_host)
{
    clear_error();
    if (!lanes_dev || !out_host) return invalid("neat_lanes_query: null pointer");
    LanesHeader h;
    cudaError_t e = cudaMemcpy(&h, lanes_dev, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_query: read");
    if (h.magic != kLanesMagic) return invalid("neat_lanes_query: not a packed lanes buffer");
    out_host->pop = h.pop;
    out_host->warps = h.warps;
    out_host->max_warp_bytes = h.max_warp_bytes;
    out_host->warp_stride = (uint32_t)h.warp_stride;
    out_host->unordered = h.unordered;
    out_host->recurrent = h.recurrent;
    return NEAT_OK;
}

extern "C" int neat_forward_lanes(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                  float *outputs_dev, uint32_t stage_bytes, void *stream)
{
    TraceRange trace_range("neat_forward_lanes");
    clear_error();
    LanesArgs a;
    int warps = 0;
    int rc = make_lanes_args(lanes_dev, pop, d, inputs_dev, outputs_dev, stage_bytes, &a, &warps);
    if (rc) return rc;
    return launch_lanes(a, warps, false, as_stream(stream));
}

struct neat_lanes_cache {
    const void *lanes = nullptr;
    int32_t pop = -1;
    neat_dims d = {};
    const float *x = nullptr;
    int64_t xs = 0;
    float *y = nullptr;
    int64_t ys = 0;
    int32_t steps = -1;
    uint32_t cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int neat_forward_lanes_steps(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                        int64_t in_step_stride, float *outputs_dev, int64_t out_step_stride,
                                        int32_t steps, uint32_t stage_bytes, neat_lanes_cache **cache, void *stream)
{
    TraceRange trace_range("neat_forward_lanes_steps");
    clear_error();
    if (!cache) return invalid("neat_forward_lanes_steps: null cache pointer");
    if (steps < 0) return invalid("neat_forward_lanes_steps: steps < 0");
    if (steps == 0) return NEAT_OK;
    LanesArgs a;
    int warps = 0;
    int rc = make_lanes_args(lanes_dev, pop, d, inputs_dev, outputs_dev, stage_bytes, &a, &warps);
    if (rc) return rc;
    if (steps > 1 && (in_step_stride < (int64_t)pop * d.num_inputs || out_step_stride < (int64_t)pop * d.num_outputs))
        return invalid("neat_forward_lanes_steps: step strides smaller than one step");
    if (!*cache) *cache = new neat_lanes_cache();
    neat_lanes_cache &c = **cache;
    const bool same = c.exec && c.lanes == lanes_dev && c.pop == pop && c.d.num_inputs == d.num_inputs &&
                      c.d.num_outputs == d.num_outputs && c.d.max_nodes == d.max_nodes &&
                      c.d.max_conns == d.max_conns && c.x == inputs_dev && c.xs == in_step_stride &&
                      c.y == outputs_dev && c.ys == out_step_stride && c.steps == steps && c.cap == a.cap;
    if (!same) {
        if (c.exec) {
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
        }
        cudaError_t e;
        if (!c.cap_stream) {
            e = cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes_steps: stream create");
        }
        e = cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes_steps: begin capture");
        for (int st = 0; st < steps && rc == NEAT_OK; ++st) {
            LanesArgs as = a;
            as.x = inputs_dev ? inputs_dev + (size_t)st * in_step_stride : nullptr;
            as.y = outputs_dev + (size_t)st * out_step_stride;
            rc = launch_lanes(as, warps, st > 0, c.cap_stream);   // the first step fully waits for prior work
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c.cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes_steps: end capture");
        e = cudaGraphInstantiate(&c.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c.exec = nullptr;
            return cuda_fail(e, "neat_forward_lanes_steps: instantiate");
        }
        c.lanes = lanes_dev;
        c.pop = pop;
        c.d = d;
        c.x = inputs_dev;
        c.xs = in_step_stride;
        c.y = outputs_dev;
        c.ys = out_step_stride;
        c.steps = steps;
        c.cap = a.cap;
    }
    cudaError_t e = cudaGraphLaunch(c.exec, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "neat_forward_lanes_steps: graph launch");
    return NEAT_OK;
}

extern "C" void neat_lanes_cache_destroy(neat_lanes_cache *c)
{
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

extern "C" int neat_lanes_tune(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                               int64_t in_step_stride, float *outputs_dev, int64_t out_step_stride, int32_t steps,
                               uint32_t *stage_bytes, void *stream)
{
    TraceRange trace_range("neat_lanes_tune");
    clear_error();
    if (!stage_bytes) return invalid("neat_lanes_tune: null stage_bytes");
    if (steps < 1) return invalid("neat_lanes_tune: steps < 1");
    LanesArgs a;
    int warps = 0;
    int rc = make_lanes_args(lanes_dev, pop, d, inputs_dev, outputs_dev, 0, &a, &warps);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    LanesHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, lanes_dev, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_tune: read header");
    if (h.magic != kLanesMagic || h.pop != pop) return invalid("neat_lanes_tune: lanes buffer not packed for this pop");
    const uint32_t first = align16(std::max<uint32_t>(h.max_warp_bytes, 16u));
    *stage_bytes = first;
    if (warps == 0) return NEAT_OK;
    // candidates: the smallest reservation for each number of resident
    // blocks per SM, from the most the largest program allows down to the
    // fewest that still hold one step's blocks in one wave
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t tile = lanes_tile_bytes(d.max_nodes);
    const uint32_t last = (uint32_t)std::min<uint64_t>(h.warp_stride, kMaxSmemPerBlock - kLaneBar - tile);
    rc = allow_dynamic_smem(reinterpret_cast<const void *>(lanes_kernel<true>), kLaneBar + tile + last,
                            "neat_lanes_tune: shared memory per block");
    if (rc) return rc;
    std::vector<uint32_t> caps;
    int prev = -1;
    for (uint32_t cap = first; cap <= last; cap += 128u) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lanes_kernel<true>, 32, kLaneBar + tile + cap);
        if (e != cudaSuccess) return cuda_fail(e, "neat_lanes_tune: occupancy");
        if ((int64_t)occ * sms < warps) break;
        if (occ != prev) caps.push_back(cap);
        prev = occ;
    }
    if (caps.size() <= 1) return NEAT_OK;
    // time a graph of up to 64 steps at each candidate (best of three)
    const int n = std::min(steps, 64);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 0.0f;
    for (uint32_t cap : caps) {
        neat_lanes_cache *c = nullptr;
        float ms_min = 0.0f;
        for (int r = 0; r < 4 && rc == NEAT_OK; ++r) {
            cudaEventRecord(e0, s);
            rc = neat_forward_lanes_steps(lanes_dev, pop, d, inputs_dev, in_step_stride, outputs_dev, out_step_stride,
                                          n, cap, &c, stream);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            if (rc == NEAT_OK && e != cudaSuccess) rc = cuda_fail(e, "neat_lanes_tune: timing");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && (r == 1 || ms < ms_min)) ms_min = ms;     // the first run captures the graph
        }
        neat_lanes_cache_destroy(c);
        if (rc) break;
        if (cap == caps.front() || ms_min < best_ms) {
            best_ms = ms_min;
            *stage_bytes = cap;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

namespace neat {
int read_lanes_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_lanes_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "neat_device_error: lanes word");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_lanes_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "neat_device_error: lanes word");
    }
    return NEAT_OK;
}
}  // namespace neat
