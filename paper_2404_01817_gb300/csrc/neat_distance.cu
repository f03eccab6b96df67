// Genome distance for speciation (Algorithm 1 divides the population by
// distances between networks; the hyperparameters weight disjoint and
// homologous genes and set a speciation threshold).  Genes are the present
// rows of the node and connection tensors (Section 3.1); node genes are
// homologous when their keys match, connection genes when their (in key,
// out key) pairs match.  For genomes a and b
//   d = (c_d D_n + c_h S_n) / max(n_a, n_b) + (c_d D_c + c_h S_c) / max(m_a, m_b)
// with D the disjoint gene count, S the sum over homologous pairs of
// |bias diff| + |response diff| + [aggregation differs] + [activation differs]
// (nodes) or |weight diff| + [enabled differs] (connections), n and m the
// node and connection gene counts, and a term with a zero denominator 0.
//
// GB300 mapping:
//  * neat_distance_prepare: each genome's node keys and connection key pairs
//    are sorted (bitonic) and written as a compact gene record: header,
//    sorted node keys, node attributes, sorted pair keys, connection
//    attributes.  Duplicates show up as equal neighbours.  Genomes of at most
//    64 node rows and 256 connection rows take one warp each: present rows
//    are compacted by ballots, and the keys, padded to the next power of
//    two, are sorted in registers across the warp's lanes by shuffles;
//    larger genomes take one block each and sort in shared memory.
//  * neat_distance: a block stages a tile of up to 16 b-records in shared
//    memory with TMA bulk copies (one mbarrier, bounded wait) and indexes
//    them in one of three ways: for small genomes (at most 255 node and 255
//    connection genes) one open-addressing table per gene kind over the
//    union of the tile's keys, each entry holding the key's row index in
//    every staged record (one byte per record: row + 1, 0 where absent), so a gene
//    is probed once for the whole tile; otherwise one hash table per record;
//    records too large for tables are searched by binary search in their
//    sorted keys.  Its warps stream a-genomes from global memory
//    (L2-resident across blocks), two per warp: lane l of a half-warp loads
//    a's genes l, l+16, ... once each and looks every one up in all staged
//    b-records (independent lookups in flight, per-representative sums in
//    registers); the counts and sums are reduced across the half-warp along
//    a fixed tree, so every result is a function of the two genomes alone,
//    whichever form or lookup finds the homologous gene.
//  * neat_speciate: one warp per genome scans its distance row for the
//    nearest representative under the threshold.
#include <algorithm>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"

namespace neat {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kDistThreads = 256;
constexpr int kDistWarps = kDistThreads / 32;
constexpr int kMaxTile = 16;
constexpr uint32_t kGeneHeaderBytes = 16;

// Gene record offsets for n node genes and m connection genes.
struct GeneLayout {
    uint32_t nkey, nattr, ckey, cattr, used;
};

__host__ __device__ inline GeneLayout gene_layout(uint32_t n, uint32_t m)
{
    GeneLayout L;
    L.nkey = kGeneHeaderBytes;
    L.nattr = L.nkey + align16(4u * n);
    L.ckey = L.nattr + 16u * n;
    L.cattr = L.ckey + 8u * m;
    L.used = align16(L.cattr + 8u * m);
    return L;
}

inline size_t gene_stride(const neat_dims &d)
{
    const size_t b = gene_layout((uint32_t)d.max_nodes, (uint32_t)d.max_conns).used;
    return (b + 127) & ~(size_t)127;
}

struct PrepArgs {
    const float *nodes;
    const float *conns;
    uint8_t *out;
    uint32_t *status;
    size_t stride;
    int N, C, Np2, Cp2;
    int pop;
};

constexpr int kPrepWarpGenomes = 4;   // genomes (one per warp) per block of the warp form
constexpr int kWarpMaxNodes = 64, kWarpMaxConns = 256;

__global__ void __launch_bounds__(kPrepThreads) prepare_kernel(const PrepArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *nk = reinterpret_cast<unsigned long long *>(sm);   // key << 32 | row
    unsigned long long *ck = nk + a.Np2;                                     // (in << 24 | out) << 13 | row
    __shared__ unsigned int st;
    __shared__ int n_nodes, n_conns;
    const int g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const float *nd = a.nodes + (size_t)g * a.N * 5;
    const float4 *cn = reinterpret_cast<const float4 *>(a.conns + (size_t)g * a.C * 4);
    if (tid == 0) {
        st = 0;
        n_nodes = 0;
        n_conns = 0;
    }
    __syncthreads();
    unsigned int lst = 0;
    for (int r = tid; r < a.Np2; r += nt) {
        unsigned long long v = ~0ull;
        if (r < a.N) {
            const float k = __ldg(nd + (size_t)r * 5);
            if (!isnan(k)) {
                if (is_key(k)) {
                    v = ((unsigned long long)(uint32_t)k << 32) | (unsigned)r;
                    atomicAdd(&n_nodes, 1);
                } else {
                    lst |= NEAT_G_BADKEY;
                }
            }
        }
        nk[r] = v;
    }
    for (int c = tid; c < a.Cp2; c += nt) {
        unsigned long long v = ~0ull;
        if (c < a.C) {
            const float4 row = __ldg(cn + c);
            if (!(isnan(row.x) || isnan(row.y) || isnan(row.z))) {
                if (is_key(row.x) && is_key(row.y)) {
                    const unsigned long long pair = ((unsigned long long)(uint32_t)row.x << 24) | (uint32_t)row.y;
                    v = (pair << 13) | (unsigned)c;
                    atomicAdd(&n_conns, 1);
                } else {
                    lst |= NEAT_G_BADKEY;
                }
            }
        }
        ck[c] = v;
    }
    if (lst) atomicOr(&st, lst);
    __syncthreads();
    bitonic_sort(nk, a.Np2);
    bitonic_sort(ck, a.Cp2);
    const int n = n_nodes, m = n_conns;
    lst = 0;
    for (int i = tid + 1; i < n; i += nt)
        if ((nk[i] >> 32) == (nk[i - 1] >> 32)) lst |= NEAT_G_DUPKEY;
    for (int i = tid + 1; i < m; i += nt)
        if ((ck[i] >> 13) == (ck[i - 1] >> 13)) lst |= NEAT_G_DUPCONN;
    if (lst) atomicOr(&st, lst);
    __syncthreads();
    const uint32_t status = st;
    uint8_t *rec = a.out + (size_t)g * a.stride;
    if (status) {
        if (tid == 0) {
            *reinterpret_cast<uint4 *>(rec) = make_uint4(0u, 0u, status, kGeneHeaderBytes);
            if (a.status) a.status[g] = status;
        }
        return;
    }
    const GeneLayout L = gene_layout((uint32_t)n, (uint32_t)m);
    uint32_t *okey = reinterpret_cast<uint32_t *>(rec + L.nkey);
    uint4 *oattr = reinterpret_cast<uint4 *>(rec + L.nattr);
    for (int j = tid; j < n; j += nt) {
        const unsigned long long v = nk[j];
        const float *row = nd + (size_t)(v & 0xffffffffu) * 5;
        okey[j] = (uint32_t)(v >> 32);
        oattr[j] = make_uint4(__float_as_uint(__ldg(row + 1)), __float_as_uint(__ldg(row + 2)),
                              __float_as_uint(__ldg(row + 3)), __float_as_uint(__ldg(row + 4)));
    }
    for (int j = n + tid; j < (int)((L.nattr - L.nkey) / 4); j += nt) okey[j] = 0xffffffffu;   // pad
    unsigned long long *ockey = reinterpret_cast<unsigned long long *>(rec + L.ckey);
    float2 *ocattr = reinterpret_cast<float2 *>(rec + L.cattr);
    for (int j = tid; j < m; j += nt) {
        const unsigned long long v = ck[j];
        const float4 row = __ldg(cn + (v & 0x1fffu));
        ockey[j] = v >> 13;
        ocattr[j] = make_float2(row.w, row.z != 0.0f ? 1.0f : 0.0f);
    }
    if (tid == 0) {
        *reinterpret_cast<uint4 *>(rec) = make_uint4((uint32_t)n, (uint32_t)m, 0u, L.used);
        if (a.status) a.status[g] = 0u;
    }
}

// Ascending bitonic sort of the 32 R keys a warp holds, key e in lane e % 32,
// register e / 32 (registers R.. of v are left alone).  A compare-exchange
// partner 32 j' or more positions away sits in another register of the same
// lane; a nearer one in another lane at the same register.
template <int R, typename T, int NR>
__device__ __forceinline__ void warp_bitonic(T (&v)[NR], int lane)
{
    static_assert(R <= NR, "registers");
    constexpr int n2 = 32 * R;
    for (int k = 2; k <= n2; k <<= 1) {
#pragma unroll
        for (int jr = R / 2; jr >= 1; jr >>= 1) {
            if (32 * jr <= (k >> 1)) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!(r & jr)) {
                        const bool up = (((r << 5) | lane) & k) == 0;
                        const T x = v[r], y = v[r | jr];
                        if ((x > y) == up) {
                            v[r] = y;
                            v[r | jr] = x;
                        }
                    }
                }
            }
        }
        for (int j = min(k >> 1, 16); j >= 1; j >>= 1) {
            const bool lower = (lane & j) == 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T x = v[r];
                const T y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool up = (((r << 5) | lane) & k) == 0;
                // in an ascending run the lower position keeps the smaller key
                v[r] = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
            }
        }
    }
}

template <typename T, int NR>
__device__ __forceinline__ void warp_bitonic_any(T (&v)[NR], int regs, int lane)
{
    if (regs <= 1) warp_bitonic<1>(v, lane);
    else if (regs <= 2) warp_bitonic<(NR < 2 ? NR : 2)>(v, lane);
    else if (regs <= 4) warp_bitonic<(NR < 4 ? NR : 4)>(v, lane);
    else warp_bitonic<NR>(v, lane);
}

// True in some lane when two of the first `count` sorted keys agree in the
// bits above `shift`.
template <typename T, int NR>
__device__ __forceinline__ bool warp_has_equal_neighbours(const T (&v)[NR], int regs, int count, int shift, int lane)
{
    bool dup = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r < regs) {
            const T up1 = __shfl_up_sync(0xffffffffu, v[r], 1);
            const T last = r ? __shfl_sync(0xffffffffu, v[r ? r - 1 : 0], 31) : T(0);
            const T prev = lane ? up1 : last;
            const int e = (r << 5) | lane;
            if (e >= 1 && e < count && (v[r] >> shift) == (prev >> shift)) dup = true;
        }
    }
    return dup;
}

// Gene records, one warp per genome of at most 64 node rows and 256
// connection rows; the records are those of prepare_kernel.
__global__ void __launch_bounds__(32 * kPrepWarpGenomes) prepare_warp_kernel(const PrepArgs a)
{
    __shared__ unsigned long long s_keys[kPrepWarpGenomes][kWarpMaxNodes + kWarpMaxConns];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kPrepWarpGenomes + warp;
    if (g >= a.pop) return;
    unsigned long long *nk = s_keys[warp], *ck = nk + kWarpMaxNodes;
    const float *nd = a.nodes + (size_t)g * a.N * 5;
    const float4 *cn = reinterpret_cast<const float4 *>(a.conns + (size_t)g * a.C * 4);
    const uint32_t below = (1u << lane) - 1u;
    uint32_t st = 0;
    // present rows, compacted in row order (the sort makes the order moot)
    int n = 0, m = 0;
    uint32_t wide = 0;   // key bits at or above 2^12 in any connection
    for (int base = 0; base < a.N; base += 32) {
        const int r = base + lane;
        bool ok = false;
        unsigned long long v = 0;
        if (r < a.N) {
            const float k = __ldg(nd + (size_t)r * 5);
            if (!isnan(k)) {
                if (is_key(k)) {
                    ok = true;
                    v = ((unsigned long long)(uint32_t)k << 32) | (unsigned)r;
                } else {
                    st |= NEAT_G_BADKEY;
                }
            }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, ok);
        if (ok) nk[n + __popc(b & below)] = v;
        n += __popc(b);
    }
    for (int base = 0; base < a.C; base += 32) {
        const int c = base + lane;
        bool ok = false;
        unsigned long long v = 0;
        if (c < a.C) {
            const float4 row = __ldg(cn + c);
            if (!(isnan(row.x) || isnan(row.y) || isnan(row.z))) {
                if (is_key(row.x) && is_key(row.y)) {
                    ok = true;
                    const unsigned long long pair = ((unsigned long long)(uint32_t)row.x << 24) | (uint32_t)row.y;
                    v = (pair << 13) | (unsigned)c;
                    wide |= ((uint32_t)row.x | (uint32_t)row.y) >> 12;
                } else {
                    st |= NEAT_G_BADKEY;
                }
            }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, ok);
        if (ok) ck[m + __popc(b & below)] = v;
        m += __popc(b);
    }
    __syncwarp();
    // n <= 64 and m <= 256 present rows: 2 and 8 registers a lane at most.
    // Sort keys in 32 bits where they fit, in the order of the 64-bit ones:
    // node key << 6 | row (keys below 2^24, rows below 64), and for
    // connections whose keys are all below 2^12, in << 20 | out << 8 | row.
    uint32_t vn[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = (r << 5) | lane;
        vn[r] = e < n ? (uint32_t)(nk[e] >> 32) << 6 | (uint32_t)(nk[e] & 63u) : 0xffffffffu;
    }
    const int rn = (n + 31) >> 5, rc = (m + 31) >> 5;   // registers in use (0 for none)
    warp_bitonic_any(vn, rn, lane);
    if (warp_has_equal_neighbours(vn, rn, n, 6, lane)) st |= NEAT_G_DUPKEY;
    const bool narrow = __reduce_or_sync(0xffffffffu, wide) == 0u;
    // the sorted keys go back to the warp's shared arrays (the register
    // arrays end with the sort)
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = (r << 5) | lane;
        if (e < n) nk[e] = vn[r];
    }
    if (narrow) {
        uint32_t v32[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = (r << 5) | lane;
            const unsigned long long v = e < m ? ck[e] : 0ull;
            const uint32_t in = (uint32_t)(v >> 37), out = (uint32_t)(v >> 13) & 0xfffu;
            v32[r] = e < m ? in << 20 | out << 8 | (uint32_t)(v & 0xffu) : 0xffffffffu;
        }
        warp_bitonic_any(v32, rc, lane);
        if (warp_has_equal_neighbours(v32, rc, m, 8, lane)) st |= NEAT_G_DUPCONN;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = (r << 5) | lane;
            const unsigned long long pair = (unsigned long long)(v32[r] >> 20) << 24 | ((v32[r] >> 8) & 0xfffu);
            if (e < m) ck[e] = pair << 13 | (v32[r] & 0xffu);
        }
    } else {
        unsigned long long vc[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = (r << 5) | lane;
            vc[r] = e < m ? ck[e] : ~0ull;
        }
        warp_bitonic_any(vc, rc, lane);
        if (warp_has_equal_neighbours(vc, rc, m, 13, lane)) st |= NEAT_G_DUPCONN;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = (r << 5) | lane;
            if (e < m) ck[e] = vc[r];
        }
    }
    __syncwarp();
    st = __reduce_or_sync(0xffffffffu, st);
    uint8_t *rec = a.out + (size_t)g * a.stride;
    if (st) {
        if (lane == 0) {
            *reinterpret_cast<uint4 *>(rec) = make_uint4(0u, 0u, st, kGeneHeaderBytes);
            if (a.status) a.status[g] = st;
        }
        return;
    }
    const GeneLayout L = gene_layout((uint32_t)n, (uint32_t)m);
    uint32_t *okey = reinterpret_cast<uint32_t *>(rec + L.nkey);
    uint4 *oattr = reinterpret_cast<uint4 *>(rec + L.nattr);
    for (int e = lane; e < n; e += 32) {
        const uint32_t v = (uint32_t)nk[e];
        const float *row = nd + (size_t)(v & 63u) * 5;
        okey[e] = v >> 6;
        oattr[e] = make_uint4(__float_as_uint(__ldg(row + 1)), __float_as_uint(__ldg(row + 2)),
                              __float_as_uint(__ldg(row + 3)), __float_as_uint(__ldg(row + 4)));
    }
    for (int j = n + lane; j < (int)((L.nattr - L.nkey) / 4); j += 32) okey[j] = 0xffffffffu;   // pad
    unsigned long long *ockey = reinterpret_cast<unsigned long long *>(rec + L.ckey);
    float2 *ocattr = reinterpret_cast<float2 *>(rec + L.cattr);
    for (int e = lane; e < m; e += 32) {
        const unsigned long long v = ck[e];
        const float4 row = __ldg(cn + (v & 0x1fffu));
        ockey[e] = v >> 13;
        ocattr[e] = make_float2(row.w, row.z != 0.0f ? 1.0f : 0.0f);
    }
    if (lane == 0) {
        *reinterpret_cast<uint4 *>(rec) = make_uint4((uint32_t)n, (uint32_t)m, 0u, L.used);
        if (a.status) a.status[g] = 0u;
    }
}

struct DistArgs {
    const uint8_t *a;
    const uint8_t *b;
    size_t stride;
    int pa, pb;
    float cd, ch;
    float *out;
    long long ldo;
    int tile;             // b-records per block
    int a_per_block;      // a-genomes per block
    uint32_t slot_bytes;  // shared memory per staged b-record: the record, then (kHash) its two tables
    uint32_t lgn, lgc;    // log2 of the node / connection hash-table capacities (kHash, kUnion)
    uint32_t union_off;   // offset of the two union tables after the staged records (kUnion)
};

// How a block finds a-genes in its staged b-records.
constexpr int kSearch = 0;   // binary search in each record's sorted keys
constexpr int kHash = 1;     // one hash table per record
constexpr int kUnion = 2;    // one table over the tile's keys, row indices of every record per entry

__device__ unsigned int g_distance_error;

constexpr unsigned long long kEmpty = ~0ull;

// Index of `key` among n ascending keys, or -1.
template <typename K>
__device__ __forceinline__ int find_key(const K *keys, int n, K key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

// Open addressing with linear probing.  Node table entries: key << 32 |
// index; connection table entries: (in << 24 | out) << 13 | index; kEmpty
// marks a free slot.  Capacities are powers of two above 1.5x the gene
// count, so a probe sequence always reaches a free slot.
__device__ __forceinline__ uint32_t slot_of(uint32_t x, uint32_t lg) { return (x * 0x9E3779B1u) >> (32u - lg); }

__device__ __forceinline__ uint32_t fold_pair(unsigned long long pair)
{
    return (uint32_t)pair * 0x85EBCA6Bu ^ (uint32_t)(pair >> 32);
}

__device__ __forceinline__ void table_insert(unsigned long long *tab, uint32_t lg, uint32_t slot,
                                             unsigned long long v)
{
    const uint32_t mask = (1u << lg) - 1u;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        if (atomicCAS(tab + slot, kEmpty, v) == kEmpty) return;
        slot = (slot + 1u) & mask;
    }
}

__device__ __forceinline__ int node_lookup(const unsigned long long *tab, uint32_t lg, uint32_t key)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(key, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = tab[s];
        const uint32_t k = (uint32_t)(v >> 32);        // all ones in a free slot, never a key
        if (k == key) return (int)(uint32_t)v;
        if (k == 0xffffffffu) return -1;
        s = (s + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ int conn_lookup(const unsigned long long *tab, uint32_t lg, unsigned long long pair)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(fold_pair(pair), lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = tab[s];
        if (v == kEmpty) return -1;
        if ((v >> 13) == pair) return (int)(v & 0x1fffu);
        s = (s + 1u) & mask;
    }
    return -1;
}

// Union tables (kUnion) of 16-byte entries: node entries {key, row indices
// in records 0-3, in records 4-7, unused}, connection entries {pair (64
// bits), row indices in records 0-3, in records 4-7}, one index byte per
// staged record holding row + 1 (rows 0-254), 0 where the record lacks the
// gene.  A free entry has key 0xFFFFFFFF (keys are below 2^24) or pair ~0
// (pairs have 48 bits) and zero index bytes.  Linear probing; capacities
// are powers of two above 1.25x the largest union a tile can have, so a
// probe sequence always reaches a free entry.  Rows of one record are
// distinct per key (duplicates make an error record, which holds no genes),
// so each index byte has one writer.
constexpr int kUnionMaxTile = 8;

__device__ __forceinline__ void union_insert_node(uint4 *tab, uint32_t lg, uint32_t key, int t, uint32_t row)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(key, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t old = atomicCAS(&tab[s].x, 0xffffffffu, key);
        if (old == 0xffffffffu || old == key) {
            reinterpret_cast<unsigned char *>(tab + s)[4 + t] = (unsigned char)(row + 1u);
            return;
        }
        s = (s + 1u) & mask;
    }
}

__device__ __forceinline__ void union_insert_conn(uint4 *tab, uint32_t lg, unsigned long long pair, int t,
                                                  uint32_t row)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(fold_pair(pair), lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long *>(tab + s), kEmpty, pair);
        if (old == kEmpty || old == pair) {
            reinterpret_cast<unsigned char *>(tab + s)[8 + t] = (unsigned char)(row + 1u);
            return;
        }
        s = (s + 1u) & mask;
    }
}

// The index bytes of `key` (records 0-3, records 4-7); all 0 when no staged
// record has it.
__device__ __forceinline__ uint2 union_find_node(const uint4 *tab, uint32_t lg, uint32_t key)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(key, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint4 e = tab[s];
        if (e.x == key) return make_uint2(e.y, e.z);
        if (e.x == 0xffffffffu) break;
        s = (s + 1u) & mask;
    }
    return make_uint2(0u, 0u);
}

__device__ __forceinline__ uint2 union_find_conn(const uint4 *tab, uint32_t lg, unsigned long long pair)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = slot_of(fold_pair(pair), lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint4 e = tab[s];
        if ((((unsigned long long)e.y << 32) | e.x) == pair) return make_uint2(e.z, e.w);
        if (e.y == 0xffffffffu) break;
        s = (s + 1u) & mask;
    }
    return make_uint2(0u, 0u);
}

// Row + 1 in record t (0 where absent) among the index bytes of a union
// entry (t a constant after unrolling).
__device__ __forceinline__ uint32_t union_row(uint2 ix, int t)
{
    return ((t < 4 ? ix.x : ix.y) >> (8 * (t & 3))) & 0xffu;
}

// One homologous gene pair's distance terms.
__device__ __forceinline__ float node_term(uint4 x, uint4 y)
{
    return fabsf(__uint_as_float(x.x) - __uint_as_float(y.x)) + fabsf(__uint_as_float(x.y) - __uint_as_float(y.y)) +
           ((__uint_as_float(x.z) != __uint_as_float(y.z)) ? 1.0f : 0.0f) +
           ((__uint_as_float(x.w) != __uint_as_float(y.w)) ? 1.0f : 0.0f);
}

__device__ __forceinline__ float conn_term(float2 x, float2 y)
{
    return fabsf(x.x - y.x) + ((x.y != y.y) ? 1.0f : 0.0f);
}

// v where the mask is all ones, +0 where it is 0 (the term is computed
// either way, with no branch around it).
__device__ __forceinline__ float masked(float v, uint32_t mask)
{
    return __uint_as_float(__float_as_uint(v) & mask);
}

__host__ __device__ constexpr int log2_tile(int t) { return t >= 16 ? 4 : t >= 8 ? 3 : t >= 4 ? 2 : t >= 2 ? 1 : 0; }

// Half-warp totals of TILE per-lane values, one reduce-scatter: lane l ends
// with its half's total of v[(l & 15) >> (4 - log2 TILE)].  The first
// log2 TILE exchange steps (offsets 8, 4, ...) each send half of the lane's
// remaining values to the partner and keep the other half, the rest add
// whole values; lanes are paired in the order 8, 4, 2, 1 throughout, so
// every total is the sum tree of a butterfly reduction of that value alone.
template <int TILE, typename T>
__device__ __forceinline__ T half_sum_scatter(const T (&v)[TILE], int lane)
{
    constexpr int LG = log2_tile(TILE);
    static_assert((1 << LG) == TILE, "TILE is a power of two");
    T w[TILE];
#pragma unroll
    for (int i = 0; i < TILE; ++i) w[i] = v[i];
#pragma unroll
    for (int s = 0; s < LG; ++s) {
        const int o = 8 >> s, half = TILE >> (s + 1);
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T send = hi ? w[i] : w[i + half];
            const T keep = hi ? w[i + half] : w[i];
            w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 8 >> LG; o > 0; o >>= 1) w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    return w[0];
}

// Three blocks per SM at the Ant size (shared memory allows no more): the
// hint lets the union form keep its per-record offsets and sums in registers.
template <int MODE, int TILE>
__global__ void __launch_bounds__(kDistThreads, 3) distance_kernel(const DistArgs p)
{
    static_assert(MODE != kUnion || TILE <= kUnionMaxTile, "union entries hold 8 index bytes");
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar_mem;
    __shared__ int failed;
    __shared__ uint32_t s_n[TILE], s_m[TILE], s_st[TILE], s_nattr[TILE], s_ckey[TILE], s_cattr[TILE];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b0 = blockIdx.y * p.tile;
    const int nb = min(p.tile, p.pb - b0);
    const uint32_t bar = smem_addr(&bar_mem);
    if (tid == 0) {
        // copy sizes: the record's used bytes, never more than its stride
        failed = 0;
        uint32_t total = 0;
        for (int t = 0; t < nb; ++t)
            total += min(align16(__ldg(reinterpret_cast<const uint32_t *>(p.b + (size_t)(b0 + t) * p.stride) + 3)),
                         (uint32_t)p.stride);
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, total);
        for (int t = 0; t < nb; ++t) {
            const uint8_t *src = p.b + (size_t)(b0 + t) * p.stride;
            const uint32_t bytes = min(align16(__ldg(reinterpret_cast<const uint32_t *>(src) + 3)), (uint32_t)p.stride);
            bulk_g2s(smem_addr(sm + (size_t)t * p.slot_bytes), src, bytes, bar);
        }
    }
    if constexpr (MODE == kHash) {
        // the tables sit after each record's stride, outside the copied bytes
        const uint32_t words = (p.slot_bytes - (uint32_t)p.stride) / 8u;
        for (int t = 0; t < nb; ++t) {
            unsigned long long *tab = reinterpret_cast<unsigned long long *>(sm + (size_t)t * p.slot_bytes + p.stride);
            for (uint32_t i = tid; i < words; i += kDistThreads) tab[i] = kEmpty;
        }
    }
    if constexpr (MODE == kUnion) {
        // after the tile's records, outside the copied bytes
        uint4 *u = reinterpret_cast<uint4 *>(sm + p.union_off);
        const uint32_t entries = (1u << p.lgn) + (1u << p.lgc);
        const uint32_t node_entries = 1u << p.lgn;
        for (uint32_t i = tid; i < entries; i += kDistThreads)
            u[i] = i < node_entries ? make_uint4(~0u, 0u, 0u, 0u) : make_uint4(~0u, ~0u, 0u, 0u);
    }
    __syncthreads();
    if (!mbar_wait(bar, 0)) failed = 1;
    __syncthreads();
    const int a_begin = blockIdx.x * p.a_per_block;
    const int a_end = min(p.pa, a_begin + p.a_per_block);
    if (failed) {
        if (tid == 0) atomicOr(&g_distance_error, kErrWaitExpired);
        mbar_wait(bar, 0);
        for (int a = a_begin + warp; a < a_end; a += kDistWarps)
            for (int t = lane; t < nb; t += 32) p.out[(size_t)a * p.ldo + b0 + t] = __int_as_float(0x7fc00000);
        return;
    }
    if (tid < nb) {
        const uint4 hb = *reinterpret_cast<const uint4 *>(sm + (size_t)tid * p.slot_bytes);
        const GeneLayout Lb = gene_layout(hb.x, hb.y);
        s_n[tid] = hb.x;
        s_m[tid] = hb.y;
        s_st[tid] = hb.z;
        s_nattr[tid] = Lb.nattr;
        s_ckey[tid] = Lb.ckey;
        s_cattr[tid] = Lb.cattr;
    }
    if constexpr (MODE == kHash) {
        for (int t = 0; t < nb; ++t) {
            unsigned char *rb = sm + (size_t)t * p.slot_bytes;
            const uint4 hb = *reinterpret_cast<const uint4 *>(rb);
            const GeneLayout Lb = gene_layout(hb.x, hb.y);
            unsigned long long *ntab = reinterpret_cast<unsigned long long *>(rb + p.stride);
            unsigned long long *ctab = ntab + (1u << p.lgn);
            const uint32_t *nkey = reinterpret_cast<const uint32_t *>(rb + Lb.nkey);
            const unsigned long long *ckey = reinterpret_cast<const unsigned long long *>(rb + Lb.ckey);
            for (uint32_t j = tid; j < hb.x; j += kDistThreads)
                table_insert(ntab, p.lgn, slot_of(nkey[j], p.lgn), ((unsigned long long)nkey[j] << 32) | j);
            for (uint32_t j = tid; j < hb.y; j += kDistThreads)
                table_insert(ctab, p.lgc, slot_of(fold_pair(ckey[j]), p.lgc), (ckey[j] << 13) | j);
        }
    }
    if constexpr (MODE == kUnion) {
        uint4 *un = reinterpret_cast<uint4 *>(sm + p.union_off);
        uint4 *uc = un + (1u << p.lgn);
        for (int t = 0; t < nb; ++t) {
            const unsigned char *rb = sm + (size_t)t * p.slot_bytes;
            const uint4 hb = *reinterpret_cast<const uint4 *>(rb);
            const GeneLayout Lb = gene_layout(hb.x, hb.y);
            const uint32_t *nkey = reinterpret_cast<const uint32_t *>(rb + Lb.nkey);
            const unsigned long long *ckey = reinterpret_cast<const unsigned long long *>(rb + Lb.ckey);
            // an index byte addresses rows 0-254 (the host takes this form
            // only for at most 255 genes of each kind)
            for (uint32_t j = tid; j < min(hb.x, 255u); j += kDistThreads) union_insert_node(un, p.lgn, nkey[j], t, j);
            for (uint32_t j = tid; j < min(hb.y, 255u); j += kDistThreads) union_insert_conn(uc, p.lgc, ckey[j], t, j);
        }
    }
    __syncthreads();
    // byte offsets of every staged record's row "-1" of node and connection
    // attributes (the union form reads row b - 1 of every record for index
    // byte b and discards the rows of records that lack the gene, b = 0:
    // those reads land in the record's 16 bytes before its attributes, or
    // at the start of shared memory past the tile)
    uint32_t noff[TILE], coff[TILE];
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
        noff[t] = t < nb ? (uint32_t)t * p.slot_bytes + s_nattr[t] - 16u : 0u;
        coff[t] = t < nb ? (uint32_t)t * p.slot_bytes + s_cattr[t] - 8u : 0u;
    }
    constexpr int LG = log2_tile(TILE);
    const int half = lane >> 4, hl = lane & 15;
    const int out_t = hl >> (4 - LG);                // the representative whose totals this lane ends with
    // two a-genomes per warp, one per half-warp (16 lanes fit the ~50 node
    // genes of a small genome better than 32)
    for (int a0 = a_begin + 2 * warp; a0 < a_end; a0 += 2 * kDistWarps) {
        const int a = a0 + half;
        const bool live = a < a_end;
        const uint8_t *ra = p.a + (size_t)(live ? a : a0) * p.stride;
        uint4 ha = __ldg(reinterpret_cast<const uint4 *>(ra));
        if (!live) ha = make_uint4(0u, 0u, 0u, kGeneHeaderBytes);   // no genes: the half idles to the reductions
        const int n_a = (int)ha.x, m_a = (int)ha.y;
        const GeneLayout La = gene_layout(ha.x, ha.y);
        // lane l ends up with its half's totals of representative out_t
        int my_hn = 0, my_hc = 0;
        float my_sn = 0.0f, my_sc = 0.0f;
        {
            // node genes: each of a's genes is loaded once and looked up in
            // every staged representative (independent lookups in flight)
            int hn[TILE];
            float sn[TILE];
#pragma unroll
            for (int t = 0; t < TILE; ++t) {
                hn[t] = 0;
                sn[t] = 0.0f;
            }
            const uint32_t *ka = reinterpret_cast<const uint32_t *>(ra + La.nkey);
            const uint4 *aa = reinterpret_cast<const uint4 *>(ra + La.nattr);
            for (int j = hl; j < n_a; j += 16) {
                const uint32_t key = __ldg(ka + j);
                const uint4 x = __ldg(aa + j);
                if constexpr (MODE == kUnion) {
                    // one probe for the tile, then the rows it names
                    const uint2 ix = union_find_node(reinterpret_cast<const uint4 *>(sm + p.union_off), p.lgn, key);
#pragma unroll
                    for (int t = 0; t < TILE; ++t) {
                        // partial sums are >= +0, so adding +0 for an absent gene changes no bit
                        const uint32_t b = union_row(ix, t);
                        const uint32_t keep = (uint32_t)(-(int32_t)b >> 31);   // all ones where present
                        const uint4 y = *reinterpret_cast<const uint4 *>(sm + noff[t] + b * 16u);
                        hn[t] -= (int)keep;
                        sn[t] += masked(node_term(x, y), keep);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < TILE; ++t) {
                        if (t < nb) {
                            const unsigned char *rb = sm + (size_t)t * p.slot_bytes;
                            int i;
                            if constexpr (MODE == kHash)
                                i = node_lookup(reinterpret_cast<const unsigned long long *>(rb + p.stride), p.lgn,
                                                key);
                            else
                                i = find_key(reinterpret_cast<const uint32_t *>(rb + kGeneHeaderBytes), (int)s_n[t],
                                             key);
                            if (i >= 0) {
                                const uint4 y = reinterpret_cast<const uint4 *>(rb + s_nattr[t])[i];
                                ++hn[t];
                                sn[t] += node_term(x, y);
                            }
                        }
                    }
                }
            }
            my_hn = half_sum_scatter<TILE>(hn, lane);
            my_sn = half_sum_scatter<TILE>(sn, lane);
        }
        {
            // connection genes, the same way
            int hc[TILE];
            float sc[TILE];
#pragma unroll
            for (int t = 0; t < TILE; ++t) {
                hc[t] = 0;
                sc[t] = 0.0f;
            }
            const unsigned long long *ka = reinterpret_cast<const unsigned long long *>(ra + La.ckey);
            const float2 *aa = reinterpret_cast<const float2 *>(ra + La.cattr);
            for (int j = hl; j < m_a; j += 16) {
                const unsigned long long key = __ldg(ka + j);
                const float2 x = __ldg(aa + j);
                if constexpr (MODE == kUnion) {
                    const uint2 ix = union_find_conn(reinterpret_cast<const uint4 *>(sm + p.union_off) + (1u << p.lgn),
                                                     p.lgc, key);
#pragma unroll
                    for (int t = 0; t < TILE; ++t) {
                        const uint32_t b = union_row(ix, t);
                        const uint32_t keep = (uint32_t)(-(int32_t)b >> 31);
                        const float2 y = *reinterpret_cast<const float2 *>(sm + coff[t] + b * 8u);
                        hc[t] -= (int)keep;
                        sc[t] += masked(conn_term(x, y), keep);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < TILE; ++t) {
                        if (t < nb) {
                            const unsigned char *rb = sm + (size_t)t * p.slot_bytes;
                            int i;
                            if constexpr (MODE == kHash)
                                i = conn_lookup(reinterpret_cast<const unsigned long long *>(rb + p.stride) +
                                                    (1u << p.lgn),
                                                p.lgc, key);
                            else
                                i = find_key(reinterpret_cast<const unsigned long long *>(rb + s_ckey[t]), (int)s_m[t],
                                             key);
                            if (i >= 0) {
                                const float2 y = reinterpret_cast<const float2 *>(rb + s_cattr[t])[i];
                                ++hc[t];
                                sc[t] += conn_term(x, y);
                            }
                        }
                    }
                }
            }
            my_hc = half_sum_scatter<TILE>(hc, lane);
            my_sc = half_sum_scatter<TILE>(sc, lane);
        }
        if (live && (hl & ((16 >> LG) - 1)) == 0 && out_t < nb) {
            float d;
            if (ha.z | s_st[out_t]) {
                d = __int_as_float(0x7fc00000);
            } else {
                const int n_b = (int)s_n[out_t], m_b = (int)s_m[out_t];
                const int nmax = max(n_a, n_b), mmax = max(m_a, m_b);
                const float dn = nmax ? fmaf(p.cd, (float)(n_a + n_b - 2 * my_hn), p.ch * my_sn) / (float)nmax : 0.0f;
                const float dc = mmax ? fmaf(p.cd, (float)(m_a + m_b - 2 * my_hc), p.ch * my_sc) / (float)mmax : 0.0f;
                d = dn + dc;
            }
            p.out[(size_t)a * p.ldo + b0 + out_t] = d;
        }
    }
}

// Nearest representative closer than the threshold (lowest index on ties),
// -1 if none; NaN never qualifies.
__global__ void __launch_bounds__(256) speciate_kernel(const float *dist, int pop, int reps, long long ld,
                                                      float threshold, int32_t *species)
{
    const int g = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= pop) return;
    float best = __int_as_float(0x7f800000);
    int bi = -1;
    for (int s = lane; s < reps; s += 32) {
        const float d = __ldg(dist + (size_t)g * ld + s);
        if (d < threshold && d < best) {
            best = d;
            bi = s;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ob < best || (ob == best && oi < bi))) {
            best = ob;
            bi = oi;
        }
    }
    if (lane == 0) species[g] = bi;
}

int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

int read_distance_error(unsigned int *v, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(v, g_distance_error, sizeof(*v));
    if (e != cudaSuccess) return cuda_fail(e, "distance error word: read");
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_distance_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_fail(e, "distance error word: clear");
    }
    return NEAT_OK;
}

}  // namespace neat

using namespace neat;

extern "C" size_t neat_gene_stride(neat_dims d)
{
    return dims_ok(d) ? gene_stride(d) : 0;
}

extern "C" int neat_distance_prepare(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                                     void *genes_dev, size_t genes_bytes, uint32_t *status_dev, void *stream)
{
    TraceRange trace_range("neat_distance_prepare");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_distance_prepare: invalid dims");
    if (pop < 0) return invalid("neat_distance_prepare: pop < 0");
    if (pop == 0) return NEAT_OK;
    if (!nodes_dev || (!conns_dev && d.max_conns > 0) || !genes_dev)
        return invalid("neat_distance_prepare: null pointer");
    if ((reinterpret_cast<uintptr_t>(conns_dev) & 15u) || (reinterpret_cast<uintptr_t>(genes_dev) & 15u))
        return invalid("neat_distance_prepare: conns and genes must be 16-byte aligned");
    PrepArgs a;
    a.nodes = nodes_dev;
    a.conns = conns_dev;
    a.out = static_cast<uint8_t *>(genes_dev);
    a.status = status_dev;
    a.stride = gene_stride(d);
    if (genes_bytes < a.stride * (size_t)pop) return invalid("neat_distance_prepare: genes buffer too small");
    a.N = d.max_nodes;
    a.C = d.max_conns;
    a.Np2 = next_pow2(a.N);
    a.Cp2 = next_pow2(a.C > 0 ? a.C : 1);
    const size_t smem = 8u * ((size_t)a.Np2 + (size_t)a.Cp2);
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(prepare_kernel), smem,
                                "neat_distance_prepare: shared memory per block");
    if (rc) return rc;
    a.pop = pop;
    if (a.N <= kWarpMaxNodes && a.C <= kWarpMaxConns) {
        const int blocks = (pop + kPrepWarpGenomes - 1) / kPrepWarpGenomes;
        prepare_warp_kernel<<<blocks, 32 * kPrepWarpGenomes, 0, as_stream(stream)>>>(a);
    } else {
        const int threads = (a.N <= 64 && a.C <= 512) ? 128 : kPrepThreads;   // small genomes: more blocks per SM
        prepare_kernel<<<pop, threads, smem, as_stream(stream)>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_distance_prepare: launch");
    return NEAT_OK;
}

extern "C" int neat_distance(const void *genes_a, int32_t pop_a, const void *genes_b, int32_t pop_b, neat_dims d,
                             float c_disjoint, float c_homologous, float *out_dev, int64_t ld_out, void *stream)
{
    TraceRange trace_range("neat_distance");
    clear_error();
    if (!dims_ok(d)) return invalid("neat_distance: invalid dims");
    if (pop_a < 0 || pop_b < 0) return invalid("neat_distance: populations must be >= 0");
    if (pop_a == 0 || pop_b == 0) return NEAT_OK;
    if (!genes_a || !genes_b || !out_dev) return invalid("neat_distance: null pointer");
    if (ld_out < pop_b) return invalid("neat_distance: ld_out < pop_b");
    if ((reinterpret_cast<uintptr_t>(genes_a) & 15u) || (reinterpret_cast<uintptr_t>(genes_b) & 15u))
        return invalid("neat_distance: gene records must be 16-byte aligned");
    DistArgs p;
    p.a = static_cast<const uint8_t *>(genes_a);
    p.b = static_cast<const uint8_t *>(genes_b);
    p.stride = gene_stride(d);
    p.pa = pop_a;
    p.pb = pop_b;
    p.cd = c_disjoint;
    p.ch = c_homologous;
    p.out = out_dev;
    p.ldo = ld_out;
    const size_t budget = 200u * 1024u, shared_budget = 76u * 1024u;   // one block / three blocks per SM
    if (p.stride > budget) return invalid("neat_distance: gene record exceeds 200 KB of shared memory");
    // hash tables of capacity 2^lg > 1.5x the largest gene count, when they fit
    auto lg_cap = [](int n) {
        uint32_t lg = 1;
        while ((1u << lg) < (uint32_t)(n + n / 2 + 1)) ++lg;
        return lg;
    };
    p.lgn = lg_cap(d.max_nodes);
    p.lgc = lg_cap(d.max_conns);
    const size_t slot_hash = p.stride + 8u * ((size_t(1) << p.lgn) + (size_t(1) << p.lgc));
    const bool hash = slot_hash <= budget;
    p.slot_bytes = (uint32_t)(hash ? slot_hash : p.stride);
    const size_t per_block = p.slot_bytes <= shared_budget ? shared_budget : budget;
    p.tile = (int)std::min<size_t>({(size_t)kMaxTile, per_block / p.slot_bytes, (size_t)pop_b});
    p.union_off = 0;
    size_t smem = (size_t)p.tile * p.slot_bytes;
    // union tables (at most 255 genes of each kind: byte row indices) of
    // capacity 2^lg > 1.25x the tile's largest possible union, taken when
    // they stage as many records per block as the per-record tables (up to
    // 8, the records an entry indexes), three blocks per SM: a gene is then
    // probed once per tile instead of once per record
    bool use_union = false;
    if (d.max_nodes <= 255 && d.max_conns <= 255) {
        auto lg_union = [](long n) {
            uint32_t lg = 1;
            while ((1L << lg) < n + n / 4 + 1) ++lg;
            return lg;
        };
        const int want = std::min(kUnionMaxTile, p.tile);
        for (int t = std::min(kUnionMaxTile, (int)pop_b); t >= want; --t) {
            const uint32_t ln = lg_union((long)t * d.max_nodes), lc = lg_union((long)t * d.max_conns);
            const size_t bytes = (size_t)t * p.stride + 16u * ((size_t(1) << ln) + (size_t(1) << lc));
            if (bytes <= shared_budget) {
                use_union = true;
                p.tile = t;
                p.lgn = ln;
                p.lgc = lc;
                p.slot_bytes = (uint32_t)p.stride;
                p.union_off = (uint32_t)((size_t)t * p.stride);
                smem = bytes;
                break;
            }
        }
    }
    const int tiles = (pop_b + p.tile - 1) / p.tile;
    if (tiles > 65535) return invalid("neat_distance: too many b-genomes");
    int dev = 0, sms = 152, smem_sm = 228 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    // one wave: as many blocks as fit at once, the a-genomes split evenly
    const int resident = std::max(1, std::min(3, (int)(smem_sm / (smem + 1024u))));
    const long want_x = std::max<long>(1, ((long)sms * resident + tiles - 1) / tiles);
    long apb = (pop_a + want_x - 1) / want_x;
    apb = std::max<long>(2 * kDistWarps, (apb + 2 * kDistWarps - 1) / (2 * kDistWarps) * (2 * kDistWarps));
    p.a_per_block = (int)std::min<long>(apb, 1L << 30);
    const long gx = (pop_a + p.a_per_block - 1) / p.a_per_block;
    using Kern = void (*)(DistArgs);
    Kern kern;
    if (use_union) {
        if (p.tile > 4) kern = distance_kernel<kUnion, 8>;
        else if (p.tile > 2) kern = distance_kernel<kUnion, 4>;
        else if (p.tile > 1) kern = distance_kernel<kUnion, 2>;
        else kern = distance_kernel<kUnion, 1>;
    } else if (p.tile > 8) {
        kern = hash ? distance_kernel<kHash, 16> : distance_kernel<kSearch, 16>;
    } else if (p.tile > 4) {
        kern = hash ? distance_kernel<kHash, 8> : distance_kernel<kSearch, 8>;
    } else if (p.tile > 2) {
        kern = hash ? distance_kernel<kHash, 4> : distance_kernel<kSearch, 4>;
    } else if (p.tile > 1) {
        kern = hash ? distance_kernel<kHash, 2> : distance_kernel<kSearch, 2>;
    } else {
        kern = hash ? distance_kernel<kHash, 1> : distance_kernel<kSearch, 1>;
    }
    int rc = allow_dynamic_smem(reinterpret_cast<const void *>(kern), smem, "neat_distance: shared memory per block");
    if (rc) return rc;
    kern<<<dim3((unsigned)gx, (unsigned)tiles), kDistThreads, smem, as_stream(stream)>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_distance: launch");
    return NEAT_OK;
}

extern "C" int neat_speciate(const float *distances_dev, int32_t pop, int32_t n_reps, int64_t ld, float threshold,
                             int32_t *species_dev, void *stream)
{
    TraceRange trace_range("neat_speciate");
    clear_error();
    if (pop < 0 || n_reps < 0) return invalid("neat_speciate: sizes must be >= 0");
    if (pop == 0) return NEAT_OK;
    if (!species_dev || (n_reps > 0 && !distances_dev)) return invalid("neat_speciate: null pointer");
    if (ld < n_reps) return invalid("neat_speciate: ld < n_reps");
    const long threads = (long)pop * 32;
    speciate_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, as_stream(stream)>>>(distances_dev, pop, n_reps, ld,
                                                                                      threshold, species_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_speciate: launch");
    return NEAT_OK;
}
