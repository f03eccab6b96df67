// Internal declarations shared by the CUDA translation units of libneat.so.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/neat.h"

namespace neat {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);   // records and returns NEAT_ECUDA
int invalid(const char *what);                     // records and returns NEAT_EINVAL

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------ record geometry
constexpr uint32_t kHeaderBytes = 32;
constexpr uint32_t kNodeBytes = 16;
constexpr uint32_t kEdgeBytes = 8;
constexpr uint8_t kInputAct = 255;

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Largest record (all rows present, every connection enabled).
__host__ __device__ inline uint32_t record_max_bytes(int I, int O, int N, int C)
{
    uint32_t off_edge = kHeaderBytes + kNodeBytes * (uint32_t)N;
    uint32_t off_level = align16(off_edge + kEdgeBytes * (uint32_t)C);
    uint32_t off_io = align16(off_level + 2u * (uint32_t)(N + 1));
    return align16(off_io + 2u * (uint32_t)(I + O));
}

inline size_t record_stride(const neat_dims &d)
{
    size_t b = record_max_bytes(d.num_inputs, d.num_outputs, d.max_nodes, d.max_conns);
    return (b + 127) & ~(size_t)127;
}

bool dims_ok(const neat_dims &d);

// Shared memory per block on sm_103 (static + dynamic).
constexpr size_t kMaxSmemPerBlock = 227u * 1024u;

// Let `kernel` launch with `dynamic_bytes` of dynamic shared memory on the
// current device, counting its static shared memory: raises the kernel's
// limit when static + dynamic exceeds the 48 KB default (never lowers it).
// NEAT_EINVAL (message `what`) when the total exceeds kMaxSmemPerBlock.
int allow_dynamic_smem(const void *kernel, size_t dynamic_bytes, const char *what);

// ---------------------------------------------------------- forward args
// Shared memory one group's record and value tiles may take in a default
// launch shape (room left for the block's barriers).
constexpr size_t kMaxGroupSmem = 200u * 1024u;

// Threads per tile row for a genome of up to n nodes and a batch of several
// input vectors: about one per 32 nodes (a level of a large genome holds
// tens of nodes), a power of two in 1..16.
inline int tile_row_threads(int n)
{
    int nsub = 1;
    while (nsub < 16 && nsub * 2 * 32 <= n) nsub <<= 1;
    return nsub;
}

struct ForwardArgs {
    const uint8_t *rec;      // records, one per genome, `stride` bytes apart
    size_t stride;
    const float *x;          // [pop][B][I]
    float *y;                // [pop][B][O]
    int pop, I, O, N;
    int B;                   // input vectors per genome
    int group;               // threads per work item (power of two)
    int tile;                // columns per work item (power of two)
    int lg_split;            // log2 of threads per node when tile == 1
    int tiles;               // ceil(B / tile)
    int rec_words;           // 16-byte words of shared memory reserved for a record
    int val_floats;          // floats of shared memory for node values (N * tile, rounded to 4)
    int rec_copy_bytes;      // bytes of each record copied in one piece (0: read the size from its header)
    const int32_t *order;    // genome of work item k / tiles (NULL: identity)
};

// 16-byte words before the groups' regions in a forward block's shared
// memory: one mbarrier (8 B) and one flag (4 B) per group.
__host__ __device__ inline int forward_header_words(int groups) { return (groups * 12 + 15) / 16; }

// Launch one forward over a single population (defined in neat_forward.cu).
int launch_forward(const ForwardArgs &a, const neat_launch &L, cudaStream_t s);
int make_forward_args(const void *transformed, int32_t pop, const neat_dims &d,
                      const float *inputs, int32_t batch, float *outputs,
                      const neat_launch &L, ForwardArgs *out);
int check_launch(const neat_launch &L);

// One bucket of the persistent multi-population kernel (neat_plan.cu): a
// set of genomes of one population evaluated with one launch shape.
struct BucketDev {
    const uint8_t *rec;
    const int32_t *gidx;     // genome indices (within the population) of this bucket
    const float *x;
    float *y;
    int64_t x_step, y_step;  // floats between steps
    uint64_t stride;
    int n_genomes;
    int I, O, B;
    int tile, tiles, lg_split;
    int G, lgG, gpc;
    int region_words;        // 16-byte words of one group's region (record + values)
    int rec_words;           // 16-byte words reserved for the record
    int rec_copy_bytes;
    int cta_begin, cta_items;
};

// A whole population as one bucket with the heuristic launch shape; gidx_dev
// must list genomes 0..pop-1.  *footprint: shared memory of its groups.
int fill_population_bucket(const neat_pop_desc &pd, const int32_t *gidx_dev, int block_threads, int cta_begin,
                           BucketDev *out, size_t *footprint);
// Launch the persistent kernel over a bucket table already in device memory
// (counter_dev must be zero).
int launch_plan_table(const BucketDev *table_dev, int nb, int total_items, unsigned int *counter_dev, int step,
                      size_t smem_regions, int block_threads, cudaStream_t s);
int read_plan_error(unsigned int *v, int clear);   // neat_plan.cu
int read_cppn_error(unsigned int *v, int clear);   // neat_cppn.cu
int read_rnn_error(unsigned int *v, int clear);    // neat_recurrent.cu
int read_distance_error(unsigned int *v, int clear);   // neat_distance.cu
int read_fused_error(unsigned int *v, int clear);      // neat_fused.cu
int read_substrate_error(unsigned int *v, int clear);  // neat_substrate.cu
int read_lanes_error(unsigned int *v, int clear);      // neat_lanes.cu
// Groups per block that put `items` groups of `group` threads, each needing
// `per_group` bytes of shared memory, in the fewest waves with the busiest SM
// least loaded (neat_forward.cu).
int groups_per_block_for(long items, int group, size_t per_group);

}  // namespace neat
