/*
 * neat.h -- C ABI of libneat.so: population-wide evaluation of NEAT genomes
 * on one GB300 (sm_103a).
 *
 * The method is the tensorized inference of Section 3.3 ("Tensorized Network
 * Inference"): a population of networks, each encoded as a NaN-padded node
 * tensor and connection tensor (Section 3.1, "Tensorized Encodings"), is
 * first *transformed* once (topological order of the nodes plus the incoming
 * connections of every node; this library stores a compact per-node list in
 * place of the dense |N|max x |N|max expanded-connection tensor C_exp), then
 * *forwarded* on any number of input vectors.  The function names mirror the
 * genome interface's transform(nodes, conns) / forward(inputs, transformed)
 * (Appendix "Interfaces", Listing 2).
 *
 * Conventions for every call below
 *   - Pointers named *_dev are DEVICE pointers owned by the caller; pointers
 *     named *_host are host pointers.  Nothing is retained after return
 *     except where a call says so.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it and return
 *     without synchronising; results are ready when the stream reaches them.
 *   - Return value: NEAT_OK (0) or a negative NEAT_E* code.  On error nothing
 *     was enqueued and neat_last_error() (thread-local) describes the cause.
 *   - No call on the forward path allocates device memory.
 *
 * Genome encoding (Section 3.1)
 *   nodes_dev f32 [pop][max_nodes][5]: (key, bias, response, aggregation, activation)
 *   conns_dev f32 [pop][max_conns][4]: (in key, out key, enabled, weight);
 *     with max_conns = 0 it holds nothing and may be NULL
 *   A node row is present when its key is not NaN; a connection row when its
 *   in key, out key and enabled flag are not NaN.  Absent (NaN) rows may sit
 *   anywhere, also between present rows (node or connection removal writes
 *   NaN into a row, Section 3.2).
 *   Keys are historical markers: exact integers in [0, 2^24), looked up,
 *   never used as row indices.  Input j is the node with key j (0 <= j < I),
 *   output j the node with key I + j (the interface's input_idx = arange(I),
 *   output_idx = arange(I, I+O)).
 *   Categorical attributes are stored as integer-valued floats (Section 3.1
 *   gives tanh = 1, sigmoid = 2):
 *     activation 0 identity, 1 tanh, 2 sigmoid 1/(1+e^-z), 3 relu max(z,0),
 *                4 sin, 5 gauss e^(-z^2), 6 abs
 *     aggregation 0 sum, 1 product, 2 max, 3 mean
 *   A connection is enabled when its flag is non-zero; disabled connections
 *   take no part in the order or the forward pass (the C_exp rule maps them
 *   to NaN).
 *
 * Node rule (Section 3.3): f_c(x | w) = w x and
 *   v[k] = act_k(bias_k + response_k * agg_k(w_c v[src_c] for the enabled
 *          connections c into k, in ascending connection row)),
 * the response factor being this library's reading (the paper lists response
 * among the node hyperparameters, Appendix "Hyperparameters").  An empty
 * incoming set aggregates to 0.  Input nodes pass their input value through;
 * their other attributes are ignored.
 * Arithmetic is IEEE float32 in a fixed order: a node's incoming edges
 * (ascending connection row) are dealt round-robin into four partials,
 * partial k holding edges k, k+4, k+8, ... accumulated in that order (sum and
 * mean with fused multiply-add), and the aggregate is ((p0 . p1) . (p2 . p3))
 * for the aggregation's operation "." (then / count for the mean).  The order
 * depends on the genome alone, so its outputs are a function of the genome
 * and the input, bit for bit, whatever the launch shape or co-scheduled work.
 */
#ifndef NEAT_H
#define NEAT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NEAT_API __attribute__((visibility("default")))
#else
#define NEAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ constants */

enum {
    NEAT_OK = 0,
    NEAT_EINVAL = -1,      /* bad argument: null pointer, size out of range */
    NEAT_ENOMEM = -2,      /* a buffer is too small, or host/device allocation failed */
    NEAT_ECUDA = -3,       /* a CUDA runtime call failed (see neat_last_error) */
    NEAT_EBUDGET = -4,     /* request can never fit the server's memory budget */
    NEAT_EAGAIN = -5,      /* not finished yet */
    NEAT_ETIMEOUT = -6,    /* a bounded wait expired */
    NEAT_ECANCELLED = -7   /* request was cancelled */
};

/* Per-genome status word written by neat_transform.  The low byte holds
 * errors: a genome with any of them is not evaluated and every one of its
 * outputs is NaN.  Bits 8.. are warnings: the offending rows are ignored and
 * the genome is evaluated. */
enum {
    NEAT_G_CYCLE = 1u,        /* enabled connections form a cycle */
    NEAT_G_DUPKEY = 2u,       /* two present node rows share a key */
    NEAT_G_BADKEY = 4u,       /* a key is not an integer in [0, 2^24) */
    NEAT_G_BADENUM = 8u,      /* activation or aggregation id out of range */
    NEAT_G_DUPCONN = 16u,     /* two present connections join the same keys */
    NEAT_G_BADATTR = 32u,     /* NaN bias/response, or NaN weight of an enabled connection */
    NEAT_G_MISSING_IO = 64u,  /* an input or output key has no node */
    NEAT_W_DANGLING = 256u,   /* enabled connection to/from an absent key (ignored) */
    NEAT_W_INTO_INPUT = 512u  /* enabled connection into an input node (ignored) */
};
#define NEAT_G_ERROR_MASK 0xffu

/* Limits of this implementation. */
#define NEAT_MAX_NODES 1024
#define NEAT_MAX_CONNS 8192

typedef struct neat_dims {
    int32_t num_inputs;   /* I  >= 0 */
    int32_t num_outputs;  /* O  >= 1; I + O <= max_nodes */
    int32_t max_nodes;    /* |N|max, 1..NEAT_MAX_NODES */
    int32_t max_conns;    /* |C|max, 0..NEAT_MAX_CONNS */
} neat_dims;

/* ------------------------------------------------- transformed records
 *
 * neat_transform writes one record per genome at byte offset g * stride of
 * the `transformed` buffer (stride = neat_record_stride(d), a multiple of
 * 128).  A record is packed in topological-position space: position p is the
 * p-th node of the order; every reference to a node is its position.
 *
 *   offset 0   neat_record_header
 *   offset 32  node entries [n_nodes]      (neat_node_entry, 16 B each)
 *   off_edge   edge entries [n_edges]      (neat_edge_entry, 8 B each)
 *   off_level  uint16 level_ptr[n_levels + 1]: level l = positions
 *              [level_ptr[l], level_ptr[l+1])
 *   off_io     uint16 in_pos[I] (position of input key j), then
 *              uint16 out_pos[O] (position of output key I + j)
 *   used_bytes total bytes written, a multiple of 16
 * The order is the layered Kahn order: level 0 holds the present nodes with
 * no enabled incoming connection, level l+1 the nodes whose last incoming
 * connection comes from level l, and within a level positions follow
 * ascending node row.  A node's incoming edges are
 * [edge_begin, edge_begin + edge_count) in ascending connection row.
 * When the status has an error bit only the header is meaningful
 * (n_levels = 0).
 */
typedef struct neat_record_header {
    uint16_t n_nodes;     /* present node rows */
    uint16_t n_levels;
    int32_t n_edges;      /* enabled connections kept */
    uint32_t status;      /* NEAT_G_* / NEAT_W_* bits */
    uint8_t uniform_activation;   /* activation id shared by every non-input node, else 255 */
    uint8_t uniform_aggregation;  /* aggregation id shared by every non-input node, else 255 */
    uint16_t lead_inputs; /* positions 0 .. lead_inputs-1 are all input nodes */
    uint32_t used_bytes;
    uint32_t off_edge;
    uint32_t off_level;
    uint32_t off_io;
} neat_record_header;

typedef struct neat_node_entry {
    float bias;
    float response;
    uint16_t edge_begin;
    uint16_t edge_count;
    uint8_t activation;   /* 0..6, or 255 for an input node */
    uint8_t aggregation;  /* 0..3 */
    uint16_t row;         /* node row in the genome tensor */
} neat_node_entry;

typedef struct neat_edge_entry {
    float weight;
    uint32_t src;         /* position of the source node */
} neat_edge_entry;

/* Bytes of one genome's record for these dimensions (0 if they are invalid). */
NEAT_API size_t neat_record_stride(neat_dims d);

/* Bytes of the transformed buffer for `pop` genomes (0 if invalid). */
NEAT_API size_t neat_transformed_bytes(int32_t pop, neat_dims d);

/*
 * Transformation stage (Section 3.3): for each of `pop` genomes, check the
 * rows, resolve keys, build the layered Kahn order and the incoming edge
 * lists, and write its record into transformed_dev.
 *   nodes_dev, conns_dev   genome tensors as above (16-byte aligned)
 *   transformed_dev        >= neat_transformed_bytes(pop, d) bytes, 16-byte aligned
 *   status_dev             uint32 [pop], may be NULL (the status is also in each header)
 * Errors: NEAT_EINVAL (null pointer, pop < 0, invalid dims), NEAT_ENOMEM
 * (transformed_bytes too small), NEAT_ECUDA (launch failed).  Malformed
 * genomes are not call errors: they are reported in their status word.
 */
NEAT_API int neat_transform(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                   void *transformed_dev, size_t transformed_bytes, uint32_t *status_dev,
                   void *stream);

/*
 * Calculation stage (Section 3.3): outputs of every genome on `batch` input
 * vectors each.
 *   transformed_dev  records written by neat_transform with the same dims
 *   inputs_dev       f32 [pop][batch][I]
 *   outputs_dev      f32 [pop][batch][O] (written; NaN for genomes with an error bit)
 * The launch shape is chosen from (dims, batch); the results do not depend on it.
 * Errors: NEAT_EINVAL, NEAT_ECUDA.
 */
NEAT_API int neat_forward(const void *transformed_dev, int32_t pop, neat_dims d,
                 const float *inputs_dev, int32_t batch, float *outputs_dev, void *stream);

/*
 * Launch shape of the forward kernel.  A work item is (genome, tile of
 * `tile` input vectors), evaluated by a group of `group` threads: tile
 * columns times group/tile threads that split each level's nodes.
 * `groups_per_block` groups share a thread block.  `pdl` != 0 launches with
 * programmatic dependent launch: the record is staged before the kernel waits
 * on the previous kernel in the stream, the inputs after.
 * Constraints: group a power of two in 1..1024, tile a power of two <= group,
 * group * groups_per_block <= 1024.
 */
typedef struct neat_launch {
    int32_t group;
    int32_t tile;
    int32_t groups_per_block;
    int32_t pdl;
    int32_t split;   /* tile == 1: at most this many threads (1, 2 or 4) share one node's edges,
                        chosen per level from its width; else ignored (1) */
    int32_t reserved;
    const int32_t *order_dev;   /* optional genome order (device, a permutation of 0..pop-1, e.g.
                                   from neat_schedule): work item k evaluates genome order_dev[k];
                                   outputs stay in genome order.  NULL: identity */
} neat_launch;

/*
 * Genome order for the forward: genomes sorted by level count, deepest
 * first (counts above 63 share one bin), then by the number of non-input
 * nodes, most first (64 bins over max_nodes), into order_dev (int32 [pop],
 * device).  Groups that share a warp then walk similar numbers of levels and
 * nodes; recurrent records (one level each) are ordered by node count.
 * Reads the record headers only; runs on `stream` (one block).  The order
 * changes speed, never results.
 */
NEAT_API int neat_schedule(const void *transformed_dev, int32_t pop, neat_dims d, int32_t *order_dev, void *stream);

/* The launch shape neat_forward uses for (pop, d, batch): for one input
 * vector per genome, 8 to 32 threads per genome by max_nodes; for several,
 * tiles of up to 32 vectors with a power of two of threads per tile row
 * (about one per 32 nodes, at most 16), the tile halved until a group's
 * record and value tile fit one block; then the number of groups per block
 * giving the fewest waves on the current device, genomes spread evenly over
 * its SMs. */
NEAT_API int neat_default_launch(int32_t pop, neat_dims d, int32_t batch, neat_launch *out_host);

/* neat_forward with an explicit launch shape (NULL = default). */
NEAT_API int neat_forward_ex(const void *transformed_dev, int32_t pop, neat_dims d,
                    const float *inputs_dev, int32_t batch, float *outputs_dev,
                    const neat_launch *launch_host, void *stream);

/*
 * Steps loop as one CUDA graph: `steps` forwards of the same transformed
 * population, step s reading inputs_dev + s * in_step_stride floats and
 * writing outputs_dev + s * out_step_stride floats, each launched with
 * programmatic dependent launch so that a step stages its records while the
 * previous step drains.  The graph is built on first use and kept in `*cache`
 * (opaque, initialise to NULL; freed by neat_steps_cache_destroy); it is
 * rebuilt when any argument changes.  Enqueued on `stream`.
 */
typedef struct neat_steps_cache neat_steps_cache;
NEAT_API int neat_forward_steps(const void *transformed_dev, int32_t pop, neat_dims d,
                       const float *inputs_dev, int64_t in_step_stride, int32_t batch,
                       float *outputs_dev, int64_t out_step_stride, int32_t steps,
                       const neat_launch *launch_host, neat_steps_cache **cache, void *stream);
NEAT_API void neat_steps_cache_destroy(neat_steps_cache *cache);

/* Many forwards in one launch, for input sequences known in advance (a fixed
 * evaluation set, or observations that do not depend on the previous step's
 * outputs): step s reads inputs_dev + s * in_step_stride ([pop][batch][I])
 * and writes outputs_dev + s * out_step_stride ([pop][batch][O]), as
 * neat_forward_steps, but each group keeps its genome's record in shared
 * memory across all steps (read once per launch) and the next step's inputs
 * are loaded during the current step.  Outputs are bit-identical to per-step
 * forwards with the same record.  launch: NULL = neat_default_launch.
 * Errors: NEAT_EINVAL (strides smaller than one step, launch shape),
 * NEAT_ECUDA. */
NEAT_API int neat_forward_fused(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                int64_t in_step_stride, int32_t batch, float *outputs_dev, int64_t out_step_stride,
                                int32_t steps, const neat_launch *launch, void *stream);

/* ------------------------------------------------------ lane programs
 *
 * The calculation of Section 3.3 for ONE input vector per genome per call
 * (a control loop that steps every genome once per environment step),
 * compiled per transformed population into lane programs: two threads
 * ("lanes") evaluate one genome, one node each per "beat", and the 16
 * genomes of a warp share one instruction stream, with one warp barrier per
 * beat.  neat_lanes_pack compiles (once per transform); neat_forward_lanes /
 * neat_forward_lanes_steps run.  Outputs are bit-identical to neat_forward
 * with batch 1 (same node rule, same aggregation order; the padding edges
 * of a lane program change no bit of any partial).  Limits: max_nodes <=
 * 128; records from neat_transform (feedforward; a genome whose record has
 * no topological order gets NaN outputs and is counted in
 * neat_lanes_info.unordered).
 *
 * Compilation: per genome a list schedule of beats of up to two nodes whose
 * sources are all computed in earlier beats (longest remaining path first);
 * genomes sorted by (beats, edge quads), deepest first, 16 to a warp; each
 * warp program holds its beats' node entries and the nodes' incoming edges
 * in quads of four, interleaved by lane.
 *
 * Recurrent networks (records of neat_transform_recurrent) compile with
 * neat_lanes_pack_recurrent and run with neat_forward_lanes_recurrent: every
 * non-input node is evaluated once per iteration from the previous
 * iteration's values, so a genome's nodes are simply dealt to its two lanes
 * by edge count (most first); each iteration runs the beats from one value
 * tile into the other with one warp barrier.  A buffer packed for one
 * forward gives NaN outputs in the other.
 */
typedef struct neat_lanes_info {
    int32_t pop;
    int32_t warps;              /* ceil(pop / 32): blocks of 32 threads per forward */
    uint32_t max_warp_bytes;    /* largest warp program: a stage_bytes that stages every program */
    uint32_t warp_stride;       /* bytes reserved for each warp program */
    uint32_t unordered;         /* genomes with no feedforward order (NaN outputs) */
    uint32_t recurrent;         /* 1: packed by neat_lanes_pack_recurrent */
} neat_lanes_info;

/* Bytes of the lanes buffer for `pop` genomes (0 if the dims are invalid or
 * max_nodes > 128). */
NEAT_API size_t neat_lanes_bytes(int32_t pop, neat_dims d);

/* Compile the lane programs of `pop` transformed genomes (records of
 * neat_transform with the same dims) into lanes_dev (caller-owned device
 * buffer of >= neat_lanes_bytes(pop, d) bytes, 128-byte aligned).  Three
 * small kernels on `stream`; nothing is allocated.  Recompile after every
 * transform.  Errors: NEAT_EINVAL (dims, null pointer, alignment),
 * NEAT_ENOMEM (buffer too small), NEAT_ECUDA. */
NEAT_API int neat_lanes_pack(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev,
                             size_t lanes_bytes, void *stream);

/* Header of a packed buffer into *out_host (synchronous: a device-to-host
 * copy on the legacy stream, after the pack has completed). */
NEAT_API int neat_lanes_query(const void *lanes_dev, neat_lanes_info *out_host);

/* One forward from lane programs: inputs f32 [pop][I] -> outputs f32
 * [pop][O] (genome order; NaN for genomes with an error bit).  Each warp
 * program is copied into shared memory when it fits stage_bytes (0: the
 * smaller of warp_stride and 48 KB); a larger one is read from device
 * memory (same results, slower).  stage_bytes is also the shared memory
 * each block reserves for its program, so it sets how many blocks share an
 * SM (neat_lanes_tune picks it).  pop and d must be those of the pack.
 * Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_forward_lanes(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                float *outputs_dev, uint32_t stage_bytes, void *stream);

/* `steps` forwards from lane programs as one CUDA graph, step s reading
 * inputs_dev + s * in_step_stride and writing outputs_dev + s *
 * out_step_stride floats; every step after the first launches with
 * programmatic dependent launch (its programs are staged while the previous
 * step drains; its inputs are read after the previous step completes).  The
 * graph is built on first use, kept in *cache
 * (initialise to NULL; free with neat_lanes_cache_destroy) and rebuilt when
 * an argument changes.  Repacking the same lanes buffer between replays is
 * allowed. */
typedef struct neat_lanes_cache neat_lanes_cache;
NEAT_API int neat_forward_lanes_steps(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                      int64_t in_step_stride, float *outputs_dev, int64_t out_step_stride,
                                      int32_t steps, uint32_t stage_bytes, neat_lanes_cache **cache, void *stream);
NEAT_API void neat_lanes_cache_destroy(neat_lanes_cache *cache);

/* Recurrent lane programs (Section 3.3 names recurrent networks beside
 * feedforward ones; the iteration rule is that of neat_forward_recurrent):
 * as neat_lanes_pack, for records of neat_transform_recurrent (cycles and
 * self-loops allowed), into a buffer of >= neat_lanes_bytes(pop, d) bytes.
 * Errors as neat_lanes_pack. */
NEAT_API int neat_lanes_pack_recurrent(const void *transformed_dev, int32_t pop, neat_dims d, void *lanes_dev,
                                       size_t lanes_bytes, void *stream);

/* `iterations` synchronous iterations of recurrent lane programs for one
 * input vector per genome: inputs f32 [pop][I] -> outputs f32 [pop][O]
 * (genome order), bit-identical to neat_forward_recurrent with batch 1 and
 * the same records: non-input nodes start at 0, iteration k computes every
 * non-input node from iteration k-1's values, the outputs are the values
 * after the last iteration (0 for non-input outputs when iterations is 0).
 * stage_bytes as for neat_forward_lanes (0: the smaller of warp_stride and
 * 48 KB; neat_lanes_info.max_warp_bytes from neat_lanes_query stages every
 * program with the least shared memory, which is what keeps a population's
 * blocks in one wave); pdl = 1 launches with programmatic dependent launch (the programs
 * are staged while the previous kernel in the stream drains; the inputs
 * are read after it completes).  NaN outputs for genomes with an error bit
 * and for a buffer packed by neat_lanes_pack.  Errors: NEAT_EINVAL
 * (iterations < 0, dims, stage_bytes), NEAT_ECUDA. */
NEAT_API int neat_forward_lanes_recurrent(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                          int32_t iterations, float *outputs_dev, uint32_t stage_bytes, int32_t pdl,
                                          void *stream);

/* Picks stage_bytes for neat_forward_lanes_steps on this population and
 * device: one candidate per number of blocks an SM holds (the smallest
 * reservation for each, from the most the largest program allows down to
 * the fewest that still hold one step's blocks at once); each is timed as a
 * graph of min(steps, 64) forwards on `stream` (best of three replays; the
 * forwards write outputs_dev as neat_forward_lanes_steps does) and the
 * fastest is written to *stage_bytes.  Arguments as for
 * neat_forward_lanes_steps; synchronous (reads the pack's header and waits
 * for the timed graphs).  Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_lanes_tune(const void *lanes_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                             int64_t in_step_stride, float *outputs_dev, int64_t out_step_stride, int32_t steps,
                             uint32_t *stage_bytes, void *stream);

/*
 * Device error word of the forward (single-step, fused and lane-program), plan, CPPN, recurrent and distance kernels: bit 0 is set when a
 * bounded on-device wait (a record copy into shared memory, 1 s) ran out;
 * the affected outputs are NaN.  Copies the word to *out_host and clears it if `clear`.
 * Synchronous (a device-to-host copy on the legacy stream).
 */
NEAT_API int neat_device_error(int32_t clear, uint32_t *out_host);

/* ------------------------------------------------------ recurrent nets
 *
 * Networks whose enabled connections form cycles (Section 3.3 names
 * recurrent networks beside feedforward ones; the paper gives no algorithm
 * for them).  This library's definition: input nodes hold their inputs,
 * every other node starts at 0, and `iterations` synchronous iterations
 * follow, each computing every non-input node from the previous iterate:
 *   v_k[n] = act_n(bias_n + response_n * agg_n(w_c v_{k-1}[src_c]))
 * (same rule, ids and aggregation order as the feedforward path).  The
 * outputs are the last iterate at the output keys.  On an acyclic genome,
 * as many iterations as it has levels give the feedforward outputs.
 */

/* Transform for recurrent networks: the checks and record layout of
 * neat_transform, but cycles (self-loops included) are allowed, there is no
 * topological sort (positions follow node rows, one level) and
 * NEAT_G_CYCLE is never set. */
NEAT_API int neat_transform_recurrent(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                                      void *transformed_dev, size_t transformed_bytes, uint32_t *status_dev,
                                      void *stream);

/* Recurrent forward on records from neat_transform_recurrent: inputs
 * f32 [pop][batch][I] -> outputs f32 [pop][batch][O] after `iterations`
 * (>= 0) synchronous iterations, default launch shape.  Errors as
 * neat_forward, plus NEAT_EINVAL for iterations < 0. */
NEAT_API int neat_forward_recurrent(const void *transformed_dev, int32_t pop, neat_dims d, const float *inputs_dev,
                                    int32_t batch, int32_t iterations, float *outputs_dev, void *stream);

/* As neat_forward_recurrent with an explicit launch shape (NULL = the
 * default).  Fields as for neat_forward_ex, with `split` = 1 (every node of
 * an iteration is in flight at once, so nodes are not split); shared memory
 * per group is the record plus two value tiles. */
NEAT_API int neat_forward_recurrent_ex(const void *transformed_dev, int32_t pop, neat_dims d,
                                       const float *inputs_dev, int32_t batch, int32_t iterations,
                                       float *outputs_dev, const neat_launch *launch, void *stream);

/* Default launch shape of the recurrent forward (host only; queries the
 * current device once). */
NEAT_API int neat_default_launch_recurrent(int32_t pop, neat_dims d, int32_t batch, neat_launch *out);

/* ------------------------------------------------- genome distance
 *
 * Distances between genomes for speciation (Algorithm 1 divides the
 * population into species by distances between networks; the
 * hyperparameters compatibility_disjoint and compatibility_homologous weight
 * disjoint and homologous genes, and compatibility_threshold bounds a
 * species).  The paper gives no formula; this library's definition:
 *   genes are the present rows of the node tensor and the connection tensor
 *   (inputs and disabled connections included); node genes are homologous
 *   when their keys are equal, connection genes when their (in key, out key)
 *   pairs are equal; every other gene is disjoint.
 *   d(a, b) = (c_d D_n + c_h S_n) / max(n_a, n_b) + (c_d D_c + c_h S_c) / max(m_a, m_b)
 *   D = number of disjoint genes, n / m = number of node / connection genes,
 *   S_n = sum over homologous node pairs of |bias diff| + |response diff|
 *         + [aggregation ids differ] + [activation ids differ],
 *   S_c = sum over homologous connection pairs of |weight diff|
 *         + [enabled flags differ] (enabled <=> value != 0);
 *   a term whose denominator is 0 is 0.  A genome with a non-integer key
 *   (NEAT_G_BADKEY), a duplicated node key (NEAT_G_DUPKEY) or a duplicated
 *   connection pair (NEAT_G_DUPCONN) has NaN distances.
 * Computed in float; results are deterministic (a function of the two
 * genomes). */

/* Bytes of one genome's gene record (a multiple of 128); 0 for invalid dims. */
NEAT_API size_t neat_gene_stride(neat_dims d);

/* Gene records of `pop` genomes (nodes f32 [pop][max_nodes][5], conns f32
 * [pop][max_conns][4], device, conns 16-byte aligned) into genes_dev
 * (>= pop * neat_gene_stride(d) bytes, 16-byte aligned, caller-owned):
 * node keys and (in, out) pairs sorted, with their attributes.  status_dev
 * (optional, u32 [pop]) receives the bits above (0 = valid).
 * Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_distance_prepare(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                                   void *genes_dev, size_t genes_bytes, uint32_t *status_dev, void *stream);

/* out_dev[i * ld_out + j] = d(a_i, b_j) for i < pop_a, j < pop_b, from gene
 * records of the same dims (ld_out >= pop_b; a and b may be the same buffer).
 * Errors: NEAT_EINVAL (sizes, alignment, a record above 200 KB), NEAT_ECUDA. */
NEAT_API int neat_distance(const void *genes_a, int32_t pop_a, const void *genes_b, int32_t pop_b, neat_dims d,
                           float c_disjoint, float c_homologous, float *out_dev, int64_t ld_out, void *stream);

/* Species assignment from a distance matrix f32 [pop][ld] (device), columns
 * 0..n_reps-1 being the species representatives: species_dev[i] = the column
 * j with the smallest distance among those with distance < threshold (the
 * lowest such column on ties), or -1 when there is none (a NaN distance never
 * qualifies).  Creating new species for the -1 genomes is left to the caller.
 * Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_speciate(const float *distances_dev, int32_t pop, int32_t n_reps, int64_t ld, float threshold,
                           int32_t *species_dev, void *stream);

/* --------------------------------------------- mutation and crossover
 *
 * Tensorized NEAT operators (Section 3.2: node addition writes the first NaN
 * row, removal writes NaN over a row, attribute modification overwrites a
 * column; mutation and crossover are built from these), applied to a whole
 * population.  The paper lists the hyperparameters (below) but no algorithm;
 * this library's rules:
 *   Random numbers are inputs.  Per genome, `words` uint32 [W] and `normals`
 *   f32 [Z] (sizes from neat_mutation_sizes):
 *     words 0..8 structural: 0 node-addition decision, 1 its connection;
 *       2 node-deletion decision, 3 its node; 4 connection-addition
 *       decision, 5 its source, 6 its target; 7 connection-deletion
 *       decision, 8 its connection;
 *     node row r: words 16 + 6r + {0 bias, 1 response, 2 activation
 *       decision, 3 activation choice, 4 aggregation decision, 5 aggregation
 *       choice}; connection row c: words 16 + 6 max_nodes + 2c + {0 weight,
 *       1 enabled};
 *     normals: 0 the new connection's weight; node row r: 4 + 2r + {0 bias,
 *       1 response}; connection row c: 4 + 2 max_nodes + c.
 *   A decision with rate p happens when word < T(p) = min(floor(p 2^32), 2^32)
 *   (computed in double); a choice among k candidates (in row order) takes
 *   index floor(word k / 2^32).
 *   Present rows: node key not NaN; connection in, out, enabled not NaN.
 *   Structural steps, in order:
 *     1. node addition: a present enabled connection is disabled; the first
 *        free node row gets (new_keys[g], bias_init_mean, response_init_mean,
 *        aggregation_default, activation_default); the first free connection
 *        row (in, new, 1, 1.0) and the next (new, out, 1, old weight).
 *        Skipped without a free node row, two free connection rows, or when
 *        the new key is already present.
 *     2. node deletion: a present node with key >= I + O and every present
 *        connection touching its key become NaN rows.
 *     3. connection addition: source among present nodes, target among
 *        present nodes with key >= I.  An existing present (source, target)
 *        row is enabled instead; with `feedforward`, a self-loop or a target
 *        from which the source is reachable through present connections
 *        between present nodes is rejected; otherwise the first free row gets
 *        (source, target, 1, weight_init_mean + weight_init_std * normal).
 *     4. connection deletion: a present connection becomes a NaN row.
 *   Attribute step, every present row afterwards (node rows with key >= I):
 *     value: word < T(mutate_rate) -> value + mutate_power * normal,
 *            else word < T(mutate_rate + replace_rate) -> init_mean + init_std * normal
 *     (bias, response, weight); activation / aggregation: decision <
 *     T(replace_rate) -> options[choice]; enabled flips when its word <
 *     T(enabled_mutate_rate).
 *   Arithmetic in float with one rounding (fused multiply-add).  Genomes
 *   must have valid keys (exact integers below 2^24). */
typedef struct {
    float node_add, node_delete, conn_add, conn_delete;
    float bias_init_mean, bias_init_std, bias_mutate_power, bias_mutate_rate, bias_replace_rate;
    float response_init_mean, response_init_std, response_mutate_power, response_mutate_rate, response_replace_rate;
    float weight_init_mean, weight_init_std, weight_mutate_power, weight_mutate_rate, weight_replace_rate;
    float activation_replace_rate, aggregation_replace_rate, enabled_mutate_rate;
    int32_t activation_default, aggregation_default;
    int32_t n_activation_options, n_aggregation_options;   /* <= 8, <= 4 */
    int32_t activation_options[8], aggregation_options[4];
    int32_t feedforward;                                   /* reject connections that close a cycle */
} neat_mutation;

/* Random inputs per genome for neat_mutate: *words uint32, *normals float. */
NEAT_API int neat_mutation_sizes(neat_dims d, int64_t *words, int64_t *normals);

/* Mutate `pop` genomes in place (nodes f32 [pop][max_nodes][5], conns f32
 * [pop][max_conns][4], 16-byte aligned, device) with the rules above; words
 * uint32 [pop][W], normals f32 [pop][Z], new_keys int32 [pop] (the key a node
 * addition gives its node; unique per genome is the caller's choice).
 * Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_mutate(float *nodes_dev, float *conns_dev, int32_t pop, neat_dims d, const neat_mutation *m,
                         const uint32_t *words_dev, const float *normals_dev, const int32_t *new_keys_dev,
                         void *stream);

/* Crossover: child k of parents (parents_dev[2k], parents_dev[2k+1]), the
 * first the fitter, is the first parent's tensors, except that a present row
 * whose node key (connection (in, out) pair) is also present in the second
 * parent takes the second parent's attributes (node: bias, response,
 * aggregation, activation; connection: enabled, weight; its lowest such row)
 * when words_dev[k][row] (words_dev[k][max_nodes + row] for connections),
 * uint32 [n_children][max_nodes + max_conns], is >= 2^31.  Outputs
 * [n_children][...] must not overlap the inputs.  A child with a parent
 * index outside [0, pop) is written empty (every row NaN).  Errors:
 * NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_crossover(const float *nodes_dev, const float *conns_dev, int32_t pop, neat_dims d,
                            const int32_t *parents_dev, int32_t n_children, const uint32_t *words_dev,
                            float *nodes_out_dev, float *conns_out_dev, void *stream);

/* Random words for the operators: words_dev[e] (e < n) = component e mod 4
 * of Philox-4x32-10 (Salmon et al., SC 2011) with key `seed` applied to the
 * counter (e / 4 low 32 bits, e / 4 high 32 bits, stream low 32 bits,
 * stream high 32 bits xor 0x574f5244); distinct `stream` values give
 * independent sequences.  Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_fill_words(uint64_t seed, uint64_t stream, uint32_t *words_dev, int64_t n, void *stream_handle);

/* ---------------------------------------------------------- CPPN query
 *
 * CPPN / HyperNEAT extension (Section 4.3): each genome is a CPPN with the
 * five inputs (x_s, y_s, x_t, y_t, 1) and one output, queried at every pair
 * (source node of layer l, target node of layer l+1) of a substrate of
 * `layers` layers, each a res x res grid over [-1,1]^2 with coordinate
 * -1 + 2 i / (res - 1) (computed in double, rounded to float) and node index
 * res * iy + ix.  The weight is the CPPN output, set to 0 when
 * |w| < threshold (the comparison made in float32).
 */
typedef struct neat_substrate {
    int32_t resolution;   /* nodes per side of a layer, 2..181 */
    int32_t layers;       /* >= 2 */
} neat_substrate;

/* weights_dev: f32 [pop][layers-1][res*res][res*res] (written; NaN for
 * genomes with an error bit).  d must have num_inputs = 5, num_outputs = 1
 * and max_nodes <= 160.  Errors: NEAT_EINVAL, NEAT_ECUDA. */
NEAT_API int neat_cppn_query(const void *transformed_dev, int32_t pop, neat_dims d, neat_substrate sub,
                             float threshold, float *weights_dev, void *stream);

/* HyperNEAT substrate evaluation: the layered network that the weight
 * blocks of neat_cppn_query define (weights f32 [pop][layers-1][R][R],
 * source-major, R = resolution^2), on inputs f32 [pop][batch][R] (one value
 * per node of the first layer) -> outputs f32 [pop][batch][R] (the last
 * layer).  Layer l+1 node t = act(sum_s W_l[s][t] v_l[s]), no bias;
 * act = hidden_act for inner layers, output_act for the last (ids as for
 * nodes).  The paper gives no substrate rule; this is this library's.
 * Float arithmetic: each source sum is split into a fixed number of slices
 * of consecutive sources, each a compensated dot product (Dot2, Ogita, Rump
 * and Oishi, 2005: as accurate as twice the float precision), the slices
 * added in order with their errors carried, one rounding at the end; the
 * result is deterministic and does not depend on the batch size.  A weight
 * stage that does not arrive within the bounded wait gives NaN outputs and
 * sets the device error word (neat_device_error).  Errors: NEAT_EINVAL,
 * NEAT_ECUDA. */
NEAT_API int neat_substrate_forward(const float *weights_dev, int32_t pop, neat_substrate sub, const float *inputs_dev,
                                    int32_t batch, int32_t hidden_act, int32_t output_act, float *outputs_dev,
                                    void *stream);

/* ------------------------------------------------------------ batching
 *
 * A plan evaluates several transformed populations -- of different
 * dimensions and batch sizes -- with one persistent kernel launch per step.
 * At creation the plan reads every record header once, splits each
 * population into size buckets by node count (powers of two from 16, the
 * bucket boundaries; or one bucket per population), picks a launch shape per
 * bucket (heuristic, or timed on the plan's own data when `autotune` is set)
 * and orders the buckets' work largest first.  Each step the persistent
 * blocks pull work from a device counter, so uneven buckets balance across
 * SMs.  Results are bit-identical to neat_forward on each population (the
 * aggregation order is a function of the genome alone).
 */
typedef struct neat_pop_desc {
    const void *transformed_dev;   /* records from neat_transform */
    int32_t pop;
    neat_dims dims;
    int32_t batch;                 /* input vectors per genome per step */
    const float *inputs_dev;       /* step s reads inputs_dev + s * in_step_stride: [pop][batch][I] */
    int64_t in_step_stride;        /* floats */
    float *outputs_dev;            /* step s writes outputs_dev + s * out_step_stride: [pop][batch][O] */
    int64_t out_step_stride;       /* floats */
} neat_pop_desc;

typedef struct neat_plan_options {
    int32_t autotune;       /* 1: time candidate shapes per bucket at creation (runs kernels on the plan's buffers) */
    int32_t size_buckets;   /* 1: split populations by node count; 0: one bucket per population */
    int32_t block_threads;  /* threads of a persistent block (0: with autotune, the fastest of
                               256, 512 and 1024 on the plan's data; without, 256) */
    int32_t pdl;            /* 1: steps after the first use programmatic dependent launch */
} neat_plan_options;

typedef struct neat_plan neat_plan;

/* Build a plan (synchronous on `stream`: reads headers, allocates its tables
 * and work counters, optionally autotunes).  opt_host may be NULL (defaults:
 * size buckets on, no autotune, 256 threads, pdl on).  Errors: NEAT_EINVAL,
 * NEAT_ENOMEM, NEAT_ECUDA. */
NEAT_API int neat_plan_create(const neat_pop_desc *pops_host, int32_t npops, const neat_plan_options *opt_host,
                              void *stream, neat_plan **out_host);

/* One step for every population of the plan (one kernel launch, plus a
 * counter reset). */
NEAT_API int neat_plan_forward(neat_plan *plan, int32_t step, void *stream);

/* Steps first_step .. first_step+steps-1 as one CUDA graph (built on first
 * use for these arguments, then replayed). */
NEAT_API int neat_plan_forward_steps(neat_plan *plan, int32_t first_step, int32_t steps, void *stream);

/* JSON description of the plan's buckets and launch shapes into buf (always
 * NUL-terminated); returns the full length needed. */
NEAT_API int neat_plan_describe(const neat_plan *plan, char *buf_host, int32_t len);

/* Free the plan, its device tables and graphs (after its work completed). */
NEAT_API void neat_plan_destroy(neat_plan *plan);

/*
 * Allocation-free batched forward.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a real-time control
 * loop that must never stall on the device allocator, or a process whose
 * device memory all belongs to another framework's pool.  It evaluates one
 * step of up to 64 populations (at most 32768 genomes each) with the same
 * persistent kernel as neat_plan_forward, one bucket per population and
 * heuristic launch shapes, and allocates nothing: its scratch (work counter,
 * bucket table, genome index list; about 136 KB) is a fixed array in device
 * memory that every GPU loading this library holds until the process exits.
 * Inputs and outputs are the caller's, as in neat_pop_desc; step s reads
 * inputs_dev + s * in_step_stride and writes outputs_dev + s * out_step_stride.
 * The first call on a device, with that device current, looks up the array's
 * device address and fills its index list (a small kernel on `stream`, which
 * that call waits for before returning); make that first call before any
 * stream capture.  Each call writes its bucket table into the array with one
 * small kernel (the table is a kernel argument; nothing is copied from host
 * memory), then launches the persistent kernel.  Every call shares the array and
 * rewrites it: calls that overlap on the GPU (other streams, other threads)
 * race, so serialise them.  Results equal neat_forward on each population.
 * Errors: NEAT_EINVAL (more than 64 populations, more than 32768 genomes in
 * one, a genome too large for one block, more than 2^31 - 1 block work
 * items, bad arguments), NEAT_ECUDA.
 */
NEAT_API int neat_forward_multi_noalloc(const neat_pop_desc *pops_host, int32_t npops, int32_t step, void *stream);

/* ------------------------------------------------------------- serving
 *
 * Continuous batching of evaluation requests.  The server owns one device
 * pool of hbm_budget_bytes (allocated at create) and a scheduler thread.
 * Queued requests are admitted, in arrival order (a later one that fits may
 * pass one that does not), as pool memory frees up; their genome tensors are
 * copied in and transformed once.  Every scheduler tick advances each active
 * request by one step -- one kernel generating the step's observations, one
 * persistent-kernel launch evaluating all active requests together -- so
 * requests that arrive while others run share the device with them.  A
 * request's outputs are identical alone and in any mix.  Observations of step
 * s are N(0,1) values from a counter-based generator (Philox-4x32-10 with a
 * Box-Muller transform) keyed by the request's seed: neat_fill_normal
 * reproduces them.  Times are host steady-clock milliseconds.
 */
typedef struct neat_serve_cfg {
    uint64_t hbm_budget_bytes;  /* device pool for admitted requests */
    int32_t max_active;         /* requests evaluated together per tick, 1..4096 */
    int32_t reserved;
} neat_serve_cfg;

typedef struct neat_request {
    const float *nodes_host;    /* [pop][max_nodes][5], copied by submit */
    const float *conns_host;    /* [pop][max_conns][4], copied by submit */
    int32_t pop;                /* 1..65536 */
    neat_dims dims;
    int32_t batch;              /* input vectors per genome per step, >= 1 */
    int32_t steps;              /* >= 1 */
    int32_t flags;              /* NEAT_REQ_* */
    uint64_t obs_seed;          /* observations of step s: neat_fill_normal(obs_seed, s, pop*batch*I) */
    float *outputs_dev;         /* caller-owned until done; step s writes outputs_dev + s * out_step_stride */
    int64_t out_step_stride;    /* floats; 0: every step overwrites [pop][batch][O] */
} neat_request;

/* neat_request.flags: the server reads nodes_host/conns_host in place (no
 * copy at submit); they must stay valid until the request is done.  With
 * pinned host memory the copy at admission is asynchronous. */
#define NEAT_REQ_BORROW_HOST 1

typedef struct neat_result {
    int32_t status;             /* NEAT_OK or NEAT_ECANCELLED */
    int32_t reserved;
    double submit_ms, admit_ms, done_ms;
    uint64_t genome_forwards;   /* pop * batch * steps evaluated */
} neat_result;

typedef struct neat_serve_report {
    int32_t completed, cancelled, queued, active;
    double latency_p50_ms, latency_p99_ms;        /* submit -> last step done */
    double queue_wait_p50_ms, queue_wait_p99_ms;  /* submit -> admitted */
    uint64_t genome_forwards;
    double genome_forwards_per_s;                 /* over first submit .. last completion */
    int64_t ticks;
    uint64_t pool_used_bytes;
} neat_serve_report;

typedef struct neat_server neat_server;

/* Create a server on the current device.  Errors: NEAT_EINVAL, NEAT_ENOMEM, NEAT_ECUDA. */
NEAT_API int neat_serve_create(const neat_serve_cfg *cfg_host, neat_server **out_host);
/* Queue a request (the genome tensors are copied, unless NEAT_REQ_BORROW_HOST;
 * caller buffers may then be reused on return).  NEAT_EBUDGET if it can
 * never fit the pool. */
NEAT_API int neat_serve_submit(neat_server *srv, const neat_request *req_host, uint64_t *ticket_host);
/* NEAT_EAGAIN until the request is done; then its status and *res. */
NEAT_API int neat_serve_poll(neat_server *srv, uint64_t ticket, neat_result *res_host);
/* Block up to timeout_ms; NEAT_ETIMEOUT if still not done. */
NEAT_API int neat_serve_wait(neat_server *srv, uint64_t ticket, int32_t timeout_ms, neat_result *res_host);
/* Cancel: a queued request is dropped, an active one stops after its steps in flight. */
NEAT_API int neat_serve_cancel(neat_server *srv, uint64_t ticket);
NEAT_API int neat_serve_stats(neat_server *srv, neat_serve_report *st_host);
/* Cancel what is left, drain the device, free everything. */
NEAT_API void neat_serve_destroy(neat_server *srv);
/* The serving observations: count N(0,1) floats of (seed, step) into out_dev. */
NEAT_API int neat_fill_normal(uint64_t seed, int32_t step, int64_t count, float *out_dev, void *stream);

/*
 * Failure-detection self-test (synchronous): one GPU thread waits on an
 * mbarrier phase that never completes, with a bound of limit_us
 * microseconds.  The wait gives up, bit 0 of the device error word is set
 * (see neat_device_error) and the kernel returns; *result_host = 2.  (1 would
 * mean the phase completed, which cannot happen.)  No fault, no hang: the
 * context stays usable.
 */
NEAT_API int neat_selftest_bounded_wait(uint32_t limit_us, uint32_t *result_host);

/* Description of the last error on this thread ("" if none). */
NEAT_API const char *neat_last_error(void);

/* Library version string. */
NEAT_API const char *neat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NEAT_H */
