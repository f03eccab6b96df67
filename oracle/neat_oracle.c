/*
 * neat_oracle.c -- plain, slow, FP64 CPU oracle for population-wide NEAT
 * genome evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; every rule below is
 * restated here from the paper and from the readings listed with it.
 *
 * What it computes (Section 3.3, "Tensorized Network Inference"):
 *   transform: from the padded node tensor N^ and connection tensor C^
 *     (Section 3.1) build a topological order of the nodes and, in place of
 *     the dense expanded-connection tensor C_exp, a compact list of the
 *     enabled incoming connections of every node (disabled connections are
 *     dropped, as the C_exp rule maps them to NaN);
 *   forward: v[input keys] <- inputs; then, in topological order,
 *     v[k] <- f_n(f_c(v | incoming conns of k) | attributes of node k)
 *     with f_c(x | w) = w x and f_n(x | b, r, agg, act) = act(b + r agg(x)),
 *     and the outputs are v[output keys].
 *
 * Readings (where the paper is silent or ambiguous), all fixed here:
 *   - node row = (key, bias, response, aggregation id, activation id);
 *     conn row = (in key, out key, enabled, weight); a row is present when
 *     its key fields (node: key; conn: in, out, enabled) are not NaN.
 *   - keys are looked up, never used as indices; they must be exact integers
 *     in [0, 2^24).  Inputs are keys 0..I-1, outputs keys I..I+O-1 (the
 *     genome interface's input_idx / output_idx), at any row.
 *   - response multiplies the aggregate: z = bias + response * agg.
 *   - activation ids 0 identity, 1 tanh, 2 sigmoid 1/(1+e^-z), 3 relu
 *     max(z,0), 4 sin, 5 gauss e^(-z^2), 6 abs; aggregation ids 0 sum,
 *     1 product, 2 max, 3 mean; an empty incoming set aggregates to 0.
 *   - input nodes pass their input through; connections into an input node
 *     are ignored (warning bit).
 *   - enabled <=> e != 0.  Disabled connections take no part in the sort or
 *     the forward pass; their weight may be anything.
 *   - topological order: layered Kahn.  Level 0 = present nodes with no
 *     enabled incoming connection; level l+1 = nodes whose last remaining
 *     incoming connection came from level l.  Within a level, ascending row.
 *   - incoming connections of a node are taken in ascending connection-row
 *     order; that fixes the order of the aggregation.
 *   - a genome with any error bit gets NaN outputs.
 * Arithmetic is double; this file must be compiled with -ffp-contract=off so
 * that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* status word (error bits make the genome unusable; warnings do not) */
#define ORC_CYCLE        1u
#define ORC_DUPKEY       2u
#define ORC_BADKEY       4u
#define ORC_BADENUM      8u
#define ORC_DUPCONN     16u
#define ORC_BADATTR     32u
#define ORC_MISSING_IO  64u
#define ORC_DANGLING   256u
#define ORC_INTO_INPUT 512u
#define ORC_ERROR_MASK 0xffu

#define KEY_LIMIT 16777216.0 /* 2^24 */

typedef struct {
    int n_nodes;       /* present node rows */
    int n_levels;
    int n_edges;       /* enabled connections kept in the incoming lists */
    uint32_t status;
    int *order;        /* [Nmax] position -> node row, -1 past n_nodes */
    int *level_ptr;    /* [Nmax+1] position where each level starts */
    int *in_ptr;       /* [Nmax+1] by position: start of its incoming list */
    int *in_src;       /* [Cmax] source node row */
    int *in_conn;      /* [Cmax] connection row */
    double *in_w;      /* [Cmax] weight */
    int *row_key;      /* [Nmax] key of each row (-1 absent) */
    int *input_row;    /* [I] row holding input key j */
    int *output_row;   /* [O] row holding output key I+j */
} genome_t;

static int is_key(float k) { return !isnan(k) && k >= 0.0f && (double)k < KEY_LIMIT && floorf(k) == k; }
static int is_enum(float v, int n) { return !isnan(v) && floorf(v) == v && v >= 0.0f && v < (float)n; }

typedef struct { long key; int row; } keyrow_t;
static int cmp_keyrow(const void *a, const void *b)
{
    const keyrow_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->row - y->row;
}
typedef struct { long a, b; } pair_t;
static int cmp_pair(const void *p, const void *q)
{
    const pair_t *x = p, *y = q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}
static int cmp_int(const void *a, const void *b) { return *(const int *)a - *(const int *)b; }

/* lowest row holding a key, among the (key,row) pairs sorted by key then
 * row, or -1.  (A duplicated key is already an error; taking its lowest row
 * keeps the remaining status bits of such a genome well defined.) */
static int lookup(const keyrow_t *map, int n, long key)
{
    int lo = 0, hi = n;                    /* first pair with pair.key >= key */
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (map[mid].key < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && map[lo].key == key) ? map[lo].row : -1;
}

static void genome_alloc(genome_t *g, int I, int O, int Nmax, int Cmax)
{
    g->order = malloc(sizeof(int) * (size_t)Nmax);
    g->level_ptr = malloc(sizeof(int) * (size_t)(Nmax + 1));
    g->in_ptr = malloc(sizeof(int) * (size_t)(Nmax + 1));
    g->in_src = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    g->in_conn = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    g->in_w = malloc(sizeof(double) * (size_t)(Cmax > 0 ? Cmax : 1));
    g->row_key = malloc(sizeof(int) * (size_t)Nmax);
    g->input_row = malloc(sizeof(int) * (size_t)(I > 0 ? I : 1));
    g->output_row = malloc(sizeof(int) * (size_t)(O > 0 ? O : 1));
}

static void genome_free(genome_t *g)
{
    free(g->order); free(g->level_ptr); free(g->in_ptr); free(g->in_src);
    free(g->in_conn); free(g->in_w); free(g->row_key); free(g->input_row); free(g->output_row);
}

/*
 * Transform of one genome (Section 3.3, transformation stage): row checks,
 * key lookup, layered Kahn order, then the incoming-connection lists.
 */
static void transform_one(const float *nodes, const float *conns, int I, int O,
                          int Nmax, int Cmax, genome_t *g)
{
    uint32_t st = 0;
    int n = 0;
    keyrow_t *map = malloc(sizeof(keyrow_t) * (size_t)(Nmax > 0 ? Nmax : 1));

    /* 1. node rows: presence, key, enums, attributes (Section 3.1) */
    for (int r = 0; r < Nmax; r++) {
        const float *nd = nodes + (size_t)r * 5;
        g->row_key[r] = -1;
        if (isnan(nd[0])) continue;
        if (!is_key(nd[0])) { st |= ORC_BADKEY; continue; }
        if (!is_enum(nd[3], 4) || !is_enum(nd[4], 7)) st |= ORC_BADENUM;
        if (isnan(nd[1]) || isnan(nd[2])) st |= ORC_BADATTR;
        g->row_key[r] = (int)nd[0];
        map[n].key = (long)nd[0];
        map[n].row = r;
        n++;
    }
    qsort(map, (size_t)n, sizeof(keyrow_t), cmp_keyrow);
    for (int i = 1; i < n; i++)
        if (map[i].key == map[i - 1].key) st |= ORC_DUPKEY;
    for (int j = 0; j < I; j++) {
        g->input_row[j] = lookup(map, n, j);
        if (g->input_row[j] < 0) st |= ORC_MISSING_IO;
    }
    for (int j = 0; j < O; j++) {
        g->output_row[j] = lookup(map, n, I + j);
        if (g->output_row[j] < 0) st |= ORC_MISSING_IO;
    }

    /* 2. connection rows: presence, keys, endpoints, duplicates */
    int *src = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    int *dst = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    pair_t *pairs = malloc(sizeof(pair_t) * (size_t)(Cmax > 0 ? Cmax : 1));
    int npairs = 0;
    for (int c = 0; c < Cmax; c++) {
        const float *cn = conns + (size_t)c * 4;
        src[c] = dst[c] = -1;              /* -1: not an active edge */
        if (isnan(cn[0]) || isnan(cn[1]) || isnan(cn[2])) continue;
        if (!is_key(cn[0]) || !is_key(cn[1])) { st |= ORC_BADKEY; continue; }
        pairs[npairs].a = (long)cn[0];
        pairs[npairs].b = (long)cn[1];
        npairs++;
        if (cn[2] == 0.0f) continue;       /* disabled: C_exp entry is NaN */
        if (isnan(cn[3])) st |= ORC_BADATTR;
        int s = lookup(map, n, (long)cn[0]);
        int d = lookup(map, n, (long)cn[1]);
        if (s < 0 || d < 0) { st |= ORC_DANGLING; continue; }
        if ((long)cn[1] < I) { st |= ORC_INTO_INPUT; continue; }
        src[c] = s;
        dst[c] = d;
    }
    qsort(pairs, (size_t)npairs, sizeof(pair_t), cmp_pair);
    for (int i = 1; i < npairs; i++)
        if (pairs[i].a == pairs[i - 1].a && pairs[i].b == pairs[i - 1].b) st |= ORC_DUPCONN;

    /* out-edges and in-edges of every row, each in ascending connection row */
    int *out_ptr = calloc((size_t)Nmax + 1, sizeof(int));
    int *inc_ptr = calloc((size_t)Nmax + 1, sizeof(int));
    int *out_list = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    int *inc_list = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    for (int c = 0; c < Cmax; c++)
        if (dst[c] >= 0) { out_ptr[src[c] + 1]++; inc_ptr[dst[c] + 1]++; }
    for (int r = 0; r < Nmax; r++) { out_ptr[r + 1] += out_ptr[r]; inc_ptr[r + 1] += inc_ptr[r]; }
    {
        int *ofill = malloc(sizeof(int) * (size_t)(Nmax > 0 ? Nmax : 1));
        int *ifill = malloc(sizeof(int) * (size_t)(Nmax > 0 ? Nmax : 1));
        memcpy(ofill, out_ptr, sizeof(int) * (size_t)Nmax);
        memcpy(ifill, inc_ptr, sizeof(int) * (size_t)Nmax);
        for (int c = 0; c < Cmax; c++)
            if (dst[c] >= 0) { out_list[ofill[src[c]]++] = c; inc_list[ifill[dst[c]]++] = c; }
        free(ofill); free(ifill);
    }

    /* 3. layered Kahn over the active edges */
    int *indeg = calloc((size_t)(Nmax > 0 ? Nmax : 1), sizeof(int));
    for (int r = 0; r < Nmax; r++) indeg[r] = inc_ptr[r + 1] - inc_ptr[r];
    int placed = 0, levels = 0;
    g->level_ptr[0] = 0;
    for (int r = 0; r < Nmax; r++)            /* level 0, ascending row */
        if (g->row_key[r] >= 0 && indeg[r] == 0) g->order[placed++] = r;
    int level_start = 0;
    while (placed > level_start) {
        int level_end = placed;
        levels++;
        g->level_ptr[levels] = level_end;
        /* remove this level's out-edges; nodes left with none form the next */
        for (int p = level_start; p < level_end; p++) {
            int r = g->order[p];
            for (int i = out_ptr[r]; i < out_ptr[r + 1]; i++) {
                int d = dst[out_list[i]];
                if (--indeg[d] == 0) g->order[placed++] = d;
            }
        }
        qsort(g->order + level_end, (size_t)(placed - level_end), sizeof(int), cmp_int);
        level_start = level_end;
    }
    if (placed < n) st |= ORC_CYCLE;
    for (int p = placed; p < Nmax; p++) g->order[p] = -1;
    for (int l = levels + 1; l <= Nmax; l++) g->level_ptr[l] = placed;

    /* 4. incoming lists by destination position, ascending connection row */
    int e = 0;
    for (int p = 0; p < placed; p++) {
        g->in_ptr[p] = e;
        int r = g->order[p];
        for (int i = inc_ptr[r]; i < inc_ptr[r + 1]; i++) {
            int c = inc_list[i];
            g->in_src[e] = src[c];
            g->in_conn[e] = c;
            g->in_w[e] = (double)conns[(size_t)c * 4 + 3];
            e++;
        }
    }
    for (int p = placed; p <= Nmax; p++) g->in_ptr[p] = e;
    for (int i = e; i < Cmax; i++) { g->in_src[i] = -1; g->in_conn[i] = -1; g->in_w[i] = 0.0; }

    g->n_nodes = n;
    g->n_levels = (placed < n) ? 0 : levels;
    g->n_edges = e;
    g->status = st;
    free(indeg); free(out_ptr); free(inc_ptr); free(out_list); free(inc_list);
    free(pairs); free(dst); free(src); free(map);
}

/* activation functions (reading listed in the file header) */
static double act_fn(int id, double z)
{
    switch (id) {
    case 0: return z;
    case 1: return tanh(z);
    case 2: return 1.0 / (1.0 + exp(-z));
    case 3: return fmax(z, 0.0);
    case 4: return sin(z);
    case 5: return exp(-(z * z));
    case 6: return fabs(z);
    }
    return NAN;
}

/* f_n(f_c(...)) for one node: terms w * v[src] in list order, then agg */
static double node_value(const genome_t *g, const float *node_row, int p, const double *v)
{
    int b = g->in_ptr[p], e = g->in_ptr[p + 1];
    int agg = (int)node_row[3];
    double a = 0.0;
    if (e > b) {
        if (agg == 0 || agg == 3) {
            for (int i = b; i < e; i++) a = a + g->in_w[i] * v[g->in_src[i]];
            if (agg == 3) a = a / (double)(e - b);
        } else if (agg == 1) {
            a = 1.0;
            for (int i = b; i < e; i++) a = a * (g->in_w[i] * v[g->in_src[i]]);
        } else {
            a = g->in_w[b] * v[g->in_src[b]];
            for (int i = b + 1; i < e; i++) a = fmax(a, g->in_w[i] * v[g->in_src[i]]);
        }
    }
    double z = (double)node_row[1] + (double)node_row[2] * a;
    return act_fn((int)node_row[4], z);
}

/* forward of one transformed genome on one input vector x[I] -> y[O] */
static void forward_one(const genome_t *g, const float *nodes, int I, int O,
                        const float *x, double *v, double *y)
{
    if (g->status & ORC_ERROR_MASK) {
        for (int j = 0; j < O; j++) y[j] = NAN;
        return;
    }
    for (int j = 0; j < I; j++) v[g->input_row[j]] = (double)x[j];
    for (int p = 0; p < g->n_nodes; p++) {
        int r = g->order[p];
        if (g->row_key[r] < I) continue;          /* input node: pass-through */
        v[r] = node_value(g, nodes + (size_t)r * 5, p, v);
    }
    for (int j = 0; j < O; j++) y[j] = v[g->output_row[j]];
}

/* ---------------------------------------------------------------- exports */

/* Transform P genomes.  Outputs (all caller-allocated host arrays):
 *   order[P][Nmax] node row per position (-1 pad), level_ptr[P][Nmax+1],
 *   n_levels[P], n_nodes[P], n_edges[P], in_ptr[P][Nmax+1] (by position),
 *   in_src[P][Cmax] (source row), in_conn[P][Cmax] (connection row),
 *   in_w[P][Cmax] (weight as double), status[P].  Returns 0. */
int oracle_transform(const float *nodes, const float *conns, int P, int I, int O,
                     int Nmax, int Cmax, int32_t *order, int32_t *level_ptr,
                     int32_t *n_levels, int32_t *n_nodes, int32_t *n_edges,
                     int32_t *in_ptr, int32_t *in_src, int32_t *in_conn, double *in_w,
                     uint32_t *status)
{
    genome_t g;
    genome_alloc(&g, I, O, Nmax, Cmax);
    for (int k = 0; k < P; k++) {
        transform_one(nodes + (size_t)k * Nmax * 5, conns + (size_t)k * Cmax * 4, I, O, Nmax, Cmax, &g);
        for (int p = 0; p < Nmax; p++) order[(size_t)k * Nmax + p] = g.order[p];
        for (int p = 0; p <= Nmax; p++) {
            level_ptr[(size_t)k * (Nmax + 1) + p] = g.level_ptr[p];
            in_ptr[(size_t)k * (Nmax + 1) + p] = g.in_ptr[p];
        }
        for (int i = 0; i < Cmax; i++) {
            in_src[(size_t)k * Cmax + i] = g.in_src[i];
            in_conn[(size_t)k * Cmax + i] = g.in_conn[i];
            in_w[(size_t)k * Cmax + i] = g.in_w[i];
        }
        n_levels[k] = g.n_levels;
        n_nodes[k] = g.n_nodes;
        n_edges[k] = g.n_edges;
        status[k] = g.status;
    }
    genome_free(&g);
    return 0;
}

/* Forward of P genomes, B input vectors each: inputs[P][B][I] -> out[P][B][O]
 * (double).  Each genome is transformed once, then evaluated B times. */
int oracle_forward(const float *nodes, const float *conns, int P, int I, int O,
                   int Nmax, int Cmax, const float *inputs, int B, double *out)
{
    genome_t g;
    genome_alloc(&g, I, O, Nmax, Cmax);
    double *v = malloc(sizeof(double) * (size_t)(Nmax > 0 ? Nmax : 1));
    for (int k = 0; k < P; k++) {
        const float *nd = nodes + (size_t)k * Nmax * 5;
        transform_one(nd, conns + (size_t)k * Cmax * 4, I, O, Nmax, Cmax, &g);
        for (int b = 0; b < B; b++)
            forward_one(&g, nd, I, O, inputs + ((size_t)k * B + b) * I, v,
                        out + ((size_t)k * B + b) * O);
    }
    free(v);
    genome_free(&g);
    return 0;
}

/*
 * CPPN query on a HyperNEAT substrate (Section 4.3, CPPN and HyperNEAT
 * extensions).  Substrate: `layers` layers of res x res nodes on a grid over
 * [-1,1]^2, node index = res*iy + ix with coordinate -1 + 2*i/(res-1).  Block
 * l (0 <= l < layers-1) connects layer l to layer l+1; the CPPN (inputs
 * x_s, y_s, x_d, y_d, 1; one output) is queried at every (src, dst) pair and
 * the weight is zeroed when |w| < threshold, the comparison made on w rounded
 * to float.  The genomes must have I = 5, O = 1.
 * Query list q[Q][4] = (genome, block, src, dst); raw[Q] gets the CPPN value,
 * weight[Q] the thresholded weight.  Genomes are transformed once each, in
 * the order they first appear in the list.
 */
int oracle_cppn_query(const float *nodes, const float *conns, int P, int Nmax, int Cmax,
                      int res, float threshold, const int32_t *q, long Q,
                      double *raw, double *weight)
{
    genome_t g;
    genome_alloc(&g, 5, 1, Nmax, Cmax);
    double *v = malloc(sizeof(double) * (size_t)(Nmax > 0 ? Nmax : 1));
    int cur = -1;
    for (long i = 0; i < Q; i++) {
        int k = q[i * 4 + 0];
        if (k < 0 || k >= P) { raw[i] = weight[i] = NAN; continue; }
        if (k != cur) {
            transform_one(nodes + (size_t)k * Nmax * 5, conns + (size_t)k * Cmax * 4, 5, 1, Nmax, Cmax, &g);
            cur = k;
        }
        int s = q[i * 4 + 2], d = q[i * 4 + 3];
        float x[5];
        x[0] = (float)(-1.0 + 2.0 * (double)(s % res) / (double)(res - 1));
        x[1] = (float)(-1.0 + 2.0 * (double)(s / res) / (double)(res - 1));
        x[2] = (float)(-1.0 + 2.0 * (double)(d % res) / (double)(res - 1));
        x[3] = (float)(-1.0 + 2.0 * (double)(d / res) / (double)(res - 1));
        x[4] = 1.0f;
        double y;
        forward_one(&g, nodes + (size_t)k * Nmax * 5, 5, 1, x, v, &y);
        raw[i] = y;
        weight[i] = (fabsf((float)y) < threshold) ? 0.0 : y;
    }
    free(v);
    genome_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------
 * Recurrent networks (Section 3.3 divides networks into feedforward and
 * recurrent ones by the presence of cycles, and the hyperparameters carry a
 * network_type; the paper gives no recurrent algorithm).  Reading, fixed
 * here: enabled connections may form cycles, self-loops included; the input
 * nodes hold their inputs; every other node starts at 0 and K synchronous
 * iterations follow, each node's new value computed from the previous
 * iterate of its sources by the same node rule:
 *   v_k[n] = act_n(bias_n + response_n * agg_n(w_c v_{k-1}[src_c])).
 * The outputs are v_K at the output keys.  The row checks and status bits
 * are the feedforward ones except ORC_CYCLE, which cannot occur.
 */
typedef struct {
    uint32_t status;
    int n_nodes;
    int *row_key;      /* [Nmax] */
    int *in_ptr;       /* [Nmax+1] by row */
    int *in_src;       /* [Cmax] source row */
    double *in_w;      /* [Cmax] */
    int *input_row, *output_row;
} rnn_t;

static void rnn_build(const float *nodes, const float *conns, int I, int O, int Nmax, int Cmax, rnn_t *g)
{
    uint32_t st = 0;
    int n = 0;
    keyrow_t *map = malloc(sizeof(keyrow_t) * (size_t)(Nmax > 0 ? Nmax : 1));
    for (int r = 0; r < Nmax; r++) {
        const float *nd = nodes + (size_t)r * 5;
        g->row_key[r] = -1;
        if (isnan(nd[0])) continue;
        if (!is_key(nd[0])) { st |= ORC_BADKEY; continue; }
        if (!is_enum(nd[3], 4) || !is_enum(nd[4], 7)) st |= ORC_BADENUM;
        if (isnan(nd[1]) || isnan(nd[2])) st |= ORC_BADATTR;
        g->row_key[r] = (int)nd[0];
        map[n].key = (long)nd[0];
        map[n].row = r;
        n++;
    }
    qsort(map, (size_t)n, sizeof(keyrow_t), cmp_keyrow);
    for (int i = 1; i < n; i++)
        if (map[i].key == map[i - 1].key) st |= ORC_DUPKEY;
    for (int j = 0; j < I; j++) {
        g->input_row[j] = lookup(map, n, j);
        if (g->input_row[j] < 0) st |= ORC_MISSING_IO;
    }
    for (int j = 0; j < O; j++) {
        g->output_row[j] = lookup(map, n, I + j);
        if (g->output_row[j] < 0) st |= ORC_MISSING_IO;
    }
    int *dst = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    int *src = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    pair_t *pairs = malloc(sizeof(pair_t) * (size_t)(Cmax > 0 ? Cmax : 1));
    int npairs = 0;
    for (int c = 0; c < Cmax; c++) {
        const float *cn = conns + (size_t)c * 4;
        src[c] = dst[c] = -1;
        if (isnan(cn[0]) || isnan(cn[1]) || isnan(cn[2])) continue;
        if (!is_key(cn[0]) || !is_key(cn[1])) { st |= ORC_BADKEY; continue; }
        pairs[npairs].a = (long)cn[0];
        pairs[npairs].b = (long)cn[1];
        npairs++;
        if (cn[2] == 0.0f) continue;
        if (isnan(cn[3])) st |= ORC_BADATTR;
        int s = lookup(map, n, (long)cn[0]), d = lookup(map, n, (long)cn[1]);
        if (s < 0 || d < 0) { st |= ORC_DANGLING; continue; }
        if ((long)cn[1] < I) { st |= ORC_INTO_INPUT; continue; }
        src[c] = s;
        dst[c] = d;
    }
    qsort(pairs, (size_t)npairs, sizeof(pair_t), cmp_pair);
    for (int i = 1; i < npairs; i++)
        if (pairs[i].a == pairs[i - 1].a && pairs[i].b == pairs[i - 1].b) st |= ORC_DUPCONN;
    /* incoming lists by destination row, ascending connection row */
    int e = 0;
    for (int r = 0; r < Nmax; r++) {
        g->in_ptr[r] = e;
        for (int c = 0; c < Cmax; c++) {
            if (dst[c] != r) continue;
            g->in_src[e] = src[c];
            g->in_w[e] = (double)conns[(size_t)c * 4 + 3];
            e++;
        }
    }
    g->in_ptr[Nmax] = e;
    g->n_nodes = n;
    g->status = st;
    free(pairs); free(src); free(dst); free(map);
}

/* One input vector: K synchronous iterations; y[O]. */
static void rnn_forward_one(const rnn_t *g, const float *nodes, int I, int O, int Nmax, int K,
                            const float *x, double *v, double *vn, double *y)
{
    if (g->status & ORC_ERROR_MASK) {
        for (int j = 0; j < O; j++) y[j] = NAN;
        return;
    }
    for (int r = 0; r < Nmax; r++) v[r] = 0.0;
    for (int j = 0; j < I; j++) v[g->input_row[j]] = (double)x[j];
    for (int k = 0; k < K; k++) {
        for (int r = 0; r < Nmax; r++) {
            vn[r] = v[r];
            if (g->row_key[r] < I) continue;       /* absent rows and inputs keep their value */
            const float *nd = nodes + (size_t)r * 5;
            int b = g->in_ptr[r], e = g->in_ptr[r + 1];
            int agg = (int)nd[3];
            double a = 0.0;
            if (e > b) {
                if (agg == 0 || agg == 3) {
                    for (int i = b; i < e; i++) a = a + g->in_w[i] * v[g->in_src[i]];
                    if (agg == 3) a = a / (double)(e - b);
                } else if (agg == 1) {
                    a = 1.0;
                    for (int i = b; i < e; i++) a = a * (g->in_w[i] * v[g->in_src[i]]);
                } else {
                    a = g->in_w[b] * v[g->in_src[b]];
                    for (int i = b + 1; i < e; i++) a = fmax(a, g->in_w[i] * v[g->in_src[i]]);
                }
            }
            vn[r] = act_fn((int)nd[4], (double)nd[1] + (double)nd[2] * a);
        }
        double *t = v; v = vn; vn = t;
    }
    for (int j = 0; j < O; j++) y[j] = v[g->output_row[j]];
}

/* Recurrent forward of P genomes, B input vectors each, K iterations:
 * inputs[P][B][I] -> out[P][B][O]; status[P] (may be NULL). */
int oracle_forward_recurrent(const float *nodes, const float *conns, int P, int I, int O, int Nmax, int Cmax,
                             const float *inputs, int B, int K, double *out, uint32_t *status)
{
    rnn_t g;
    g.row_key = malloc(sizeof(int) * (size_t)Nmax);
    g.in_ptr = malloc(sizeof(int) * (size_t)(Nmax + 1));
    g.in_src = malloc(sizeof(int) * (size_t)(Cmax > 0 ? Cmax : 1));
    g.in_w = malloc(sizeof(double) * (size_t)(Cmax > 0 ? Cmax : 1));
    g.input_row = malloc(sizeof(int) * (size_t)(I > 0 ? I : 1));
    g.output_row = malloc(sizeof(int) * (size_t)(O > 0 ? O : 1));
    double *v = malloc(sizeof(double) * (size_t)Nmax), *vn = malloc(sizeof(double) * (size_t)Nmax);
    for (int k = 0; k < P; k++) {
        const float *nd = nodes + (size_t)k * Nmax * 5;
        rnn_build(nd, conns + (size_t)k * Cmax * 4, I, O, Nmax, Cmax, &g);
        if (status) status[k] = g.status;
        for (int b = 0; b < B; b++)
            rnn_forward_one(&g, nd, I, O, Nmax, K, inputs + ((size_t)k * B + b) * I, v, vn,
                            out + ((size_t)k * B + b) * O);
    }
    free(v); free(vn);
    free(g.row_key); free(g.in_ptr); free(g.in_src); free(g.in_w); free(g.input_row); free(g.output_row);
    return 0;
}

/*
 * Genome distance for speciation.  Algorithm 1 divides the population into
 * species by distances between networks; the hyperparameters name a weight
 * for disjoint genes (compatibility_disjoint), a weight for homologous genes
 * (compatibility_homologous) and a speciation threshold; the gene interface
 * gives every gene a distance.  The paper states no formula, so this oracle
 * fixes the following reading:
 *   - genes are the present rows of N^ and C^ (inputs included; disabled
 *     connections included).  Node genes are homologous when their keys are
 *     equal, connection genes when their (in key, out key) pairs are equal;
 *     a gene present in only one genome is disjoint (no excess/disjoint
 *     distinction: the paper has one weight).
 *   - node gene distance |bias diff| + |response diff| + [aggregation ids
 *     differ] + [activation ids differ]; connection gene distance
 *     |weight diff| + [enabled flags differ], enabled <=> e != 0.
 *   - d = (c_d D_n + c_h S_n) / max(n_a, n_b) + (c_d D_c + c_h S_c) / max(m_a, m_b),
 *     D = disjoint count, S = sum of homologous gene distances, n / m = the
 *     genomes' node / connection gene counts; a term whose denominator is 0
 *     is 0.
 *   - a genome with a non-integer key, a duplicated node key or a duplicated
 *     connection pair has no well-defined homology: its distances are NaN.
 * The matching is the plain all-pairs comparison of the two genomes' rows.
 */
static uint32_t gene_status(const float *nodes, const float *conns, int Nmax, int Cmax)
{
    uint32_t st = 0;
    for (int r = 0; r < Nmax; r++) {
        const float k = nodes[(size_t)r * 5];
        if (isnan(k)) continue;
        if (!is_key(k)) { st |= ORC_BADKEY; continue; }
        for (int q = 0; q < r; q++)
            if (nodes[(size_t)q * 5] == k) st |= ORC_DUPKEY;
    }
    for (int c = 0; c < Cmax; c++) {
        const float *cn = conns + (size_t)c * 4;
        if (isnan(cn[0]) || isnan(cn[1]) || isnan(cn[2])) continue;
        if (!is_key(cn[0]) || !is_key(cn[1])) { st |= ORC_BADKEY; continue; }
        for (int q = 0; q < c; q++) {
            const float *cq = conns + (size_t)q * 4;
            if (isnan(cq[0]) || isnan(cq[1]) || isnan(cq[2])) continue;
            if (cq[0] == cn[0] && cq[1] == cn[1]) st |= ORC_DUPCONN;
        }
    }
    return st;
}

static double pair_distance(const float *na, const float *ca, const float *nb, const float *cb,
                            int Nmax, int Cmax, double c_d, double c_h)
{
    int n_a = 0, n_b = 0, hom = 0;
    double s = 0.0;
    for (int r = 0; r < Nmax; r++) n_a += !isnan(na[(size_t)r * 5]);
    for (int r = 0; r < Nmax; r++) n_b += !isnan(nb[(size_t)r * 5]);
    for (int i = 0; i < Nmax; i++) {
        const float *x = na + (size_t)i * 5;
        if (isnan(x[0])) continue;
        for (int j = 0; j < Nmax; j++) {
            const float *y = nb + (size_t)j * 5;
            if (isnan(y[0]) || y[0] != x[0]) continue;
            hom++;
            s += fabs((double)x[1] - (double)y[1]) + fabs((double)x[2] - (double)y[2]) +
                 (x[3] != y[3] ? 1.0 : 0.0) + (x[4] != y[4] ? 1.0 : 0.0);
        }
    }
    const int nmax = n_a > n_b ? n_a : n_b;
    const double d_nodes = nmax ? (c_d * (double)(n_a + n_b - 2 * hom) + c_h * s) / (double)nmax : 0.0;

    int m_a = 0, m_b = 0;
    hom = 0;
    s = 0.0;
    for (int c = 0; c < Cmax; c++) {
        const float *x = ca + (size_t)c * 4;
        m_a += !(isnan(x[0]) || isnan(x[1]) || isnan(x[2]));
    }
    for (int c = 0; c < Cmax; c++) {
        const float *y = cb + (size_t)c * 4;
        m_b += !(isnan(y[0]) || isnan(y[1]) || isnan(y[2]));
    }
    for (int i = 0; i < Cmax; i++) {
        const float *x = ca + (size_t)i * 4;
        if (isnan(x[0]) || isnan(x[1]) || isnan(x[2])) continue;
        for (int j = 0; j < Cmax; j++) {
            const float *y = cb + (size_t)j * 4;
            if (isnan(y[0]) || isnan(y[1]) || isnan(y[2])) continue;
            if (y[0] != x[0] || y[1] != x[1]) continue;
            hom++;
            s += fabs((double)x[3] - (double)y[3]) + (((x[2] != 0.0f) != (y[2] != 0.0f)) ? 1.0 : 0.0);
        }
    }
    const int mmax = m_a > m_b ? m_a : m_b;
    const double d_conns = mmax ? (c_d * (double)(m_a + m_b - 2 * hom) + c_h * s) / (double)mmax : 0.0;
    return d_nodes + d_conns;
}

int oracle_distance(const float *nodes_a, const float *conns_a, int PA, const float *nodes_b,
                    const float *conns_b, int PB, int Nmax, int Cmax, double c_d, double c_h,
                    double *out, uint32_t *status_a, uint32_t *status_b)
{
    for (int a = 0; a < PA; a++)
        status_a[a] = gene_status(nodes_a + (size_t)a * Nmax * 5, conns_a + (size_t)a * Cmax * 4, Nmax, Cmax);
    for (int b = 0; b < PB; b++)
        status_b[b] = gene_status(nodes_b + (size_t)b * Nmax * 5, conns_b + (size_t)b * Cmax * 4, Nmax, Cmax);
    for (int a = 0; a < PA; a++)
        for (int b = 0; b < PB; b++)
            out[(size_t)a * PB + b] =
                (status_a[a] | status_b[b]) ? NAN
                                            : pair_distance(nodes_a + (size_t)a * Nmax * 5,
                                                            conns_a + (size_t)a * Cmax * 4,
                                                            nodes_b + (size_t)b * Nmax * 5,
                                                            conns_b + (size_t)b * Cmax * 4, Nmax, Cmax, c_d, c_h);
    return 0;
}
