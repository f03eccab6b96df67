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

/*
 * Tensorized mutation and crossover (Section 3.2: node addition writes the
 * first NaN row, removal writes NaN over a row, attribute modification
 * overwrites one column; the operators are built from these).  The paper
 * names the operator hyperparameters but not an algorithm; this oracle fixes
 * the following reading.  Every random number is an input:
 *   u[W] uint32 words per genome, W = 16 + 6 Nmax + 2 Cmax:
 *     0..8 structural (below); node row r: 16 + 6r + {0 bias, 1 response,
 *     2 activation decision, 3 activation choice, 4 aggregation decision,
 *     5 aggregation choice}; connection row c: 16 + 6 Nmax + 2c + {0 weight,
 *     1 enabled};
 *   z[Z] float normals per genome, Z = 4 + 2 Nmax + Cmax: 0 new connection
 *     weight; node row r: 4 + 2r + {0 bias, 1 response}; connection row c:
 *     4 + 2 Nmax + c.
 *   Bernoulli(p) with word u: u < T(p), T(p) = min(floor(p 2^32), 2^32)
 *   (computed in double); choice among k with word u: floor(u k / 2^32).
 * Present rows: node key not NaN; connection in, out and enabled not NaN.
 * Free rows are the others; "first" means lowest row index.
 * Structural steps, in order (each independent draw):
 *   1. node addition (word 0): among present enabled connections pick one
 *      (word 1); needs a free node row, two free connection rows and a new
 *      key not present.  The connection is disabled; the first free node row
 *      gets (new key, bias_init_mean, response_init_mean, aggregation
 *      default, activation default); the first free connection row gets
 *      (in, new, 1, 1.0) and the next (new, out, 1, old weight).
 *   2. node deletion (word 2): among present nodes with key >= I + O pick
 *      one (word 3); its row and every present connection row touching its
 *      key become NaN.
 *   3. connection addition (word 4): source among present nodes (word 5),
 *      target among present nodes with key >= I (word 6).  An existing
 *      present (source, target) row is enabled instead (the first such row);
 *      otherwise, for feedforward networks, a self-loop or a target from
 *      which the source is reachable through present connections between
 *      present nodes is rejected; otherwise the first free connection row gets (source,
 *      target, 1, weight_init_mean + weight_init_std z[0]).
 *   4. connection deletion (word 7): among present connections pick one
 *      (word 8); its row becomes NaN.
 * Attribute step, every present row afterwards: node rows with key >= I:
 *   bias: u < T(mutate_rate) -> bias + mutate_power z;
 *         else u < T(mutate_rate + replace_rate) -> init_mean + init_std z;
 *   response the same with its own parameters;
 *   activation: decision < T(replace_rate) -> options[choice];
 *   aggregation the same.  Connection rows: weight as bias; enabled flips
 *   (0 <-> 1, any non-zero counting as enabled) when its word < T(rate).
 * Crossover of parents (p1, p2), p1 the fitter: the child is p1's tensors;
 * a present row of p1 whose node key (connection (in, out) pair), a valid
 * key, is present in p2 takes p2's attributes (node: bias, response, aggregation,
 * activation; connection: enabled, weight; p2's lowest such row) when its
 * word u[row] (u[Nmax + row] for connections) is >= 2^31.
 */
typedef struct {
    float node_add, node_delete, conn_add, conn_delete;
    float bias_init_mean, bias_init_std, bias_mutate_power, bias_mutate_rate, bias_replace_rate;
    float response_init_mean, response_init_std, response_mutate_power, response_mutate_rate, response_replace_rate;
    float weight_init_mean, weight_init_std, weight_mutate_power, weight_mutate_rate, weight_replace_rate;
    float activation_replace_rate, aggregation_replace_rate, enabled_mutate_rate;
    int activation_default, aggregation_default;
    int n_activation_options, n_aggregation_options;
    int activation_options[8], aggregation_options[4];
    int feedforward;
} orc_mutation_t;

static uint64_t thr_of(double p)
{
    if (!(p > 0.0)) return 0;
    const double t = floor(p * 4294967296.0);
    return t >= 4294967296.0 ? 4294967296ull : (uint64_t)t;
}
static int bern(uint32_t u, double p) { return (uint64_t)u < thr_of(p); }
static int choice(uint32_t u, int k) { return (int)(((uint64_t)u * (uint64_t)k) >> 32); }

static int node_present(const double *nd, int r) { return !isnan(nd[(size_t)r * 5]); }
static int conn_present(const double *cn, int c)
{
    const double *x = cn + (size_t)c * 4;
    return !(isnan(x[0]) || isnan(x[1]) || isnan(x[2]));
}
static int first_free_node(const double *nd, int N)
{
    for (int r = 0; r < N; r++) if (!node_present(nd, r)) return r;
    return -1;
}
static int nth_free_conn(const double *cn, int C, int n)
{
    for (int c = 0; c < C; c++) if (!conn_present(cn, c) && n-- == 0) return c;
    return -1;
}

static int key_present(const double *nd, int N, double k)
{
    for (int r = 0; r < N; r++) if (node_present(nd, r) && nd[(size_t)r * 5] == k) return 1;
    return 0;
}

/* is `to` reachable from `from` along present connections between present
 * nodes (dangling connections take no part, as in the transform)? */
static int reachable(const double *nd, const double *cn, int N, int C, double from, double to)
{
    double *seen = malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int ns = 0, found = (from == to);
    seen[ns++] = from;
    for (int changed = 1; changed && !found;) {
        changed = 0;
        for (int c = 0; c < C && !found; c++) {
            if (!conn_present(cn, c)) continue;
            const double a = cn[(size_t)c * 4], b = cn[(size_t)c * 4 + 1];
            if (!key_present(nd, N, a) || !key_present(nd, N, b)) continue;
            int has_a = 0, has_b = 0;
            for (int i = 0; i < ns; i++) { has_a |= seen[i] == a; has_b |= seen[i] == b; }
            if (has_a && !has_b) {
                if (ns < N) seen[ns++] = b;
                changed = 1;
                if (b == to) found = 1;
            }
        }
    }
    (void)nd;
    free(seen);
    return found;
}

static void mutate_one(double *nd, double *cn, int I, int O, int N, int C, const orc_mutation_t *m,
                       const uint32_t *u, const float *z, int new_key)
{
    /* 1. node addition */
    if (bern(u[0], m->node_add)) {
        int k = 0;
        for (int c = 0; c < C; c++) k += conn_present(cn, c) && cn[(size_t)c * 4 + 2] != 0.0;
        int key_used = 0;
        for (int r = 0; r < N; r++) key_used |= node_present(nd, r) && nd[(size_t)r * 5] == (double)new_key;
        const int rn = first_free_node(nd, N), ra = nth_free_conn(cn, C, 0), rb = nth_free_conn(cn, C, 1);
        if (k > 0 && rn >= 0 && ra >= 0 && rb >= 0 && !key_used) {
            int pick = choice(u[1], k), cs = -1;
            for (int c = 0; c < C; c++)
                if (conn_present(cn, c) && cn[(size_t)c * 4 + 2] != 0.0 && pick-- == 0) { cs = c; break; }
            double *x = cn + (size_t)cs * 4;
            const double in = x[0], out = x[1], w = x[3];
            x[2] = 0.0;
            double *n = nd + (size_t)rn * 5;
            n[0] = new_key; n[1] = m->bias_init_mean; n[2] = m->response_init_mean;
            n[3] = m->aggregation_default; n[4] = m->activation_default;
            double *a = cn + (size_t)ra * 4, *b = cn + (size_t)rb * 4;
            a[0] = in; a[1] = new_key; a[2] = 1.0; a[3] = 1.0;
            b[0] = new_key; b[1] = out; b[2] = 1.0; b[3] = w;
        }
    }
    /* 2. node deletion */
    if (bern(u[2], m->node_delete)) {
        int k = 0;
        for (int r = 0; r < N; r++) k += node_present(nd, r) && nd[(size_t)r * 5] >= (double)(I + O);
        if (k > 0) {
            int pick = choice(u[3], k);
            for (int r = 0; r < N; r++) {
                if (!(node_present(nd, r) && nd[(size_t)r * 5] >= (double)(I + O)) || pick-- != 0) continue;
                const double q = nd[(size_t)r * 5];
                for (int j = 0; j < 5; j++) nd[(size_t)r * 5 + j] = NAN;
                for (int c = 0; c < C; c++)
                    if (conn_present(cn, c) && (cn[(size_t)c * 4] == q || cn[(size_t)c * 4 + 1] == q))
                        for (int j = 0; j < 4; j++) cn[(size_t)c * 4 + j] = NAN;
                break;
            }
        }
    }
    /* 3. connection addition */
    if (bern(u[4], m->conn_add)) {
        int ks = 0, kt = 0;
        for (int r = 0; r < N; r++) {
            ks += node_present(nd, r);
            kt += node_present(nd, r) && nd[(size_t)r * 5] >= (double)I;
        }
        if (ks > 0 && kt > 0) {
            int ps = choice(u[5], ks), pt = choice(u[6], kt);
            double s = 0, t = 0;
            for (int r = 0; r < N; r++) if (node_present(nd, r) && ps-- == 0) { s = nd[(size_t)r * 5]; break; }
            for (int r = 0; r < N; r++)
                if (node_present(nd, r) && nd[(size_t)r * 5] >= (double)I && pt-- == 0) { t = nd[(size_t)r * 5]; break; }
            int existing = -1;
            for (int c = 0; c < C; c++)
                if (conn_present(cn, c) && cn[(size_t)c * 4] == s && cn[(size_t)c * 4 + 1] == t) { existing = c; break; }
            if (existing >= 0) {
                cn[(size_t)existing * 4 + 2] = 1.0;
            } else if (!(m->feedforward && reachable(nd, cn, N, C, t, s))) {
                const int rf = nth_free_conn(cn, C, 0);
                if (rf >= 0) {
                    double *x = cn + (size_t)rf * 4;
                    x[0] = s; x[1] = t; x[2] = 1.0;
                    x[3] = (double)m->weight_init_mean + (double)m->weight_init_std * (double)z[0];
                }
            }
        }
    }
    /* 4. connection deletion */
    if (bern(u[7], m->conn_delete)) {
        int k = 0;
        for (int c = 0; c < C; c++) k += conn_present(cn, c);
        if (k > 0) {
            int pick = choice(u[8], k);
            for (int c = 0; c < C; c++)
                if (conn_present(cn, c) && pick-- == 0) {
                    for (int j = 0; j < 4; j++) cn[(size_t)c * 4 + j] = NAN;
                    break;
                }
        }
    }
    /* attributes */
    for (int r = 0; r < N; r++) {
        if (!node_present(nd, r) || nd[(size_t)r * 5] < (double)I) continue;
        double *n = nd + (size_t)r * 5;
        const uint32_t *w = u + 16 + 6 * (size_t)r;
        const float *zz = z + 4 + 2 * (size_t)r;
        if (bern(w[0], m->bias_mutate_rate)) n[1] += (double)m->bias_mutate_power * (double)zz[0];
        else if (bern(w[0], (double)m->bias_mutate_rate + (double)m->bias_replace_rate))
            n[1] = (double)m->bias_init_mean + (double)m->bias_init_std * (double)zz[0];
        if (bern(w[1], m->response_mutate_rate)) n[2] += (double)m->response_mutate_power * (double)zz[1];
        else if (bern(w[1], (double)m->response_mutate_rate + (double)m->response_replace_rate))
            n[2] = (double)m->response_init_mean + (double)m->response_init_std * (double)zz[1];
        if (m->n_activation_options > 0 && bern(w[2], m->activation_replace_rate))
            n[4] = m->activation_options[choice(w[3], m->n_activation_options)];
        if (m->n_aggregation_options > 0 && bern(w[4], m->aggregation_replace_rate))
            n[3] = m->aggregation_options[choice(w[5], m->n_aggregation_options)];
    }
    for (int c = 0; c < C; c++) {
        if (!conn_present(cn, c)) continue;
        double *x = cn + (size_t)c * 4;
        const uint32_t *w = u + 16 + 6 * (size_t)N + 2 * (size_t)c;
        const double zz = z[4 + 2 * (size_t)N + c];
        if (bern(w[0], m->weight_mutate_rate)) x[3] += (double)m->weight_mutate_power * zz;
        else if (bern(w[0], (double)m->weight_mutate_rate + (double)m->weight_replace_rate))
            x[3] = (double)m->weight_init_mean + (double)m->weight_init_std * zz;
        if (bern(w[1], m->enabled_mutate_rate)) x[2] = (x[2] != 0.0) ? 0.0 : 1.0;
    }
}

int oracle_mutate(const float *nodes, const float *conns, int P, int I, int O, int N, int C,
                  const orc_mutation_t *m, const uint32_t *u, const float *z, const int *new_keys,
                  double *nodes_out, double *conns_out)
{
    const size_t W = 16 + 6 * (size_t)N + 2 * (size_t)C, Z = 4 + 2 * (size_t)N + (size_t)C;
    for (int g = 0; g < P; g++) {
        double *nd = nodes_out + (size_t)g * N * 5, *cn = conns_out + (size_t)g * C * 4;
        for (size_t i = 0; i < (size_t)N * 5; i++) nd[i] = nodes[(size_t)g * N * 5 + i];
        for (size_t i = 0; i < (size_t)C * 4; i++) cn[i] = conns[(size_t)g * C * 4 + i];
        mutate_one(nd, cn, I, O, N, C, m, u + g * W, z + g * Z, new_keys[g]);
    }
    return 0;
}

int oracle_crossover(const float *nodes, const float *conns, int N, int C, const int *parents, int K,
                     const uint32_t *u, float *nodes_out, float *conns_out)
{
    for (int k = 0; k < K; k++) {
        const float *n1 = nodes + (size_t)parents[2 * k] * N * 5, *n2 = nodes + (size_t)parents[2 * k + 1] * N * 5;
        const float *c1 = conns + (size_t)parents[2 * k] * C * 4, *c2 = conns + (size_t)parents[2 * k + 1] * C * 4;
        float *no = nodes_out + (size_t)k * N * 5, *co = conns_out + (size_t)k * C * 4;
        const uint32_t *w = u + (size_t)k * (N + C);
        memcpy(no, n1, sizeof(float) * (size_t)N * 5);
        memcpy(co, c1, sizeof(float) * (size_t)C * 4);
        for (int r = 0; r < N; r++) {
            if (!is_key(n1[(size_t)r * 5]) || w[r] < 0x80000000u) continue;
            for (int q = 0; q < N; q++) {
                if (isnan(n2[(size_t)q * 5]) || n2[(size_t)q * 5] != n1[(size_t)r * 5]) continue;
                memcpy(no + (size_t)r * 5 + 1, n2 + (size_t)q * 5 + 1, sizeof(float) * 4);
                break;
            }
        }
        for (int c = 0; c < C; c++) {
            const float *x = c1 + (size_t)c * 4;
            if (!is_key(x[0]) || !is_key(x[1]) || isnan(x[2]) || w[N + c] < 0x80000000u) continue;
            for (int q = 0; q < C; q++) {
                const float *y = c2 + (size_t)q * 4;
                if (isnan(y[0]) || isnan(y[1]) || isnan(y[2]) || y[0] != x[0] || y[1] != x[1]) continue;
                co[(size_t)c * 4 + 2] = y[2];
                co[(size_t)c * 4 + 3] = y[3];
                break;
            }
        }
    }
    return 0;
}

/*
 * HyperNEAT substrate evaluation (Section 4.3 extensions: the CPPN's
 * thresholded weights define a layered substrate network).  The paper gives
 * no substrate rule; this oracle fixes: layer 0 holds the R = res^2 inputs of
 * one input vector, and layer l+1 node t = act(sum_s W_l[s][t] v_l[s]) with
 * W_l the weight block l of the CPPN query (weights[genome][l][s][t]); no
 * bias; act = hidden_act for the inner layers and output_act for the last.
 * Plain loops in double.
 */
int oracle_substrate_forward(const float *weights, int P, int R, int L, const float *inputs, int B,
                             int hidden_act, int output_act, double *out)
{
    double *cur = malloc(sizeof(double) * (size_t)R), *nxt = malloc(sizeof(double) * (size_t)R);
    for (int g = 0; g < P; g++)
        for (int b = 0; b < B; b++) {
            const float *x = inputs + ((size_t)g * B + b) * R;
            for (int s = 0; s < R; s++) cur[s] = x[s];
            for (int l = 0; l + 1 < L; l++) {
                const float *Wl = weights + ((size_t)g * (L - 1) + l) * (size_t)R * R;
                const int act = (l + 2 == L) ? output_act : hidden_act;
                for (int t = 0; t < R; t++) {
                    double acc = 0.0;
                    for (int s = 0; s < R; s++) acc += (double)Wl[(size_t)s * R + t] * cur[s];
                    nxt[t] = act_fn(act, acc);
                }
                double *tmp = cur; cur = nxt; nxt = tmp;
            }
            for (int t = 0; t < R; t++) out[((size_t)g * B + b) * R + t] = cur[t];
        }
    free(cur); free(nxt);
    return 0;
}
