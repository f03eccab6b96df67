"""Seeded synthetic inputs for population-wide NEAT genome evaluation.

This module only *draws* inputs: genome tensors in the paper's NaN-padded
encoding (Section 3.1, "Tensorized Encodings") and observation batches.  It
holds none of the evaluation arithmetic (no topological sort, no forward pass,
no activation or aggregation function).  Both the CUDA path and the oracle are
fed from here; neither imports the other.

Genome encoding (Section 3.1):
  nodes f32[P][Nmax][5]  row = (key, bias, response, aggregation id, activation id)
  conns f32[P][Cmax][4]  row = (in key, out key, enabled, weight)
Absent rows are all-NaN.  Input nodes carry keys 0..I-1, output nodes keys
I..I+O-1 (the genome interface's ``input_idx``/``output_idx``, Appendix
"Interfaces", Listing 2), hidden nodes keys from I+O upward.

Categorical ids are stored as floats (Section 3.1 gives tanh = 1, sigmoid = 2;
the rest of the table is this library's reading):
  activation: 0 identity, 1 tanh, 2 sigmoid, 3 relu, 4 sin, 5 gauss, 6 abs
  aggregation: 0 sum, 1 product, 2 max, 3 mean

Workload recipes follow the experiment settings of Appendix "Experiment
Detail" (weights and biases N(0,1), response 1, tanh, sum) widened to the five
evaluation shapes this library is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Sequence

import numpy as np

ACT_IDENTITY, ACT_TANH, ACT_SIGMOID, ACT_RELU, ACT_SIN, ACT_GAUSS, ACT_ABS = range(7)
AGG_SUM, AGG_PRODUCT, AGG_MAX, AGG_MEAN = range(4)
ALL_ACTS = tuple(range(7))
ALL_AGGS = tuple(range(4))

NODE_COLS = 5
CONN_COLS = 4


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    """PCG64 generator for (seed, stream...) — independent substreams."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


@dataclass
class Population:
    """A population in the padded encoding plus its shape parameters."""
    nodes: np.ndarray          # f32 [P][Nmax][5]
    conns: np.ndarray          # f32 [P][Cmax][4]
    num_inputs: int
    num_outputs: int

    @property
    def pop(self) -> int:
        return self.nodes.shape[0]

    @property
    def max_nodes(self) -> int:
        return self.nodes.shape[1]

    @property
    def max_conns(self) -> int:
        return self.conns.shape[1]

    def subset(self, idx) -> "Population":
        idx = np.asarray(idx)
        return Population(np.ascontiguousarray(self.nodes[idx]),
                          np.ascontiguousarray(self.conns[idx]),
                          self.num_inputs, self.num_outputs)


def empty_population(pop: int, max_nodes: int, max_conns: int,
                     num_inputs: int, num_outputs: int) -> Population:
    nodes = np.full((pop, max_nodes, NODE_COLS), np.nan, dtype=np.float32)
    conns = np.full((pop, max_conns, CONN_COLS), np.nan, dtype=np.float32)
    return Population(nodes, conns, num_inputs, num_outputs)


def _sample_pairs(rng: np.random.Generator, n_in: int, n_non_input: int,
                  n_edges: int) -> np.ndarray:
    """Draw ``n_edges`` distinct (src, dst) pairs of a random DAG.

    Non-input nodes are indexed by a rank 0..m-1 (all inputs rank below every
    non-input).  A pair is any src of lower rank than its non-input dst.  Pairs
    are drawn uniformly without replacement by index into the concatenation of
    per-dst source lists.  Returns int64 [n_edges, 2] of (src, dst) where a
    value < n_in is input number v and v >= n_in is non-input rank v - n_in.
    """
    m = n_non_input
    counts = n_in + np.arange(m, dtype=np.int64)          # sources of rank r
    total = int(counts.sum())
    n_edges = min(n_edges, total)
    if n_edges <= 0:
        return np.zeros((0, 2), dtype=np.int64)
    cum = np.concatenate([[0], np.cumsum(counts)])
    if n_edges * 3 > total:
        picks = rng.choice(total, size=n_edges, replace=False)
    else:
        picks = np.zeros(0, dtype=np.int64)
        while picks.size < n_edges:
            extra = rng.integers(0, total, size=2 * (n_edges - picks.size) + 8)
            picks = np.unique(np.concatenate([picks, extra]))
        picks = rng.permutation(picks)[:n_edges]
    dst_rank = np.searchsorted(cum, picks, side="right") - 1
    s = picks - cum[dst_rank]
    src = np.where(s < n_in, s, n_in + (s - n_in))            # same numbering
    dst = n_in + dst_rank
    return np.stack([src, dst], axis=1)


def random_dag_population(seed: int, pop: int, num_inputs: int, num_outputs: int,
                          max_nodes: int, max_conns: int,
                          hidden: Callable[[np.random.Generator], int],
                          edges: Callable[[np.random.Generator, int], int],
                          acts: Sequence[int] = (ACT_TANH,),
                          aggs: Sequence[int] = (AGG_SUM,),
                          p_disabled: float = 0.1,
                          response: Callable[[np.random.Generator, int], np.ndarray] | None = None,
                          stream: int = 0) -> Population:
    """Random feedforward genomes in the canonical row layout.

    Per genome: H = hidden(rng) hidden nodes (clamped to capacity); the O + H
    non-input nodes get a random rank; E = edges(rng, n) connections are drawn
    without duplicates among pairs (lower rank -> higher rank, dst non-input);
    each connection is disabled with probability ``p_disabled``; connection
    rows are shuffled.  Weights and biases N(0,1); response 1 unless a sampler
    is given; activation/aggregation ids uniform over ``acts``/``aggs``.
    """
    I, O = num_inputs, num_outputs
    P = empty_population(pop, max_nodes, max_conns, I, O)
    acts = np.asarray(acts, dtype=np.float32)
    aggs = np.asarray(aggs, dtype=np.float32)
    for g in range(pop):
        rng = rng_for(seed, stream, g)
        H = int(min(max(hidden(rng), 0), max_nodes - I - O))
        n = I + O + H
        m = O + H
        keys = np.arange(n, dtype=np.float32)                 # row r holds key r
        nodes = P.nodes[g]
        nodes[:n, 0] = keys
        nodes[:n, 1] = rng.standard_normal(n).astype(np.float32)
        nodes[:n, 2] = (response(rng, n).astype(np.float32) if response is not None
                        else np.float32(1.0))
        nodes[:n, 3] = aggs[rng.integers(0, aggs.size, size=n)]
        nodes[:n, 4] = acts[rng.integers(0, acts.size, size=n)]
        # non-input rank -> node row: a random permutation of rows I..n-1
        rank_row = I + rng.permutation(m)
        E = int(min(edges(rng, n), max_conns))
        pairs = _sample_pairs(rng, I, m, E)
        E = pairs.shape[0]

        def to_row(v):
            return np.where(v < I, v, rank_row[np.clip(v - I, 0, m - 1)])

        src_row = to_row(pairs[:, 0])
        dst_row = to_row(pairs[:, 1])
        conns = P.conns[g]
        conns[:E, 0] = keys[src_row]
        conns[:E, 1] = keys[dst_row]
        conns[:E, 2] = (rng.random(E) >= p_disabled).astype(np.float32)
        conns[:E, 3] = rng.standard_normal(E).astype(np.float32)
    return P


# --------------------------------------------------------------------------
# The five evaluation shapes
# --------------------------------------------------------------------------

def xor_population(seed: int = 0, pop: int = 100, mutations: int = 5) -> Population:
    """XOR-shaped genomes grown by NEAT-style structural mutations.

    2 inputs + 1 bias input (key 2, fed 1.0), 1 output (key 3), start fully
    connected (3 conns), then ``mutations`` mutations, each add-node or
    add-conn with probability 1/2 (Section 3.2's row insertions):
      add-node: pick a random enabled conn a->b, disable it, add node c with
                conns a->c and c->b (weights N(0,1)), bias N(0,1);
      add-conn: pick uniformly among absent pairs a->b (b not an input) that
                keep the graph acyclic, using a maintained linear extension;
                no-op when none is left.
    Max 10 nodes / 20 conns, sigmoid, sum, response 1.
    """
    I, O, NMAX, CMAX = 3, 1, 10, 20
    P = empty_population(pop, NMAX, CMAX, I, O)
    for g in range(pop):
        rng = rng_for(seed, 1, g)
        node_keys = [0, 1, 2, 3]
        bias = {k: float(rng.standard_normal()) for k in node_keys}
        conns = [[k, 3, 1.0, float(rng.standard_normal())] for k in (0, 1, 2)]
        linear = [0, 1, 2, 3]              # inputs first; every edge goes forward in it
        next_key = 4
        for _ in range(mutations):
            if rng.random() < 0.5:
                enabled = [i for i, c in enumerate(conns) if c[2] != 0.0]
                if not enabled or len(node_keys) >= NMAX or len(conns) + 2 > CMAX:
                    continue
                ci = enabled[int(rng.integers(len(enabled)))]
                a, b = conns[ci][0], conns[ci][1]
                conns[ci][2] = 0.0
                c = next_key
                next_key += 1
                node_keys.append(c)
                bias[c] = float(rng.standard_normal())
                linear.insert(linear.index(b), c)
                conns.append([a, c, 1.0, float(rng.standard_normal())])
                conns.append([c, b, 1.0, float(rng.standard_normal())])
            else:
                if len(conns) >= CMAX:
                    continue
                present = {(c[0], c[1]) for c in conns}
                cand = [(a, b) for ia, a in enumerate(linear) for b in linear[ia + 1:]
                        if b >= I and (a, b) not in present]
                if not cand:
                    continue
                a, b = cand[int(rng.integers(len(cand)))]
                conns.append([a, b, 1.0, float(rng.standard_normal())])
        nd = P.nodes[g]
        for r, k in enumerate(node_keys):
            nd[r] = (k, bias[k], 1.0, AGG_SUM, ACT_SIGMOID)
        P.conns[g, :len(conns)] = np.asarray(conns, dtype=np.float32)
    return P


def xor_inputs(pop: int = 100) -> np.ndarray:
    """The 4 points of {0,1}^2 with the constant bias input: f32 [P][4][3]."""
    pts = np.array([[0, 0, 1], [0, 1, 1], [1, 0, 1], [1, 1, 1]], dtype=np.float32)
    return np.ascontiguousarray(np.broadcast_to(pts, (pop, 4, 3)))


def ant_population(seed: int = 0, pop: int = 10000) -> Population:
    """Ant-shaped control genomes: 27 inputs, 8 outputs, max 50 nodes / 200 conns.

    Hidden count uniform on 0..15: the stated 0..20 cannot fit, since
    27 + 8 + 20 > 50 rows, so it is clamped to capacity.  100..200 conns drawn
    (capped by the available acyclic pairs), 10% disabled, tanh, sum.
    """
    return random_dag_population(
        seed, pop, 27, 8, 50, 200,
        hidden=lambda r: int(r.integers(0, 16)),
        edges=lambda r, n: int(r.integers(100, 201)),
        acts=(ACT_TANH,), aggs=(AGG_SUM,), p_disabled=0.1, stream=2)


BATCHED_MAX_NODES = (16, 64, 256, 1024)


def batched_populations(seed: int = 0, pop: int = 2048,
                        max_nodes: Sequence[int] = BATCHED_MAX_NODES,
                        num_inputs: int = 8, num_outputs: int = 4) -> list[Population]:
    """Uneven populations: one per Nmax, Cmax = 4 Nmax, n ~ U{I+O..Nmax} nodes,
    E ~ U{3n..4n} conns, 10% disabled, all 7 activations and 4 aggregations
    drawn uniformly."""
    out = []
    for j, nmax in enumerate(max_nodes):
        I, O = num_inputs, num_outputs
        out.append(random_dag_population(
            seed, pop, I, O, nmax, 4 * nmax,
            hidden=lambda r, nmax=nmax: int(r.integers(0, nmax - I - O + 1)),
            edges=lambda r, n: int(r.integers(3 * n, 4 * n + 1)),
            acts=ALL_ACTS, aggs=ALL_AGGS, p_disabled=0.1, stream=10 + j))
    return out


def cppn_population(seed: int = 0, pop: int = 1000) -> Population:
    """CPPN genomes: inputs (x_s, y_s, x_d, y_d, 1), 1 output, max 32 nodes /
    96 conns, hidden U{0..26}, E ~ U{5..96}, sin/gauss/tanh/identity, sum."""
    return random_dag_population(
        seed, pop, 5, 1, 32, 96,
        hidden=lambda r: int(r.integers(0, 27)),
        edges=lambda r, n: int(r.integers(5, 97)),
        acts=(ACT_SIN, ACT_GAUSS, ACT_TANH, ACT_IDENTITY), aggs=(AGG_SUM,),
        p_disabled=0.1, stream=3)


def normal_inputs(seed: int, shape, stream: int = 0) -> np.ndarray:
    """N(0,1) float32 observations of the given shape (host memory)."""
    return rng_for(seed, 100 + stream).standard_normal(shape, dtype=np.float32)


def serving_requests(seed: int = 0, n_requests: int = 2000, rate_hz: float = 200.0,
                     pop_range=(64, 4096), nodes_range=(8, 512), batch_range=(1, 256),
                     steps: int = 100) -> list[dict]:
    """Poisson request stream: arrival times and log-uniform shapes.

    Per request: P, Nmax, B log-uniform in their ranges, Cmax = 4 Nmax,
    I = min(27, Nmax // 2), O = min(8, max(1, Nmax // 4)).  Genomes are drawn
    lazily with ``request_population``.
    """
    rng = rng_for(seed, 5)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))

    def logu(lo, hi):
        return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))

    reqs = []
    for i in range(n_requests):
        nmax = logu(*nodes_range)
        reqs.append(dict(id=i, arrival_s=float(t[i]), pop=logu(*pop_range),
                         max_nodes=nmax, max_conns=4 * nmax,
                         num_inputs=min(27, nmax // 2),
                         num_outputs=min(8, max(1, nmax // 4)),
                         batch=logu(*batch_range), steps=steps, seed=seed * 100003 + i))
    return reqs


def request_population(req: dict) -> Population:
    """Genomes of one serving request: as the Ant shape, at the request's size."""
    I, O, nmax = req["num_inputs"], req["num_outputs"], req["max_nodes"]
    cmax = req["max_conns"]
    return random_dag_population(
        req["seed"], req["pop"], I, O, nmax, cmax,
        hidden=lambda r: int(r.integers(0, max(nmax - I - O, 0) + 1)),
        edges=lambda r, n: int(r.integers(2 * n, 4 * n + 1)),
        acts=(ACT_TANH,), aggs=(AGG_SUM,), p_disabled=0.1, stream=6)


def random_dag_population_vec(seed: int, pop: int, num_inputs: int, num_outputs: int,
                              max_nodes: int, max_conns: int, hidden_max: int,
                              edge_factors=(2, 4), p_disabled: float = 0.1,
                              stream: int = 8) -> Population:
    """Random feedforward genomes drawn for the whole population at once
    (numpy array operations, no per-genome loop), for request streams that
    need many large populations quickly.  Same recipe as
    ``random_dag_population`` with tanh / sum and response 1: H ~ U{0..hidden_max}
    hidden nodes, a random rank for each non-input node, E ~ U{f0 n .. f1 n}
    connection draws (capped by Cmax and the acyclic pairs) among (lower
    rank -> higher rank, dst non-input) pairs, repeated pairs dropped (so a
    genome keeps slightly fewer connections than it drew), 10% disabled,
    weights and biases N(0,1); connection rows in pair order."""
    I, O, N, C = num_inputs, num_outputs, max_nodes, max_conns
    rng = rng_for(seed, stream)
    P = empty_population(pop, N, C, I, O)
    H = rng.integers(0, max(min(hidden_max, N - I - O), 0) + 1, size=pop)
    n = I + O + H                                   # present nodes (rows 0..n-1, key = row)
    m = O + H                                       # non-input nodes
    rows = np.arange(N)
    present = rows[None, :] < n[:, None]
    P.nodes[:, :, 0] = np.where(present, rows[None, :].astype(np.float32), np.nan)
    P.nodes[:, :, 1] = np.where(present, rng.standard_normal((pop, N), dtype=np.float32), np.nan)
    P.nodes[:, :, 2] = np.where(present, np.float32(1.0), np.nan)
    P.nodes[:, :, 3] = np.where(present, np.float32(AGG_SUM), np.nan)
    P.nodes[:, :, 4] = np.where(present, np.float32(ACT_TANH), np.nan)
    # non-input rank r -> row: a random order of the rows I..n-1
    key = rng.random((pop, N))
    key[:, :I] = np.inf
    key[~present] = np.inf
    rank_row = np.argsort(key, axis=1)              # first m entries: the non-input rows in rank order
    # pairs: index t over the concatenation of the per-rank source lists
    cum = np.concatenate([[0], np.cumsum(I + np.arange(N, dtype=np.int64))])   # cum[r] = sources of ranks < r
    total = cum[m]                                  # acyclic pairs per genome
    E = np.minimum(rng.integers(edge_factors[0] * n, edge_factors[1] * n + 1), np.minimum(total, C))
    # E draws with replacement per genome; repeated pairs are dropped (one
    # sort), so a genome keeps slightly fewer than E when draws collide
    g_of = np.repeat(np.arange(pop), E)
    t = (rng.random(g_of.size) * total[g_of]).astype(np.int64)
    span = int(total.max()) + 1
    code = g_of * span + t
    code.sort()
    first = np.ones(code.size, dtype=bool)
    first[1:] = code[1:] != code[:-1]
    code = code[first]
    g_u = code // span
    t_u = code - g_u * span
    start = np.searchsorted(g_u, np.arange(pop))
    k = np.arange(g_u.size) - start[g_u]
    dst_rank = np.searchsorted(cum, t_u, side="right") - 1
    s = t_u - cum[dst_rank]
    src_row = np.where(s < I, s, rank_row[g_u, np.maximum(s - I, 0)])
    dst_row = rank_row[g_u, dst_rank]
    P.conns[g_u, k, 0] = src_row
    P.conns[g_u, k, 1] = dst_row
    P.conns[g_u, k, 2] = (rng.random(g_u.size) >= p_disabled).astype(np.float32)
    P.conns[g_u, k, 3] = rng.standard_normal(g_u.size, dtype=np.float32)
    return P


def request_population_fast(req: dict) -> Population:
    """Genomes of one serving request drawn with ``random_dag_population_vec``:
    the Ant recipe at the request's size (hidden nodes up to capacity,
    2n..4n connections)."""
    I, O, nmax = req["num_inputs"], req["num_outputs"], req["max_nodes"]
    return random_dag_population_vec(req["seed"], req["pop"], I, O, nmax, req["max_conns"],
                                     hidden_max=max(nmax - I - O, 0), edge_factors=(2, 4))


def random_recurrent_population(seed: int, pop: int, num_inputs: int, num_outputs: int,
                                max_nodes: int, max_conns: int,
                                hidden: Callable[[np.random.Generator], int],
                                edges: Callable[[np.random.Generator, int], int],
                                acts: Sequence[int] = (ACT_TANH,), aggs: Sequence[int] = (AGG_SUM,),
                                p_disabled: float = 0.1, stream: int = 20) -> Population:
    """Recurrent genomes: connections drawn without duplicates among all
    (source any node, destination any non-input node) pairs, so cycles and
    self-loops occur; otherwise as random_dag_population."""
    I, O = num_inputs, num_outputs
    P = empty_population(pop, max_nodes, max_conns, I, O)
    acts = np.asarray(acts, dtype=np.float32)
    aggs = np.asarray(aggs, dtype=np.float32)
    for g in range(pop):
        rng = rng_for(seed, stream, g)
        H = int(min(max(hidden(rng), 0), max_nodes - I - O))
        n = I + O + H
        m = O + H
        nodes = P.nodes[g]
        nodes[:n, 0] = np.arange(n, dtype=np.float32)
        nodes[:n, 1] = rng.standard_normal(n).astype(np.float32)
        nodes[:n, 2] = 1.0
        nodes[:n, 3] = aggs[rng.integers(0, aggs.size, size=n)]
        nodes[:n, 4] = acts[rng.integers(0, acts.size, size=n)]
        total = n * m
        E = int(min(edges(rng, n), max_conns, total))
        picks = rng.choice(total, size=E, replace=False)
        src = picks // m
        dst = I + picks % m
        conns = P.conns[g]
        conns[:E, 0] = src
        conns[:E, 1] = dst
        conns[:E, 2] = (rng.random(E) >= p_disabled).astype(np.float32)
        conns[:E, 3] = rng.standard_normal(E).astype(np.float32)
    return P


def ant_recurrent_population(seed: int = 0, pop: int = 10000) -> Population:
    """Ant-shaped recurrent genomes (27 in, 8 out, max 50 nodes / 200 conns,
    tanh, sum), connections in any direction."""
    return random_recurrent_population(seed, pop, 27, 8, 50, 200,
                                       hidden=lambda r: int(r.integers(0, 16)),
                                       edges=lambda r, n: int(r.integers(100, 201)), stream=21)


def related_population(seed: int, pop: int, num_inputs: int, num_outputs: int, max_nodes: int, max_conns: int,
                       ancestor_hidden: int, ancestor_edges: int, new_nodes: int, new_conns: int,
                       key_pool: int, p_perturb: float = 0.8, sigma: float = 0.5, p_flip: float = 0.05,
                       p_drop: float = 0.1, p_act: float = 0.05, stream: int = 30,
                       acyclic: bool = False) -> Population:
    """A population in mid-evolution, for genome distances: mutated copies of
    one random ancestor DAG.  Each member perturbs weights and biases
    (N(0, sigma), probability p_perturb), flips enabled flags (p_flip), drops
    connections (p_drop), changes activations (p_act), and adds up to
    `new_nodes` hidden nodes whose keys come from a shared pool of `key_pool`
    keys (so added genes are often homologous across members) and up to
    `new_conns` connections between present nodes.  Rows are shuffled.
    acyclic: every key gets one place in a global order (the ancestor's
    topological order, pool keys at random places) and added connections
    only run forward in it, so every member stays a DAG (disabled
    connections included)."""
    I, O = num_inputs, num_outputs
    anc = random_dag_population(seed, 1, I, O, max_nodes, max_conns, hidden=lambda r: ancestor_hidden,
                                edges=lambda r, n: ancestor_edges, acts=ALL_ACTS, aggs=ALL_AGGS,
                                p_disabled=0.1, stream=stream)
    an = anc.nodes[0][~np.isnan(anc.nodes[0, :, 0])]
    ac = anc.conns[0][~np.isnan(anc.conns[0, :, 0])]
    base_key = int(an[:, 0].max()) + 1
    place = {}
    if acyclic:
        # the ancestor's topological order over all its connections (Kahn)
        indeg = {int(k): 0 for k in an[:, 0]}
        for a_, b_ in ac[:, :2].astype(np.int64):
            indeg[int(b_)] += 1
        ready = sorted(k for k, v in indeg.items() if v == 0)
        while ready:
            k = ready.pop(0)
            place[k] = float(len(place))
            for a_, b_ in ac[:, :2].astype(np.int64):
                if int(a_) == k:
                    indeg[int(b_)] -= 1
                    if indeg[int(b_)] == 0:
                        ready.append(int(b_))
        assert len(place) == len(indeg)
        prng = rng_for(seed, stream + 2)
        for j in range(key_pool):
            place[base_key + j] = float(prng.uniform(-0.5, len(indeg) - 0.5))
        for k in range(num_inputs):
            place[k] = -1.0 - k
    P = empty_population(pop, max_nodes, max_conns, I, O)
    for g in range(pop):
        rng = rng_for(seed, stream + 1, g)
        nodes = an.copy()
        pert = rng.random(len(nodes)) < p_perturb
        nodes[pert, 1] += (sigma * rng.standard_normal(int(pert.sum()))).astype(np.float32)
        newact = rng.random(len(nodes)) < p_act
        nodes[newact, 4] = rng.integers(0, 7, size=int(newact.sum()))
        conns = ac[rng.random(len(ac)) >= p_drop].copy()
        pert = rng.random(len(conns)) < p_perturb
        conns[pert, 3] += (sigma * rng.standard_normal(int(pert.sum()))).astype(np.float32)
        flip = rng.random(len(conns)) < p_flip
        conns[flip, 2] = 1.0 - conns[flip, 2]
        k = int(min(rng.integers(0, new_nodes + 1), max_nodes - len(nodes), key_pool))
        if k > 0:
            keys = base_key + rng.choice(key_pool, size=k, replace=False)
            extra = np.zeros((k, NODE_COLS), np.float32)
            extra[:, 0] = keys
            extra[:, 1] = rng.standard_normal(k)
            extra[:, 2] = 1.0
            extra[:, 3] = rng.integers(0, 4, size=k)
            extra[:, 4] = rng.integers(0, 7, size=k)
            nodes = np.concatenate([nodes, extra])
        present = nodes[:, 0].astype(np.int64)
        targets = present[present >= I]
        have = {(int(a), int(b)) for a, b in conns[:, :2]}
        add = []
        want = int(min(rng.integers(0, new_conns + 1), max_conns - len(conns)))
        for _ in range(4 * want):
            if len(add) >= want:
                break
            pair = (int(rng.choice(present)), int(rng.choice(targets)))
            if acyclic and not place[pair[0]] < place[pair[1]]:
                continue
            if pair not in have:
                have.add(pair)
                add.append((pair[0], pair[1], 1.0, float(rng.standard_normal())))
        if add:
            conns = np.concatenate([conns, np.asarray(add, np.float32)])
        P.nodes[g, rng.permutation(max_nodes)[:len(nodes)]] = nodes
        P.conns[g, rng.permutation(max_conns)[:len(conns)]] = conns
    return P


def ant_related_population(seed: int = 0, pop: int = 10000, acyclic: bool = False) -> Population:
    """Ant-shaped population in mid-evolution (27 in, 8 out, max 50 nodes /
    200 conns): an ancestor with 8 hidden nodes and 120 connections, members
    adding up to 7 nodes from a pool of 20 keys and up to 30 connections."""
    return related_population(seed, pop, 27, 8, 50, 200, ancestor_hidden=8, ancestor_edges=120, new_nodes=7,
                              new_conns=30, key_pool=20, acyclic=acyclic)


def substrate_weights(seed: int, pop: int, res: int = 16, layers: int = 3, scale: float = 0.25,
                      threshold: float = 0.2) -> np.ndarray:
    """Weight blocks shaped like a thresholded CPPN query (f32
    [pop][layers-1][res^2][res^2], source-major): N(0, scale) values with
    |w| < threshold set to 0 (about 58% zeros at the defaults)."""
    rng = rng_for(seed, 40)
    R = res * res
    w = (scale * rng.standard_normal((pop, layers - 1, R, R))).astype(np.float32)
    w[np.abs(w) < threshold] = 0.0
    return w
