"""Pins for the mutation and crossover oracle (tensorized node, connection
and attribute modification, Section 3.2; the operator hyperparameters of
the appendix).

Every random draw is an input (uint32 words, float normals), so each pin
sets the words that decide its case and checks the result against what the
operation must produce: closed forms, function preservation of the node
split, acyclicity of feedforward connection addition, identity at rate 0,
the exact rate and choice boundaries.
"""
import numpy as np

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome

NAN = np.nan
TOP = 0xFFFFFFFF


def _words(P, N, C, fill=TOP):
    W_, Z = oracle.mutation_words(N, C)
    return np.full((P, W_), fill, np.uint32), np.zeros((P, Z), np.float32)


def _same(a, b):
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(np.nan_to_num(np.asarray(a, np.float64)), np.nan_to_num(np.asarray(b, np.float64)))


def _dag(seed, pop=40):
    return W.random_dag_population(seed, pop, 3, 2, 24, 60, hidden=lambda r: int(r.integers(0, 12)),
                                   edges=lambda r, n: int(r.integers(n // 2, 2 * n)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.2)


def test_zero_rates_leave_genomes_unchanged():
    p = _dag(1)
    u, z = _words(40, 24, 60, fill=0)                       # the most permissive words
    rng = np.random.default_rng(2)
    z[:] = rng.standard_normal(z.shape)
    no, co = oracle.mutate(p.nodes, p.conns, 3, 2, oracle.mutation_config(), u, z, np.full(40, 999))
    _same(no, p.nodes)
    _same(co, p.conns)


def test_node_split_preserves_the_function():
    # 0 -> 1 with weight 0.7; the split node is identity with bias 0, response 1
    nodes, conns = genome([(0, 0, 1, 0, 0), None, (1, 0.3, 1.5, 0, 1)], [(0, 1, 1, 0.7), None, None, None], 4, 4)
    cfg = oracle.mutation_config(node_add=1.0, activation_default=0, bias_init_mean=0.0, response_init_mean=1.0)
    u, z = _words(1, 4, 4)
    u[0, 0] = 0                                             # node addition happens
    u[0, 1] = 0                                             # the only enabled connection
    no, co = oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [7])
    _same(no[0, 1], [7, 0, 1, 0, 0])                       # first free node row
    _same(co[0], np.array([[0, 1, 0, 0.7], [0, 7, 1, 1.0], [7, 1, 1, 0.7], [NAN] * 4], np.float32))
    x = np.linspace(-2, 2, 9, dtype=np.float32).reshape(1, 9, 1)
    before = oracle.forward(nodes, conns, 1, 1, x)
    after = oracle.forward(no.astype(np.float32), co.astype(np.float32), 1, 1, x)
    np.testing.assert_array_equal(after, before)


def test_node_addition_needs_room_and_a_new_key():
    nodes, conns = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 1)], [(0, 1, 1, 0.7), None], 2, 2)
    cfg = oracle.mutation_config(node_add=1.0)
    u, z = _words(1, 2, 2)
    u[0, 0] = 0
    no, co = oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [5])           # no free node row
    _same(no, nodes)
    _same(co, conns)
    nodes3, conns3 = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 1), None], [(0, 1, 1, 0.7), None, None], 3, 3)
    no, co = oracle.mutate(nodes3, conns3, 1, 1, cfg, *_set(u, 3, 3), [1])  # key 1 already present
    _same(no, nodes3)


def _set(u_small, N, C):
    u, z = _words(1, N, C)
    u[0, :9] = u_small[0, :9]
    return u, z


def test_node_deletion_removes_touching_connections():
    rows = [(0, 0, 1, 0, 0), (1, 0, 1, 0, 1), (4, 0.1, 1, 0, 1), (5, 0.2, 1, 0, 1)]
    cs = [(0, 4, 1, 1.0), (4, 1, 1, 1.0), (0, 5, 1, 1.0), (5, 1, 0, 1.0), (4, 5, 1, 2.0)]
    nodes, conns = genome(rows, cs, 4, 5)
    cfg = oracle.mutation_config(node_delete=1.0)
    for word, key in ((0, 4), (TOP, 5)):                   # first and last hidden node
        u, z = _words(1, 4, 5)
        u[0, 2], u[0, 3] = 0, word
        no, co = oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [9])
        assert not (no[0, :, 0] == key).any() and (~np.isnan(no[0, :, 0])).sum() == 3
        kept = [c for c in cs if key not in c[:2]]
        assert (~np.isnan(co[0, :, 0])).sum() == len(kept)
        assert not np.isin(co[0, :, :2], [key]).any()


def test_connection_addition_rules():
    rows = [(0, 0, 1, 0, 0), (1, 0, 1, 0, 1), (2, 0, 1, 0, 1), (3, 0, 1, 0, 1)]
    cs = [(0, 2, 1, 1.0), (2, 3, 1, 1.0), (3, 1, 1, 1.0), (0, 1, 0, 0.5), None]
    nodes, conns = genome(rows, cs, 4, 5)
    cfg = oracle.mutation_config(conn_add=1.0, weight_init_mean=0.25, weight_init_std=2.0)

    def add(src_idx, tgt_idx, feedforward=1):
        cfg.feedforward = feedforward
        u, z = _words(1, 4, 5)
        u[0, 4] = 0
        # choice(u, k) = floor(u k / 2^32): pick index i of k with u = ceil(i 2^32 / k)
        u[0, 5] = -(-(src_idx << 32) // 4)                  # sources: the 4 present nodes in row order
        u[0, 6] = -(-(tgt_idx << 32) // 3)                  # targets: keys 1, 2, 3 in row order
        z[0, 0] = -1.5
        return oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [9])
    no, co = add(0, 0)                                      # 0 -> 1 exists (disabled): enabled
    _same(co[0, 3], [0, 1, 1, 0.5])
    no, co = add(2, 1)                                      # 2 -> 2: a self-loop, rejected
    _same(co, conns)
    no, co = add(3, 1)                                      # 3 -> 2 closes 2 -> 3 -> 2: rejected
    _same(co, conns)
    no, co = add(3, 1, feedforward=0)                       # allowed for recurrent networks
    _same(co[0, 4], [3, 2, 1, 0.25 + 2.0 * -1.5])
    no, co = add(1, 1)                                      # 1 -> 2 reaches back through 2 -> 3 -> 1: rejected
    _same(co, conns)
    no, co = add(0, 2)                                      # 0 -> 3: new, acyclic
    _same(co[0, 4], [0, 3, 1, 0.25 + 2.0 * -1.5])


def test_feedforward_connection_addition_keeps_populations_acyclic():
    p = _dag(3, pop=150)
    cfg = oracle.mutation_config(conn_add=1.0, node_add=0.5, conn_delete=0.2, node_delete=0.2)
    rng = np.random.default_rng(4)
    W_, Z = oracle.mutation_words(24, 60)
    for _ in range(3):
        u = rng.integers(0, 2**32, size=(150, W_), dtype=np.uint64).astype(np.uint32)
        z = rng.standard_normal((150, Z)).astype(np.float32)
        no, co = oracle.mutate(p.nodes, p.conns, 3, 2, cfg, u, z, 100 + np.arange(150))
        p = W.Population(no.astype(np.float32), co.astype(np.float32), 3, 2)
        st = oracle.transform(p.nodes, p.conns, 3, 2)["status"]
        assert (st & 1 == 0).all()                           # no cycle
        assert (st & 0xFF == 0).all()


def test_connection_deletion_and_choice_boundaries():
    nodes, conns = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 1)], [None, (0, 1, 1, 0.1), (1, 1, 0, 0.2), None, (0, 0, 1, 0.3)],
                          2, 5)
    cfg = oracle.mutation_config(conn_delete=1.0)
    for word, gone in ((0, 1), ((1 << 32) // 3, 1), ((1 << 32) // 3 + 1, 2), (TOP, 4)):
        u, z = _words(1, 2, 5)
        u[0, 7], u[0, 8] = 0, word
        _, co = oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [9])
        assert np.isnan(co[0, gone]).all()
        assert (~np.isnan(co[0, :, 0])).sum() == 2


def test_attribute_mutation_closed_forms_and_rate_boundaries():
    p = _dag(5, pop=30)
    N, C = 24, 60
    rng = np.random.default_rng(6)
    W_, Z = oracle.mutation_words(N, C)
    z = rng.standard_normal((30, Z)).astype(np.float32)
    node_present = ~np.isnan(p.nodes[:, :, 0])
    non_input = node_present & (p.nodes[:, :, 0] >= 3)
    conn_present = ~np.isnan(p.conns[:, :, 0])
    zb = z[:, 4:4 + 2 * N:2]
    zr = z[:, 5:4 + 2 * N:2]
    zw = z[:, 4 + 2 * N:]
    # perturbation with rate 1: attr + power z (response too); inputs untouched
    cfg = oracle.mutation_config(bias_mutate_rate=1.0, bias_mutate_power=0.5, response_mutate_rate=1.0,
                                 response_mutate_power=0.25, weight_mutate_rate=1.0, weight_mutate_power=0.75)
    u = np.zeros((30, W_), np.uint32)
    u[:, :9] = TOP
    no, co = oracle.mutate(p.nodes, p.conns, 3, 2, cfg, u, z, np.zeros(30))
    np.testing.assert_allclose(no[:, :, 1][non_input], (p.nodes[:, :, 1] + 0.5 * zb.astype(np.float64))[non_input],
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(no[:, :, 2][non_input], (p.nodes[:, :, 2] + 0.25 * zr.astype(np.float64))[non_input],
                               rtol=0, atol=1e-12)
    _same(no[:, :, 1][node_present & ~non_input], p.nodes[:, :, 1][node_present & ~non_input])
    np.testing.assert_allclose(co[:, :, 3][conn_present], (p.conns[:, :, 3] + 0.75 * zw.astype(np.float64))[conn_present], rtol=0,
                               atol=1e-12)
    # replacement: init_mean + init_std z
    cfg = oracle.mutation_config(bias_replace_rate=1.0, bias_init_mean=-1.0, bias_init_std=3.0)
    no, _ = oracle.mutate(p.nodes, p.conns, 3, 2, cfg, u, z, np.zeros(30))
    np.testing.assert_allclose(no[:, :, 1][non_input], (-1.0 + 3.0 * zb.astype(np.float64))[non_input], rtol=0,
                               atol=1e-12)
    # rate boundaries: mutate 0.5, replace 0.5 -> word < 2^31 perturbs, 2^31 <= word replaces
    cfg = oracle.mutation_config(weight_mutate_rate=0.5, weight_replace_rate=0.5, weight_mutate_power=1.0,
                                 weight_init_mean=10.0)
    for word, want in (((1 << 31) - 1, p.conns[:, :, 3] + zw.astype(np.float64)), (1 << 31, 10.0 + 0 * zw)):
        u2 = u.copy()
        u2[:, 16 + 6 * N::2] = word
        _, co = oracle.mutate(p.nodes, p.conns, 3, 2, cfg, u2, z, np.zeros(30))
        np.testing.assert_allclose(co[:, :, 3][conn_present], want[conn_present], rtol=0, atol=1e-12)
    # categorical replacement picks options[floor(word k / 2^32)]; enabled flips
    cfg = oracle.mutation_config(activation_replace_rate=1.0, activation_options=[1, 2, 4],
                                 aggregation_replace_rate=1.0, aggregation_options=[3, 1], enabled_mutate_rate=1.0)
    for word, act, agg in ((0, 1, 3), (TOP, 4, 1), ((1 << 32) // 3 + 1, 2, 3)):
        u3 = u.copy()
        u3[:, 16 + 3:16 + 6 * N:6] = word
        u3[:, 16 + 5:16 + 6 * N:6] = word
        no, co = oracle.mutate(p.nodes, p.conns, 3, 2, cfg, u3, z, np.zeros(30))
        assert (no[:, :, 4][non_input] == act).all() and (no[:, :, 3][non_input] == agg).all()
        np.testing.assert_array_equal(co[:, :, 2][conn_present], (p.conns[:, :, 2] == 0)[conn_present])


def test_crossover_rules():
    a = genome([(0, 0, 1, 0, 0), (1, 0.5, 1, 0, 1), None, (4, 0.1, 2, 1, 2)], [(0, 1, 1, 0.3), (0, 4, 0, 0.6), None],
               4, 3)
    b = genome([(4, -0.1, 3, 2, 5), (0, 9, 9, 9, 9), (1, 0.7, 1.5, 3, 4), (6, 1, 1, 0, 1)],
               [(0, 4, 1, -0.6), (4, 6, 1, 1.0), (0, 1, 0, 0.9)], 4, 3)
    nodes = np.concatenate([a[0], b[0]])
    conns = np.concatenate([a[1], b[1]])
    K = 3
    words = np.zeros((K, 7), np.uint32)
    words[1] = TOP
    words[2] = TOP
    no, co = oracle.crossover(nodes, conns, [[0, 1], [0, 1], [0, 0]], words)
    _same(no[0], a[0][0])                                 # every word below 2^31: the fitter parent
    _same(co[0], a[1][0])
    want_n = [(0, 9, 9, 9, 9), (1, 0.7, 1.5, 3, 4), (NAN,) * 5, (4, -0.1, 3, 2, 5)]
    _same(no[1], np.array(want_n, np.float32))            # homologous genes from the other parent
    _same(co[1], np.array([(0, 1, 0, 0.9), (0, 4, 1, -0.6), (NAN,) * 4], np.float32))
    _same(no[2], a[0][0])                                  # a genome crossed with itself
    _same(co[2], a[1][0])


def test_dangling_connections_do_not_make_paths():
    # 2 -> 9 -> 3 with key 9 absent: adding 3 -> 2 closes no cycle among present nodes
    rows = [(0, 0, 1, 0, 0), (1, 0, 1, 0, 1), (2, 0, 1, 0, 1), (3, 0, 1, 0, 1)]
    cs = [(2, 9, 1, 1.0), (9, 3, 1, 1.0), None]
    nodes, conns = genome(rows, cs, 4, 3)
    cfg = oracle.mutation_config(conn_add=1.0)
    u, z = _words(1, 4, 3)
    u[0, 4] = 0
    u[0, 5] = -(-(3 << 32) // 4)                            # source key 3
    u[0, 6] = -(-(1 << 32) // 3)                            # target key 2
    _, co = oracle.mutate(nodes, conns, 1, 1, cfg, u, z, [8])
    _same(co[0, 2], [3, 2, 1, 0])
