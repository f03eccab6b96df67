"""Pins for the genome-distance oracle (speciation, Algorithm 1; the
compatibility_disjoint / compatibility_homologous weights and threshold of
the hyperparameter list).

Each pin comes from outside the oracle: a hand-worked example, closed forms
of one-gene edits, the linear structure in the two coefficients, identity
and symmetry, and invariance under padding and row order.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome, stack

GOLD = os.path.join(os.path.dirname(__file__), "golden", "distance_handworked.json")


def _pop(seed, pop=24, nmax=20, cmax=48):
    return W.random_dag_population(seed, pop, 3, 2, nmax, cmax, hidden=lambda r: int(r.integers(0, 12)),
                                   edges=lambda r, n: int(r.integers(n // 2, 2 * n)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.3)


def _gold_genomes(g):
    a = genome(g["a"]["nodes"], g["a"]["conns"], 6, 6)
    b = genome(g["b"]["nodes"], g["b"]["conns"], 6, 6)
    return a, b


def test_handworked_example():
    g = json.load(open(GOLD))
    (na, ca), (nb, cb) = _gold_genomes(g)
    d, sa, sb = oracle.distance(na, ca, nb, cb, g["c_disjoint"], g["c_homologous"])
    assert sa[0] == 0 and sb[0] == 0
    assert d[0, 0] == g["distance"]                     # exact: dyadic values throughout
    # the two halves separately: nodes only (connections removed) and connections only
    d_nodes, _, _ = oracle.distance(na, np.full_like(ca, np.nan), nb, np.full_like(cb, np.nan),
                                    g["c_disjoint"], g["c_homologous"])
    assert d_nodes[0, 0] == g["d_nodes"]
    assert oracle.speciate(d, g["threshold"])[0] == 0


def test_identity_and_symmetry():
    p = _pop(1)
    d, sa, _ = oracle.distance(p.nodes, p.conns, p.nodes, p.conns, 1.0, 0.5)
    assert (sa == 0).all()
    assert (np.diag(d) == 0).all()
    np.testing.assert_allclose(d, d.T, rtol=0, atol=1e-12)
    assert (d[~np.eye(24, dtype=bool)] > 0).all()


def test_linear_in_the_coefficients():
    p, q = _pop(2), _pop(3)
    d11, _, _ = oracle.distance(p.nodes, p.conns, q.nodes, q.conns, 1.0, 1.0)
    d_disj, _, _ = oracle.distance(p.nodes, p.conns, q.nodes, q.conns, 1.0, 0.0)
    d_hom, _, _ = oracle.distance(p.nodes, p.conns, q.nodes, q.conns, 0.0, 1.0)
    np.testing.assert_allclose(d11, d_disj + d_hom, rtol=0, atol=1e-12)
    d_mix, _, _ = oracle.distance(p.nodes, p.conns, q.nodes, q.conns, 2.5, 0.75)
    np.testing.assert_allclose(d_mix, 2.5 * d_disj + 0.75 * d_hom, rtol=0, atol=1e-11)
    # disjoint part: integer counts over integer denominators
    n_a = (~np.isnan(p.nodes[:, :, 0])).sum(1)
    assert (d_disj >= 0).all() and (d_disj <= 4.0).all()
    assert n_a.min() > 0


@pytest.mark.parametrize("cd,ch", [(1.0, 0.5), (2.0, 3.0)])
def test_one_gene_edits_closed_forms(cd, ch):
    base_nodes = [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.3, 1, 0, 1), (5, -0.7, 1.5, 2, 4)]
    base_conns = [(0, 2, 1, 0.8), (1, 5, 1, -1.2), (5, 2, 1, 0.4), (0, 5, 0, 2.0)]
    n, m = len(base_nodes), len(base_conns)
    A = genome(base_nodes, base_conns, 8, 8)

    def dist(nodes, conns):
        B = genome(nodes, conns, 8, 8)
        d, _, _ = oracle.distance(*A, *B, cd, ch)
        return d[0, 0]
    f = lambda v: float(np.float32(v))  # noqa: E731
    # a weight moved by delta: c_h |delta| / m
    conns = list(base_conns)
    conns[2] = (5, 2, 1, 0.4 - 0.9)
    assert abs(dist(base_nodes, conns) - ch * abs(f(-0.5) - f(0.4)) / m) < 1e-12
    # an enabled flag flipped: c_h / m; any non-zero flag counts as enabled
    conns = list(base_conns)
    conns[3] = (0, 5, 1, 2.0)
    assert abs(dist(base_nodes, conns) - ch / m) < 1e-12
    conns[3] = (0, 5, 0, 2.0)
    conns[0] = (0, 2, 2.0, 0.8)
    assert dist(base_nodes, conns) == 0.0
    # a bias, a response, an activation and an aggregation changed on one node
    nodes = list(base_nodes)
    nodes[3] = (5, -0.2, 1.0, 3, 6)
    want = ch * (abs(f(-0.2) - f(-0.7)) + abs(f(1.0) - f(1.5)) + 1 + 1) / n
    assert abs(dist(nodes, base_conns) - want) < 1e-12
    # one node added (unconnected): c_d / (n + 1); one connection added: c_d / (m + 1)
    assert abs(dist(base_nodes + [(9, 0, 1, 0, 1)], base_conns) - cd / (n + 1)) < 1e-12
    assert abs(dist(base_nodes, base_conns + [(1, 2, 1, 0.1)]) - cd / (m + 1)) < 1e-12
    # a node removed: c_d / n (the larger genome is the one compared against)
    assert abs(dist(base_nodes[:3], base_conns) - cd / n) < 1e-12
    # the same pair reversed is a different gene: two disjoint connections
    conns = list(base_conns)
    conns[0] = (2, 0, 1, 0.8)
    assert abs(dist(base_nodes, conns) - 2 * cd / m) < 1e-12


def test_empty_and_disjoint_genomes():
    empty = genome([None, None], [None], 2, 1)
    one = genome([(0, 0.5, 1, 0, 1), (3, 0.1, 1, 0, 1)], [(0, 3, 1, 1.0)], 2, 1)
    other = genome([(4, 0.5, 1, 0, 1), (7, 0.1, 1, 0, 1)], [(4, 7, 1, 1.0)], 2, 1)
    nodes, conns = stack([empty, one, other])
    d, _, _ = oracle.distance(nodes, conns, nodes, conns, 1.5, 0.5)
    assert d[0, 0] == 0.0
    assert d[0, 1] == 1.5 * 2 / 2 + 1.5 * 1 / 1        # every gene of the other genome is disjoint
    assert d[1, 2] == 1.5 * 4 / 2 + 1.5 * 2 / 1        # no shared key


def test_padding_and_row_order_invariance():
    p = _pop(4)
    rng = np.random.default_rng(5)
    d, _, _ = oracle.distance(p.nodes, p.conns, p.nodes[:7], p.conns[:7], 1.0, 0.5)
    nodes = np.full((24, 30, 5), np.nan, np.float32)
    conns = np.full((24, 60, 4), np.nan, np.float32)
    for g in range(24):
        nodes[g, rng.permutation(30)[:20]] = p.nodes[g]
        conns[g, rng.permutation(60)[:48]] = p.conns[g]
    d2, _, _ = oracle.distance(nodes, conns, nodes[:7], conns[:7], 1.0, 0.5)
    np.testing.assert_allclose(d2, d, rtol=0, atol=1e-12)


def test_invalid_genomes_give_nan():
    ok = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    dupkey = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1), (1, 0.3, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    dupconn = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), (0, 1, 0, 0.1)], 3, 2)
    badkey = genome([(0, 0, 1, 0, 0), (1.5, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    nodes, conns = stack([ok, dupkey, dupconn, badkey])
    d, sa, _ = oracle.distance(nodes, conns, nodes, conns, 1.0, 0.5)
    assert list(sa) == [0, 2, 16, 4]
    assert d[0, 0] == 0.0
    assert np.isnan(d[1:, :]).all() and np.isnan(d[:, 1:]).all()


def test_speciate_rule():
    d = np.array([[0.5, 0.2, 3.0], [4.0, 5.0, 3.5], [1.0, 1.0, np.nan], [np.nan, np.nan, 0.1]])
    np.testing.assert_array_equal(oracle.speciate(d, 3.5), [1, -1, 0, 2])
