"""Pins for the recurrent oracle (K synchronous iterations from zero)."""
import numpy as np

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome


def test_dag_reaches_the_feedforward_values_after_depth_iterations():
    pop = W.random_dag_population(4, 60, 3, 2, 20, 60, hidden=lambda r: int(r.integers(0, 12)),
                                  edges=lambda r, n: int(r.integers(n, 3 * n)), acts=W.ALL_ACTS,
                                  aggs=W.ALL_AGGS, p_disabled=0.2)
    x = W.normal_inputs(4, (60, 3, 3))
    ff = oracle.forward(pop.nodes, pop.conns, 3, 2, x)
    levels = oracle.transform(pop.nodes, pop.conns, 3, 2)["n_levels"]
    K = int(levels.max())
    rec, st = oracle.forward_recurrent(pop.nodes, pop.conns, 3, 2, x, K)
    assert (st == 0).all()
    np.testing.assert_array_equal(rec, ff)                 # bit for bit: the same sums in the same order
    # a node at level l is exact after l iterations when its level-0 ancestors are
    # inputs (l + 1 otherwise), so two iterations fewer leave the deepest off
    short, _ = oracle.forward_recurrent(pop.nodes, pop.conns, 3, 2, x, K - 2)
    deepest = levels == K
    assert not np.array_equal(short[deepest], ff[deepest])


def test_linear_self_loop_closed_form():
    # y_k = b + r (w_x x + w_s y_{k-1}), y_0 = 0  ->  y_K = c (1 - a^K) / (1 - a), a = r w_s, c = b + r w_x x
    b, r, wx, ws = np.float32(0.3), np.float32(0.9), np.float32(1.25), np.float32(-0.6)
    nodes, conns = genome([(0, 0, 1, 0, 0), (1, b, r, 0, 0)], [(0, 1, 1, wx), (1, 1, 1, ws)])
    for K in (0, 1, 2, 7, 40):
        x = np.array([[[0.75]]], np.float32)
        y, st = oracle.forward_recurrent(nodes, conns, 1, 1, x, K)
        a = float(r) * float(ws)
        c = float(b) + float(r) * float(wx) * 0.75
        want = c * (1 - a ** K) / (1 - a)
        assert st[0] == 0
        assert abs(y[0, 0, 0] - want) <= 1e-12 * max(1.0, abs(want))


def test_two_node_linear_cycle_matrix_power():
    # h_k = b_h + w_xh x + w_yh y_{k-1};  y_k = b_y + w_hy h_{k-1} + w_yy y_{k-1}
    bh, by, wxh, wyh, why, wyy = 0.1, -0.2, 0.8, -0.5, 1.1, 0.3
    rows = [(0, 0, 1, 0, 0), (1, by, 1, 0, 0), (2, bh, 1, 0, 0)]          # x, y (output), h (hidden)
    conns = [(0, 2, 1, wxh), (1, 2, 1, wyh), (2, 1, 1, why), (1, 1, 1, wyy)]
    nodes, cn = genome(rows, conns)
    f = lambda v: float(np.float32(v))  # noqa: E731
    A = np.array([[0.0, f(wyh)], [f(why), f(wyy)]])                       # state (h, y)
    xv = 0.5
    c = np.array([f(bh) + f(wxh) * xv, f(by)])
    for K in (1, 2, 5, 12):
        y, _ = oracle.forward_recurrent(nodes, cn, 1, 1, np.array([[[xv]]], np.float32), K)
        v = sum(np.linalg.matrix_power(A, j) @ c for j in range(K))
        assert abs(y[0, 0, 0] - v[1]) <= 1e-12


def test_cycles_are_allowed_and_errors_still_reported():
    rows = [(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1), (2, -0.1, 1, 0, 2)]
    cyc = [(0, 2, 1, 1.0), (2, 1, 1, 0.5), (1, 2, 1, -0.7), (2, 2, 1, 0.25)]
    nodes, cn = genome(rows, cyc)
    y, st = oracle.forward_recurrent(nodes, cn, 1, 1, np.ones((1, 2, 1), np.float32), 6)
    assert st[0] == 0 and np.isfinite(y).all()
    bad, cbad = genome(rows + [(2, 0, 1, 0, 1)], cyc)                     # duplicate key
    y, st = oracle.forward_recurrent(bad, cbad, 1, 1, np.ones((1, 1, 1), np.float32), 6)
    assert st[0] == 2 and np.isnan(y).all()


def test_recurrent_node_row_permutation_is_bit_exact():
    pop = W.random_recurrent_population(5, 30, 4, 3, 24, 80, hidden=lambda r: int(r.integers(0, 10)),
                                        edges=lambda r, n: int(r.integers(n, 3 * n)), acts=W.ALL_ACTS,
                                        aggs=(W.AGG_SUM, W.AGG_MEAN, W.AGG_MAX))
    x = W.normal_inputs(5, (30, 2, 4))
    y, st = oracle.forward_recurrent(pop.nodes, pop.conns, 4, 3, x, 5)
    rng = np.random.default_rng(6)
    nodes = np.stack([pop.nodes[g][rng.permutation(24)] for g in range(30)])
    y2, _ = oracle.forward_recurrent(nodes, pop.conns, 4, 3, x, 5)
    np.testing.assert_array_equal(y, y2)
    assert (st == 0).all()
