"""Pins for the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or mathematics fixes:
a hand-worked network with closed-form values, brute force over all
topological orders of tiny DAGs, closed forms (single layer = act(b + r Wx)),
invariants of the padded encoding (Section 3.1/3.2), and hand-built malformed
genomes for the status word.
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest

import oracle
from oracle import definitional
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome

HERE = os.path.dirname(os.path.abspath(__file__))
NAN = float("nan")

CYCLE, DUPKEY, BADKEY, BADENUM, DUPCONN, BADATTR, MISSING_IO = 1, 2, 4, 8, 16, 32, 64
DANGLING, INTO_INPUT = 256, 512


# ---------------------------------------------------------------- XOR golden

def _xor_fixture():
    with open(os.path.join(HERE, "golden", "xor_handworked.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("encoding", ["encoding_bias_in_nodes", "encoding_bias_input"])
def test_xor_handworked(encoding):
    fx = _xor_fixture()
    enc = fx[encoding]
    nodes, conns = genome([tuple(r) for r in enc["nodes"]], [tuple(r) for r in enc["conns"]],
                          max_nodes=10, max_conns=20)
    x = np.asarray(fx["inputs"], np.float32)[None]
    y = oracle.forward(nodes, conns, 3, 1, x)[0, :, 0]
    for got, want in zip(y, fx["expected_y"]):
        assert abs(got - float(want)) <= 1e-15
    # the closed form itself, recomputed independently in 40-digit arithmetic
    mpmath.mp.dps = 40
    s = lambda z: 1 / (1 + mpmath.e ** (-z))  # noqa: E731
    for (x1, x2, _), got in zip(fx["inputs"], y):
        want = s(20 * s(20 * x1 + 20 * x2 - 10) + 20 * s(-20 * x1 - 20 * x2 + 30) - 30)
        assert abs(got - float(want)) <= 1e-15


def test_xor_hidden_values():
    fx = _xor_fixture()
    # a network whose output is the OR unit alone (h1), and one for NAND (h2)
    n1 = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0, 1, 0, 0), (3, -10, 1, 0, 2)],
                [(0, 3, 1, 20), (1, 3, 1, 20)])
    n2 = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0, 1, 0, 0), (3, 30, 1, 0, 2)],
                [(0, 3, 1, -20), (1, 3, 1, -20)])
    x = np.array([[[0, 0, 1]]], np.float32)
    assert abs(oracle.forward(*n1, 3, 1, x)[0, 0, 0] - float(fx["expected_h1_00"])) <= 1e-18
    assert abs(oracle.forward(*n2, 3, 1, x)[0, 0, 0] - float(fx["expected_h2_00"])) <= 1e-15


# ------------------------------------------------- brute force on tiny DAGs

def _tiny_dag(rng, n_in, n_out, n_hidden, p_edge, act_ids, agg_ids):
    """Random small DAG with shuffled node and connection rows."""
    n = n_in + n_out + n_hidden
    keys = list(range(n))
    order = [k for k in keys if k >= n_in]
    rng.shuffle(order)
    rank = {k: -1 for k in range(n_in)}
    rank.update({k: i for i, k in enumerate(order)})
    conns = []
    for a in keys:
        for b in keys:
            if b >= n_in and rank[a] < rank[b] and rng.random() < p_edge:
                e = 0.0 if rng.random() < 0.15 else 1.0
                conns.append((a, b, e, float(np.float32(rng.standard_normal()))))
    rng.shuffle(conns)
    f32 = lambda v: float(np.float32(v))  # noqa: E731  (the genome stores float32)
    rows = [(k, f32(rng.standard_normal()), f32(rng.uniform(0.5, 1.5)),
             int(rng.choice(agg_ids)), int(rng.choice(act_ids))) for k in keys]
    rng.shuffle(rows)
    return rows, conns


def _linear_extensions(nodes_rows, conns_rows):
    """All topological orders (as row-index tuples) of the enabled graph."""
    key_row = {int(r[0]): i for i, r in enumerate(nodes_rows)}
    preds = {i: set() for i in range(len(nodes_rows))}
    for a, b, e, _ in conns_rows:
        if e != 0:
            preds[key_row[b]].add(key_row[a])
    out = []
    n = len(nodes_rows)

    def rec(prefix, placed):
        if len(prefix) == n:
            out.append(tuple(prefix))
            return
        for i in range(n):
            if i not in placed and preds[i] <= placed:
                placed.add(i)
                prefix.append(i)
                rec(prefix, placed)
                prefix.pop()
                placed.remove(i)

    rec([], set())
    return out


def _eval_in_order(nodes_rows, conns_rows, n_in, n_out, order, x):
    """Node rule of Section 3.3 applied in a given order (sum/product/max/mean)."""
    key_row = {int(r[0]): i for i, r in enumerate(nodes_rows)}
    v = {}
    acts = [lambda z: z, math.tanh, lambda z: 1.0 / (1.0 + math.exp(-z)), lambda z: max(z, 0.0),
            math.sin, lambda z: math.exp(-(z * z)), abs]
    for i in order:
        k, b, r, agg, act = nodes_rows[i]
        if k < n_in:
            v[i] = float(x[int(k)])
            continue
        terms = [w * v[key_row[a]] for (a, bb, e, w) in conns_rows if e != 0 and bb == k]
        if not terms:
            s = 0.0
        elif agg == 0 or agg == 3:
            s = 0.0
            for t in terms:
                s = s + t
            if agg == 3:
                s = s / len(terms)
        elif agg == 1:
            s = 1.0
            for t in terms:
                s = s * t
        else:
            s = terms[0]
            for t in terms[1:]:
                s = max(s, t)
        v[i] = acts[int(act)](b + r * s)
    return [v[key_row[n_in + j]] for j in range(n_out)]


def _longest_path_levels(nodes_rows, conns_rows):
    key_row = {int(r[0]): i for i, r in enumerate(nodes_rows)}
    preds = {i: [] for i in range(len(nodes_rows))}
    for a, b, e, _ in conns_rows:
        if e != 0:
            preds[key_row[b]].append(key_row[a])
    memo = {}

    def lev(i):
        if i not in memo:
            memo[i] = 0 if not preds[i] else 1 + max(lev(p) for p in preds[i])
        return memo[i]

    return [lev(i) for i in range(len(nodes_rows))]


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_all_topological_orders(seed):
    rng = np.random.default_rng(1000 + seed)
    n_in, n_out, n_hid = 2, 1 + seed % 2, 2 + seed % 4
    rows, conns = _tiny_dag(rng, n_in, n_out, n_hid, 0.5, list(range(7)), list(range(4)))
    x = rng.standard_normal(n_in).astype(np.float32)
    exts = _linear_extensions(rows, conns)
    assert len(exts) >= 1
    results = {tuple(_eval_in_order(rows, conns, n_in, n_out, o, x)) for o in exts}
    assert len(results) == 1, "every topological order must give bit-identical outputs"
    nodes, cn = genome(rows, conns, max_conns=max(len(conns), 1))
    got = oracle.forward(nodes, cn, n_in, n_out, x[None, None])[0, 0]
    assert tuple(got) == next(iter(results))
    t = oracle.transform(nodes, cn, n_in, n_out)
    assert t["status"][0] == 0
    order = tuple(int(r) for r in t["order"][0][: len(rows)])
    assert order in set(exts)
    # levels are the longest-path depths and the order is sorted by (level, row)
    lev = _longest_path_levels(rows, conns)
    lp = t["level_ptr"][0]
    got_lev = {}
    for L in range(int(t["n_levels"][0])):
        for p in range(lp[L], lp[L + 1]):
            got_lev[int(t["order"][0][p])] = L
    assert [got_lev[i] for i in range(len(rows))] == lev
    assert list(order) == sorted(range(len(rows)), key=lambda i: (lev[i], i))


@pytest.mark.parametrize("seed", range(8))
def test_definitional_evaluator_agrees(seed):
    """The C oracle equals the sort-free recursive evaluator bit for bit."""
    pop = W.random_dag_population(seed, 30, 3, 2, 14, 40,
                                  hidden=lambda r: int(r.integers(0, 10)),
                                  edges=lambda r, n: int(r.integers(n, 3 * n)),
                                  acts=W.ALL_ACTS, aggs=W.ALL_AGGS, p_disabled=0.2,
                                  response=lambda r, n: r.uniform(0.5, 1.5, n))
    x = W.normal_inputs(seed, (30, 3, 3))
    y = oracle.forward(pop.nodes, pop.conns, 3, 2, x)
    for g in range(30):
        for b in range(3):
            d = definitional.evaluate(pop.nodes[g], pop.conns[g], 3, 2, x[g, b])
            assert list(y[g, b]) == d


# ------------------------------------------------------------- closed forms

ACT_REF = {0: lambda z: z, 1: np.tanh, 2: lambda z: 1 / (1 + np.exp(-z)),
           3: lambda z: np.maximum(z, 0), 4: np.sin, 5: lambda z: np.exp(-z * z), 6: np.abs}


@pytest.mark.parametrize("act", range(7))
def test_single_layer_closed_form(act):
    """Outputs reading only inputs: y = act(b + r * (W x)) (numpy matmul)."""
    rng = np.random.default_rng(act)
    I, O = 6, 4
    Wm = rng.standard_normal((O, I)).astype(np.float32)
    b = rng.standard_normal(O).astype(np.float32)
    r = rng.uniform(0.5, 1.5, O).astype(np.float32)
    rows = [(k, 0, 1, 0, 0) for k in range(I)] + [(I + j, b[j], r[j], 0, act) for j in range(O)]
    conns = [(i, I + j, 1, Wm[j, i]) for j in range(O) for i in range(I)]
    nodes, cn = genome(rows, conns)
    x = rng.standard_normal((1, 5, I)).astype(np.float32)
    got = oracle.forward(nodes, cn, I, O, x)[0]
    z = b.astype(np.float64) + r.astype(np.float64) * (x[0].astype(np.float64) @ Wm.T.astype(np.float64))
    np.testing.assert_allclose(got, ACT_REF[act](z), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("agg", range(4))
def test_aggregations_closed_form(agg):
    rng = np.random.default_rng(40 + agg)
    I = 5
    w = rng.standard_normal(I).astype(np.float32)
    rows = [(k, 0, 1, 0, 0) for k in range(I)] + [(I, 0.25, 1.5, agg, 0)]
    conns = [(i, I, 1, w[i]) for i in range(I)]
    nodes, cn = genome(rows, conns)
    x = rng.standard_normal((1, 3, I)).astype(np.float32)
    got = oracle.forward(nodes, cn, I, 1, x)[0, :, 0]
    t = x[0].astype(np.float64) * w.astype(np.float64)
    ref = {0: t.sum(1), 1: t.prod(1), 2: t.max(1), 3: t.mean(1)}[agg]
    np.testing.assert_allclose(got, 0.25 + 1.5 * ref, rtol=1e-14, atol=1e-14)


def test_chain_is_nested_scalar_function():
    # x0 -> h (sin, w=2) -> h2 (gauss, w=-0.5) -> out (tanh, w=3), biases 0.1, 0.2, 0.3
    rows = [(0, 0, 1, 0, 0), (1, 0.3, 1, 0, 1), (2, 0.1, 1, 0, 4), (3, 0.2, 1, 0, 5)]
    conns = [(0, 2, 1, 2.0), (2, 3, 1, -0.5), (3, 1, 1, 3.0)]
    nodes, cn = genome(rows, conns)
    for xv in (-1.3, 0.0, 0.7):
        got = oracle.forward(nodes, cn, 1, 1, np.array([[[xv]]], np.float32))[0, 0, 0]
        xf = float(np.float32(xv))
        want = math.tanh(0.3 + 3.0 * math.exp(-(0.2 + -0.5 * math.sin(
            float(np.float32(0.1)) + 2.0 * xf)) ** 2))
        assert abs(got - want) < 1e-7  # biases are float32-rounded in the genome
        want32 = math.tanh(float(np.float32(0.3)) + 3.0 * math.exp(-(float(np.float32(0.2)) - 0.5 * math.sin(
            float(np.float32(0.1)) + 2.0 * xf)) ** 2))
        assert abs(got - want32) <= 1e-15


def test_empty_incoming_set_gives_act_of_bias():
    rows = [(0, 0, 1, 0, 0)] + [(1 + a, 0.5, 2.0, a, 1) for a in range(4)]
    nodes, cn = genome(rows, [None])
    got = oracle.forward(nodes, cn, 1, 4, np.array([[[3.0]]], np.float32))[0, 0]
    np.testing.assert_array_equal(got, [math.tanh(0.5)] * 4)


# --------------------------------------------------------------- invariants

def _pop_small(seed, n=40, nmax=24, cmax=80):
    return W.random_dag_population(seed, n, 4, 3, nmax, cmax,
                                   hidden=lambda r: int(r.integers(0, 9)),
                                   edges=lambda r, k: int(r.integers(k, 3 * k)),
                                   acts=W.ALL_ACTS, aggs=W.ALL_AGGS, p_disabled=0.2,
                                   response=lambda r, k: r.uniform(0.5, 1.5, k))


def test_padding_rows_and_holes_have_no_effect():
    pop = _pop_small(1)
    x = W.normal_inputs(1, (pop.pop, 4, 4))
    y = oracle.forward(pop.nodes, pop.conns, 4, 3, x)
    rng = np.random.default_rng(5)
    # re-pad into larger tensors with NaN rows inserted at random interior places
    N2, C2 = pop.max_nodes + 9, pop.max_conns + 17
    nodes = np.full((pop.pop, N2, 5), np.nan, np.float32)
    conns = np.full((pop.pop, C2, 4), np.nan, np.float32)
    for g in range(pop.pop):
        nr = np.sort(rng.choice(N2, pop.max_nodes, replace=False))
        cr = np.sort(rng.choice(C2, pop.max_conns, replace=False))
        nodes[g, nr] = pop.nodes[g]
        conns[g, cr] = pop.conns[g]
    y2 = oracle.forward(nodes, conns, 4, 3, x)
    np.testing.assert_array_equal(y, y2)


def test_disabled_connections_have_no_effect():
    pop = _pop_small(2)
    x = W.normal_inputs(2, (pop.pop, 3, 4))
    y = oracle.forward(pop.nodes, pop.conns, 4, 3, x)
    conns = pop.conns.copy()
    dis = conns[:, :, 2] == 0
    rng = np.random.default_rng(3)
    conns[..., 3][dis] = rng.standard_normal(dis.sum()) * 100
    # a disabled edge may even close a cycle
    conns[..., 0][dis], conns[..., 1][dis] = conns[..., 1][dis], conns[..., 0][dis]
    y2 = oracle.forward(pop.nodes, conns, 4, 3, x)
    np.testing.assert_array_equal(y, y2)


def test_node_row_permutation_is_bit_exact():
    pop = _pop_small(3)
    x = W.normal_inputs(3, (pop.pop, 3, 4))
    y = oracle.forward(pop.nodes, pop.conns, 4, 3, x)
    rng = np.random.default_rng(4)
    nodes = np.stack([pop.nodes[g][rng.permutation(pop.max_nodes)] for g in range(pop.pop)])
    np.testing.assert_array_equal(y, oracle.forward(nodes, pop.conns, 4, 3, x))


def test_conn_row_permutation_changes_only_rounding():
    pop = _pop_small(4)
    x = W.normal_inputs(4, (pop.pop, 3, 4))
    y = oracle.forward(pop.nodes, pop.conns, 4, 3, x)
    rng = np.random.default_rng(5)
    conns = np.stack([pop.conns[g][rng.permutation(pop.max_conns)] for g in range(pop.pop)])
    y2 = oracle.forward(pop.nodes, conns, 4, 3, x)
    np.testing.assert_allclose(y, y2, rtol=1e-12, atol=1e-12)


def test_unreachable_hidden_nodes_have_no_effect():
    pop = _pop_small(6)
    x = W.normal_inputs(6, (pop.pop, 2, 4))
    y = oracle.forward(pop.nodes, pop.conns, 4, 3, x)
    nodes = np.concatenate([pop.nodes, np.full((pop.pop, 3, 5), np.nan, np.float32)], 1)
    conns = np.concatenate([pop.conns, np.full((pop.pop, 4, 4), np.nan, np.float32)], 1)
    for g in range(pop.pop):
        k = 1000 + g
        nodes[g, -3] = (k, 0.1, 1, 0, 1)          # fed by an input, feeds nothing
        nodes[g, -2] = (k + 1, 0.2, 1, 1, 4)      # isolated
        nodes[g, -1] = (k + 2, 0.3, 1, 2, 2)      # fed by the first, feeds nothing
        conns[g, -4] = (0, k, 1, 0.5)
        conns[g, -3] = (k, k + 2, 1, 0.7)
    np.testing.assert_array_equal(y, oracle.forward(nodes, conns, 4, 3, x))


def test_only_outputs_by_key_matter():
    """Inputs and outputs are found by key at any row (genome interface)."""
    rows = [(3, 0.5, 1, 0, 1), (1, 9, 9, 3, 6), (0, 9, 9, 2, 5), (2, -0.25, 1, 0, 2)]
    conns = [(0, 2, 1, 1.5), (1, 2, 1, -2.0), (2, 3, 1, 0.75), (1, 3, 1, 0.5)]
    nodes, cn = genome(rows, conns)
    x = np.array([[[0.3, -0.8]]], np.float32)
    got = oracle.forward(nodes, cn, 2, 2, x)[0, 0]
    x0, x1 = float(np.float32(0.3)), float(np.float32(-0.8))
    h2 = 1 / (1 + math.exp(-(-0.25 + (1.5 * x0 + -2.0 * x1))))
    h3 = math.tanh(0.5 + (0.75 * h2 + 0.5 * x1))
    assert got[0] == pytest.approx(h2, abs=1e-15) and got[1] == pytest.approx(h3, abs=1e-15)


# --------------------------------------------------------------- status word

BASE_NODES = [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.1, 1, 0, 1), (3, 0.2, 1, 0, 1)]
BASE_CONNS = [(0, 3, 1, 0.5), (1, 3, 1, -0.5), (3, 2, 1, 1.0)]


def _status(nodes_rows, conns_rows, I=2, O=1):
    nodes, cn = genome(nodes_rows, conns_rows, max_nodes=8, max_conns=8)
    t = oracle.transform(nodes, cn, I, O)
    y = oracle.forward(nodes, cn, I, O, np.zeros((1, 1, I), np.float32))
    return int(t["status"][0]), y[0, 0]


@pytest.mark.parametrize("name,nodes_rows,conns_rows,want", [
    ("valid", BASE_NODES, BASE_CONNS, 0),
    ("cycle", BASE_NODES, BASE_CONNS + [(2, 3, 1, 1.0)], CYCLE),
    ("self_loop", BASE_NODES, BASE_CONNS + [(3, 3, 1, 1.0)], CYCLE),
    ("disabled_cycle_ok", BASE_NODES, BASE_CONNS + [(2, 3, 0, 1.0)], 0),
    ("dup_key", BASE_NODES + [(3, 0, 1, 0, 1)], BASE_CONNS, DUPKEY),
    ("frac_key", BASE_NODES + [(1.5, 0, 1, 0, 1)], BASE_CONNS, BADKEY),
    ("neg_key", BASE_NODES + [(-1, 0, 1, 0, 1)], BASE_CONNS, BADKEY),
    ("big_key", BASE_NODES + [(2 ** 24, 0, 1, 0, 1)], BASE_CONNS, BADKEY),
    ("frac_conn_key", BASE_NODES, BASE_CONNS + [(0.5, 2, 1, 1.0)], BADKEY),
    ("bad_act", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.1, 1, 0, 9), (3, 0.2, 1, 0, 1)], BASE_CONNS, BADENUM),
    ("bad_agg", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.1, 1, 4, 1), (3, 0.2, 1, 0, 1)], BASE_CONNS, BADENUM),
    ("frac_act", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.1, 1, 0, 1.5), (3, 0.2, 1, 0, 1)], BASE_CONNS, BADENUM),
    ("dup_conn", BASE_NODES, BASE_CONNS + [(0, 3, 1, 2.0)], DUPCONN),
    ("dup_conn_disabled", BASE_NODES, BASE_CONNS + [(0, 3, 0, 2.0)], DUPCONN),
    ("nan_weight", BASE_NODES, [(0, 3, 1, NAN)] + BASE_CONNS[1:], BADATTR),
    ("nan_weight_disabled_ok", BASE_NODES, BASE_CONNS + [(0, 2, 0, NAN)], 0),
    ("nan_bias", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, NAN, 1, 0, 1), (3, 0.2, 1, 0, 1)], BASE_CONNS, BADATTR),
    ("nan_response", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (2, 0.1, NAN, 0, 1), (3, 0.2, 1, 0, 1)], BASE_CONNS, BADATTR),
    ("missing_output", BASE_NODES[:2] + BASE_NODES[3:], [(0, 3, 1, 0.5)], MISSING_IO),
    ("missing_input", BASE_NODES[1:], [(1, 3, 1, 0.5), (3, 2, 1, 1.0)], MISSING_IO),
    ("dangling", BASE_NODES, BASE_CONNS + [(7, 2, 1, 1.0)], DANGLING),
    ("dangling_disabled_silent", BASE_NODES, BASE_CONNS + [(7, 2, 0, 1.0)], 0),
    ("into_input", BASE_NODES, BASE_CONNS + [(3, 0, 1, 1.0)], INTO_INPUT),
    # a duplicated key: one row stands for the key in every lookup (the
    # lowest), so the other checks still run and add their bits
    ("dup_key_dangling", BASE_NODES + [(3, 0, 1, 0, 1)], BASE_CONNS + [(3, 7, 1, 1.0)], DUPKEY | DANGLING),
    ("dup_key_valid_edges", BASE_NODES + [(3, 0, 1, 0, 1)], BASE_CONNS + [(2, 3, 0, 1.0)], DUPKEY),
    ("dup_key_cycle", BASE_NODES + [(3, 0, 1, 0, 1)], BASE_CONNS + [(2, 3, 1, 1.0)], DUPKEY | CYCLE),
    ("dup_key_higher_row_first", [(3, 0, 1, 0, 1)] + BASE_NODES, BASE_CONNS + [(2, 3, 1, 1.0)], DUPKEY | CYCLE),
    ("dup_input_key", BASE_NODES + [(0, 0, 1, 0, 0)], BASE_CONNS + [(3, 0, 1, 1.0)], DUPKEY | INTO_INPUT),
])
def test_status_bits(name, nodes_rows, conns_rows, want):
    st, y = _status(nodes_rows, conns_rows)
    assert st == want, name
    if want & 0xFF:
        assert np.isnan(y).all()
    else:
        assert np.isfinite(y).all()


def test_warnings_keep_outputs():
    st0, y0 = _status(BASE_NODES, BASE_CONNS)
    st1, y1 = _status(BASE_NODES, BASE_CONNS + [(7, 2, 1, 1.0), (3, 0, 1, 5.0)])
    assert st1 == DANGLING | INTO_INPUT
    np.testing.assert_array_equal(y0, y1)


def test_input_attributes_are_ignored():
    rows_a = [(0, 5.0, 3.0, 1, 4)] + BASE_NODES[1:]
    _, y0 = _status(BASE_NODES, BASE_CONNS)
    st, y1 = _status(rows_a, BASE_CONNS)
    assert st == 0
    np.testing.assert_array_equal(y0, y1)


# -------------------------------------------------------------------- CPPN

def test_cppn_substrate_coordinates_and_threshold():
    """A CPPN that outputs x_s exposes the grid; one that outputs 0.5 x_d - 0.1
    exposes the |w| < 0.2 threshold (made on float32)."""
    res = 16
    lin = np.linspace(-1, 1, res)
    q = np.array([(0, b, s, d) for b in (0, 1) for s in (0, 5, 17, 255) for d in (0, 3, 100, 120, 255)],
                 np.int32)
    ident = genome([(k, 0, 1, 0, 0) for k in range(5)] + [(5, 0, 1, 0, 0)], [(0, 5, 1, 1.0)])
    raw, w = oracle.cppn_query(*ident, res, 0.2, q)
    np.testing.assert_array_equal(raw, lin[q[:, 2] % res].astype(np.float32).astype(np.float64))
    lin_y = genome([(k, 0, 1, 0, 0) for k in range(5)] + [(5, -0.1, 1, 0, 0)], [(3, 5, 1, 0.5)])
    raw, w = oracle.cppn_query(*lin_y, res, 0.2, q)
    yd = lin[q[:, 3] // res].astype(np.float32).astype(np.float64)
    want_raw = float(np.float32(-0.1)) + 0.5 * yd
    np.testing.assert_allclose(raw, want_raw, rtol=0, atol=1e-16)
    np.testing.assert_array_equal(w, np.where(np.abs(want_raw.astype(np.float32)) < np.float32(0.2), 0.0, want_raw))
    assert (w == 0).any() and (w != 0).any()


# ------------------------------------------------------- generator sanity

def test_generated_workloads_are_valid():
    for pop, I, O in [(W.xor_population(0, 100), 3, 1), (W.ant_population(0, 300), 27, 8),
                      (W.cppn_population(0, 200), 5, 1)] + [(p, 8, 4) for p in W.batched_populations(0, 40)]:
        t = oracle.transform(pop.nodes, pop.conns, I, O)
        assert (t["status"] == 0).all()
        assert (t["n_levels"] >= 2).all()
