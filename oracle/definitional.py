"""Sort-free definitional evaluator of one NEAT network, in double.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It is the node-value
rule of Section 3.3 written as a memoized recursion over predecessors:

    value(k) = x_j                                   if k is input key j
    value(k) = act_k(bias_k + response_k *
                     agg_k([w_c * value(src_c) for enabled conns c into k,
                            in ascending connection-row order]))

with no topological sort at all, so it checks the oracle's ordering and list
building independently.  Pure Python: tiny genomes only.  It assumes a valid,
acyclic genome (no status handling) and uses the same readings as the C
oracle (activation/aggregation ids, empty aggregate = 0, edges into inputs and
dangling edges ignored).
"""
from __future__ import annotations

import math


def _act(a: int, z: float) -> float:
    if a == 0:
        return z
    if a == 1:
        return math.tanh(z)
    if a == 2:
        return 1.0 / (1.0 + math.exp(-z))
    if a == 3:
        return max(z, 0.0)
    if a == 4:
        return math.sin(z)
    if a == 5:
        return math.exp(-(z * z))
    if a == 6:
        return abs(z)
    raise ValueError(a)


def evaluate(nodes, conns, num_inputs: int, num_outputs: int, x) -> list[float]:
    """Outputs of one genome (node rows, conn rows as nested sequences)."""
    rows = {}
    for r, nd in enumerate(nodes):
        if not math.isnan(float(nd[0])):
            rows[int(nd[0])] = [float(v) for v in nd]
    incoming = {k: [] for k in rows}
    for c in conns:
        ki, ko, e, w = (float(v) for v in c)
        if math.isnan(ki) or math.isnan(ko) or math.isnan(e) or e == 0.0:
            continue
        ki, ko = int(ki), int(ko)
        if ki not in rows or ko not in rows or ko < num_inputs:
            continue
        incoming[ko].append((ki, w))
    memo: dict[int, float] = {}

    def value(k: int) -> float:
        if k < num_inputs:
            return float(x[k])
        if k in memo:
            return memo[k]
        terms = [w * value(s) for s, w in incoming[k]]
        _key, bias, resp, agg, act = rows[k]
        agg = int(agg)
        if not terms:
            a = 0.0
        elif agg == 0:
            a = 0.0
            for t in terms:
                a = a + t
        elif agg == 1:
            a = 1.0
            for t in terms:
                a = a * t
        elif agg == 2:
            a = terms[0]
            for t in terms[1:]:
                a = max(a, t)
        else:
            a = 0.0
            for t in terms:
                a = a + t
            a = a / len(terms)
        memo[k] = _act(int(act), bias + resp * a)
        return memo[k]

    return [value(num_inputs + j) for j in range(num_outputs)]
