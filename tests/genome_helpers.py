"""Small helpers for building hand-made genomes in the padded encoding."""
import numpy as np

NAN = float("nan")


def genome(node_rows, conn_rows, max_nodes=None, max_conns=None):
    """One genome as (nodes f32[1][Nmax][5], conns f32[1][Cmax][4]).

    node_rows: (key, bias, response, agg, act) or None for an all-NaN row.
    conn_rows: (in, out, enabled, weight) or None.
    """
    N = max_nodes or len(node_rows)
    C = max_conns or max(len(conn_rows), 1)
    nodes = np.full((1, N, 5), np.nan, np.float32)
    conns = np.full((1, C, 4), np.nan, np.float32)
    for r, row in enumerate(node_rows):
        if row is not None:
            nodes[0, r] = row
    for r, row in enumerate(conn_rows):
        if row is not None:
            conns[0, r] = row
    return nodes, conns


def stack(genomes):
    """Stack single genomes (same Nmax/Cmax) into a population."""
    return (np.concatenate([g[0] for g in genomes]), np.concatenate([g[1] for g in genomes]))
