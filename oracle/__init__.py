"""FP64 CPU oracle for population-wide NEAT genome evaluation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the library's product path
never does.  It imports nothing from the CUDA package and shares no code with
it.  ``neat_oracle.c`` is the oracle proper (transform + forward + CPPN query,
recurrent forward and genome distance, in double); ``definitional.py`` is a second, sort-free evaluator
used only to check it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "neat_oracle.c")
_LIB = os.path.join(_HERE, "libneat_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.oracle_transform.argtypes = [P, P, i, i, i, i, i] + [P] * 10
        L.oracle_forward.argtypes = [P, P, i, i, i, i, i, P, i, P]
        L.oracle_cppn_query.argtypes = [P, P, i, i, i, i, ctypes.c_float, P, ctypes.c_long, P, P]
        L.oracle_forward_recurrent.argtypes = [P, P, i, i, i, i, i, P, i, i, P, P]
        L.oracle_distance.argtypes = [P, P, i, P, P, i, i, i, ctypes.c_double, ctypes.c_double, P, P, P]
        for f in (L.oracle_transform, L.oracle_forward, L.oracle_cppn_query, L.oracle_forward_recurrent,
                  L.oracle_distance):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _genome_arrays(nodes, conns):
    nodes = np.ascontiguousarray(nodes, dtype=np.float32)
    conns = np.ascontiguousarray(conns, dtype=np.float32)
    assert nodes.ndim == 3 and nodes.shape[2] == 5 and conns.ndim == 3 and conns.shape[2] == 4
    assert nodes.shape[0] == conns.shape[0]
    return nodes, conns


def transform(nodes, conns, num_inputs: int, num_outputs: int) -> dict:
    """Transform P genomes: order (node row per position), level_ptr, n_levels,
    n_nodes, n_edges, in_ptr (by position), in_src (source row), in_conn
    (connection row), in_w (weight), status."""
    nodes, conns = _genome_arrays(nodes, conns)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    out = dict(order=np.empty((P, N), np.int32), level_ptr=np.empty((P, N + 1), np.int32),
               n_levels=np.empty(P, np.int32), n_nodes=np.empty(P, np.int32),
               n_edges=np.empty(P, np.int32), in_ptr=np.empty((P, N + 1), np.int32),
               in_src=np.empty((P, C), np.int32), in_conn=np.empty((P, C), np.int32),
               in_w=np.empty((P, C), np.float64), status=np.empty(P, np.uint32))
    lib().oracle_transform(_ptr(nodes), _ptr(conns), P, num_inputs, num_outputs, N, C,
                           *[_ptr(out[k]) for k in ("order", "level_ptr", "n_levels", "n_nodes",
                                                     "n_edges", "in_ptr", "in_src", "in_conn",
                                                     "in_w", "status")])
    return out


def forward(nodes, conns, num_inputs: int, num_outputs: int, inputs) -> np.ndarray:
    """Outputs (double [P][B][O]) of P genomes on inputs f32 [P][B][I]."""
    nodes, conns = _genome_arrays(nodes, conns)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    inputs = np.ascontiguousarray(inputs, dtype=np.float32)
    assert inputs.shape[0] == P and inputs.shape[2] == num_inputs
    B = inputs.shape[1]
    out = np.empty((P, B, num_outputs), np.float64)
    lib().oracle_forward(_ptr(nodes), _ptr(conns), P, num_inputs, num_outputs, N, C,
                         _ptr(inputs), B, _ptr(out))
    return out


def cppn_query(nodes, conns, res: int, threshold: float, queries) -> tuple[np.ndarray, np.ndarray]:
    """CPPN values and thresholded substrate weights at queries
    int32 [Q][4] = (genome, block, src, dst)."""
    nodes, conns = _genome_arrays(nodes, conns)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    q = np.ascontiguousarray(queries, dtype=np.int32).reshape(-1, 4)
    raw = np.empty(q.shape[0], np.float64)
    w = np.empty(q.shape[0], np.float64)
    lib().oracle_cppn_query(_ptr(nodes), _ptr(conns), P, N, C, res, float(threshold),
                            _ptr(q), q.shape[0], _ptr(raw), _ptr(w))
    return raw, w


def forward_recurrent(nodes, conns, num_inputs: int, num_outputs: int, inputs, iterations: int):
    """Recurrent networks: K synchronous iterations from zero (see
    neat_oracle.c).  Returns (outputs double [P][B][O], status uint32 [P])."""
    nodes, conns = _genome_arrays(nodes, conns)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    inputs = np.ascontiguousarray(inputs, dtype=np.float32)
    assert inputs.shape[0] == P and inputs.shape[2] == num_inputs
    B = inputs.shape[1]
    out = np.empty((P, B, num_outputs), np.float64)
    st = np.empty(P, np.uint32)
    lib().oracle_forward_recurrent(_ptr(nodes), _ptr(conns), P, num_inputs, num_outputs, N, C,
                                   _ptr(inputs), B, iterations, _ptr(out), _ptr(st))
    return out, st


def distance(nodes_a, conns_a, nodes_b, conns_b, c_disjoint: float, c_homologous: float):
    """Genome distances (see neat_oracle.c): double [PA][PB], NaN where either
    genome's homology is undefined; with the status words of both sides."""
    nodes_a, conns_a = _genome_arrays(nodes_a, conns_a)
    nodes_b, conns_b = _genome_arrays(nodes_b, conns_b)
    assert nodes_a.shape[1:] == nodes_b.shape[1:] and conns_a.shape[1:] == conns_b.shape[1:]
    PA, PB, N, C = nodes_a.shape[0], nodes_b.shape[0], nodes_a.shape[1], conns_a.shape[1]
    out = np.empty((PA, PB), np.float64)
    sa, sb = np.empty(PA, np.uint32), np.empty(PB, np.uint32)
    lib().oracle_distance(_ptr(nodes_a), _ptr(conns_a), PA, _ptr(nodes_b), _ptr(conns_b), PB, N, C,
                          float(c_disjoint), float(c_homologous), _ptr(out), _ptr(sa), _ptr(sb))
    return out, sa, sb


def speciate(distances, threshold: float) -> np.ndarray:
    """Species of each genome (Algorithm 1, dividing the population by
    distance): the representative (column) nearest to it among those closer
    than the threshold, the lowest column on ties; -1 when none is.  NaN
    distances never qualify."""
    d = np.asarray(distances, np.float64)
    out = np.full(d.shape[0], -1, np.int32)
    for g in range(d.shape[0]):
        best = None
        for s in range(d.shape[1]):
            if d[g, s] < threshold and (best is None or d[g, s] < d[g, best]):
                best = s
        if best is not None:
            out[g] = best
    return out
