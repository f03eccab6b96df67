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


class MutationConfig(ctypes.Structure):
    """Operator hyperparameters (the appendix's list; see neat_oracle.c for
    how each is used)."""
    _fields_ = [(n, ctypes.c_float) for n in (
        "node_add", "node_delete", "conn_add", "conn_delete",
        "bias_init_mean", "bias_init_std", "bias_mutate_power", "bias_mutate_rate", "bias_replace_rate",
        "response_init_mean", "response_init_std", "response_mutate_power", "response_mutate_rate",
        "response_replace_rate",
        "weight_init_mean", "weight_init_std", "weight_mutate_power", "weight_mutate_rate", "weight_replace_rate",
        "activation_replace_rate", "aggregation_replace_rate", "enabled_mutate_rate")] + [
        ("activation_default", ctypes.c_int), ("aggregation_default", ctypes.c_int),
        ("n_activation_options", ctypes.c_int), ("n_aggregation_options", ctypes.c_int),
        ("activation_options", ctypes.c_int * 8), ("aggregation_options", ctypes.c_int * 4),
        ("feedforward", ctypes.c_int)]


def mutation_config(**kw) -> MutationConfig:
    """All rates 0 and defaults (tanh, sum, response 1) unless given;
    activation_options / aggregation_options as lists."""
    m = MutationConfig()
    m.response_init_mean = 1.0
    m.activation_default, m.aggregation_default = 1, 0
    m.feedforward = 1
    acts = kw.pop("activation_options", [1])
    aggs = kw.pop("aggregation_options", [0])
    m.n_activation_options, m.n_aggregation_options = len(acts), len(aggs)
    for i, a in enumerate(acts):
        m.activation_options[i] = a
    for i, a in enumerate(aggs):
        m.aggregation_options[i] = a
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def mutation_words(max_nodes: int, max_conns: int) -> tuple[int, int]:
    """(uint32 words, float normals) per genome."""
    return 16 + 6 * max_nodes + 2 * max_conns, 4 + 2 * max_nodes + max_conns


def mutate(nodes, conns, num_inputs: int, num_outputs: int, cfg: MutationConfig, words, normals, new_keys):
    """Mutated copies (double) of P genomes; words uint32 [P][W], normals
    f32 [P][Z], new_keys int32 [P]."""
    nodes, conns = _genome_arrays(nodes, conns)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    W, Z = mutation_words(N, C)
    words = np.ascontiguousarray(words, dtype=np.uint32).reshape(P, W)
    normals = np.ascontiguousarray(normals, dtype=np.float32).reshape(P, Z)
    new_keys = np.ascontiguousarray(new_keys, dtype=np.int32).reshape(P)
    no = np.empty((P, N, 5), np.float64)
    co = np.empty((P, C, 4), np.float64)
    L = lib()
    L.oracle_mutate.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 5 + [ctypes.POINTER(MutationConfig)] + \
        [ctypes.c_void_p] * 5
    L.oracle_mutate(_ptr(nodes), _ptr(conns), P, num_inputs, num_outputs, N, C, ctypes.byref(cfg), _ptr(words),
                    _ptr(normals), _ptr(new_keys), _ptr(no), _ptr(co))
    return no, co


def crossover(nodes, conns, parents, words):
    """Children (float32) of parent pairs int32 [K][2] (first = fitter);
    words uint32 [K][Nmax + Cmax]."""
    nodes, conns = _genome_arrays(nodes, conns)
    N, C = nodes.shape[1], conns.shape[1]
    parents = np.ascontiguousarray(parents, dtype=np.int32).reshape(-1, 2)
    K = parents.shape[0]
    words = np.ascontiguousarray(words, dtype=np.uint32).reshape(K, N + C)
    no = np.empty((K, N, 5), np.float32)
    co = np.empty((K, C, 4), np.float32)
    L = lib()
    L.oracle_crossover.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p, ctypes.c_int] + \
        [ctypes.c_void_p] * 3
    L.oracle_crossover(_ptr(nodes), _ptr(conns), N, C, _ptr(parents), K, _ptr(words), _ptr(no), _ptr(co))
    return no, co


def substrate_forward(weights, inputs, hidden_act: int = 1, output_act: int = 1):
    """HyperNEAT substrate outputs (double [P][B][R]) from CPPN weight blocks
    f32 [P][L-1][R][R] (source-major) and inputs f32 [P][B][R]."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    x = np.ascontiguousarray(inputs, dtype=np.float32)
    P, Lm1, R = w.shape[0], w.shape[1], w.shape[2]
    assert w.shape == (P, Lm1, R, R) and x.shape[0] == P and x.shape[2] == R
    B = x.shape[1]
    out = np.empty((P, B, R), np.float64)
    L = lib()
    L.oracle_substrate_forward.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p]
    L.oracle_substrate_forward(_ptr(w), P, R, Lm1 + 1, _ptr(x), B, hidden_act, output_act, _ptr(out))
    return out
