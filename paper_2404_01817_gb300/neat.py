"""Python binding of libneat.so (include/neat.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; PyTorch provides
device memory (``tensor.data_ptr()``) and streams.  Nothing is computed in
Python: if the CUDA library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libneat.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                      f"g.build()\"` (needs nvcc); there is no fallback implementation")

_lib = ctypes.CDLL(LIB_PATH)

NEAT_OK, NEAT_EINVAL, NEAT_ENOMEM, NEAT_ECUDA, NEAT_EBUDGET, NEAT_EAGAIN, NEAT_ETIMEOUT, NEAT_ECANCELLED = \
    0, -1, -2, -3, -4, -5, -6, -7
G_CYCLE, G_DUPKEY, G_BADKEY, G_BADENUM, G_DUPCONN, G_BADATTR, G_MISSING_IO = 1, 2, 4, 8, 16, 32, 64
W_DANGLING, W_INTO_INPUT = 256, 512
G_ERROR_MASK = 0xFF
MAX_NODES, MAX_CONNS = 1024, 8192


class Dims(ctypes.Structure):
    _fields_ = [("num_inputs", ctypes.c_int32), ("num_outputs", ctypes.c_int32),
                ("max_nodes", ctypes.c_int32), ("max_conns", ctypes.c_int32)]


class Launch(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("groups_per_block", ctypes.c_int32), ("pdl", ctypes.c_int32), ("split", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("order_dev", ctypes.c_void_p)]

    def __init__(self, group=8, tile=1, groups_per_block=1, pdl=0, split=1, order=None):
        super().__init__(group, tile, groups_per_block, pdl, split, 0, None if order is None else order.data_ptr())

    def __repr__(self):
        return (f"Launch(group={self.group}, tile={self.tile}, groups_per_block={self.groups_per_block}, "
                f"pdl={self.pdl}, split={self.split})")


_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class PopDesc(ctypes.Structure):
    _fields_ = [("transformed", _P), ("pop", _i32), ("dims", Dims), ("batch", _i32),
                ("inputs", _P), ("in_step_stride", _i64), ("outputs", _P), ("out_step_stride", _i64)]


class Substrate(ctypes.Structure):
    _fields_ = [("resolution", _i32), ("layers", _i32)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_active", _i32), ("reserved", _i32)]


class Request(ctypes.Structure):
    _fields_ = [("nodes_host", _P), ("conns_host", _P), ("pop", _i32), ("dims", Dims), ("batch", _i32),
                ("steps", _i32), ("flags", _i32), ("obs_seed", ctypes.c_uint64), ("outputs_dev", _P),
                ("out_step_stride", _i64)]


REQ_BORROW_HOST = 1


class Result(ctypes.Structure):
    _fields_ = [("status", _i32), ("reserved", _i32), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double), ("genome_forwards", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", _i32), ("cancelled", _i32), ("queued", _i32), ("active", _i32),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("queue_wait_p50_ms", ctypes.c_double), ("queue_wait_p99_ms", ctypes.c_double),
                ("genome_forwards", ctypes.c_uint64), ("genome_forwards_per_s", ctypes.c_double),
                ("ticks", _i64), ("pool_used_bytes", ctypes.c_uint64)]


class Mutation(ctypes.Structure):
    """neat_mutation: the operator hyperparameters (see include/neat.h)."""
    _fields_ = [(n, ctypes.c_float) for n in (
        "node_add", "node_delete", "conn_add", "conn_delete",
        "bias_init_mean", "bias_init_std", "bias_mutate_power", "bias_mutate_rate", "bias_replace_rate",
        "response_init_mean", "response_init_std", "response_mutate_power", "response_mutate_rate",
        "response_replace_rate",
        "weight_init_mean", "weight_init_std", "weight_mutate_power", "weight_mutate_rate", "weight_replace_rate",
        "activation_replace_rate", "aggregation_replace_rate", "enabled_mutate_rate")] + [
        ("activation_default", _i32), ("aggregation_default", _i32),
        ("n_activation_options", _i32), ("n_aggregation_options", _i32),
        ("activation_options", _i32 * 8), ("aggregation_options", _i32 * 4), ("feedforward", _i32)]


def mutation(**kw) -> Mutation:
    """A Mutation with every rate 0, tanh / sum defaults, response 1 and the
    feedforward check on, then the given fields; activation_options and
    aggregation_options as lists."""
    m = Mutation()
    m.response_init_mean = 1.0
    m.activation_default, m.aggregation_default, m.feedforward = 1, 0, 1
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


class LanesInfo(ctypes.Structure):
    _fields_ = [("pop", _i32), ("warps", _i32), ("max_warp_bytes", ctypes.c_uint32),
                ("warp_stride", ctypes.c_uint32), ("unordered", ctypes.c_uint32), ("recurrent", ctypes.c_uint32)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("autotune", _i32), ("size_buckets", _i32), ("block_threads", _i32), ("pdl", _i32)]

_sig = {
    "neat_record_stride": (ctypes.c_size_t, [Dims]),
    "neat_transformed_bytes": (ctypes.c_size_t, [_i32, Dims]),
    "neat_transform": (ctypes.c_int, [_P, _P, _i32, Dims, _P, ctypes.c_size_t, _P, _P]),
    "neat_forward": (ctypes.c_int, [_P, _i32, Dims, _P, _i32, _P, _P]),
    "neat_default_launch": (ctypes.c_int, [_i32, Dims, _i32, ctypes.POINTER(Launch)]),
    "neat_device_error": (ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_uint32)]),
    "neat_schedule": (ctypes.c_int, [_P, _i32, Dims, _P, _P]),
    "neat_transform_recurrent": (ctypes.c_int, [_P, _P, _i32, Dims, _P, ctypes.c_size_t, _P, _P]),
    "neat_forward_recurrent": (ctypes.c_int, [_P, _i32, Dims, _P, _i32, _i32, _P, _P]),
    "neat_forward_recurrent_ex": (ctypes.c_int, [_P, _i32, Dims, _P, _i32, _i32, _P, ctypes.POINTER(Launch), _P]),
    "neat_default_launch_recurrent": (ctypes.c_int, [_i32, Dims, _i32, ctypes.POINTER(Launch)]),
    "neat_gene_stride": (ctypes.c_size_t, [Dims]),
    "neat_distance_prepare": (ctypes.c_int, [_P, _P, _i32, Dims, _P, ctypes.c_size_t, _P, _P]),
    "neat_distance": (ctypes.c_int, [_P, _i32, _P, _i32, Dims, ctypes.c_float, ctypes.c_float, _P, ctypes.c_int64,
                                     _P]),
    "neat_speciate": (ctypes.c_int, [_P, _i32, _i32, ctypes.c_int64, ctypes.c_float, _P, _P]),
    "neat_mutation_sizes": (ctypes.c_int, [Dims, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "neat_mutate": (ctypes.c_int, [_P, _P, _i32, Dims, ctypes.POINTER(Mutation), _P, _P, _P, _P]),
    "neat_crossover": (ctypes.c_int, [_P, _P, _i32, Dims, _P, _i32, _P, _P, _P, _P]),
    "neat_fill_words": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, _P, _i64, _P]),
    "neat_substrate_forward": (ctypes.c_int, [_P, _i32, Substrate, _P, _i32, _i32, _i32, _P, _P]),
    "neat_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "neat_forward_ex": (ctypes.c_int, [_P, _i32, Dims, _P, _i32, _P, ctypes.POINTER(Launch), _P]),
    "neat_forward_steps": (ctypes.c_int, [_P, _i32, Dims, _P, _i64, _i32, _P, _i64, _i32,
                                          ctypes.POINTER(Launch), ctypes.POINTER(_P), _P]),
    "neat_steps_cache_destroy": (None, [_P]),
    "neat_lanes_bytes": (ctypes.c_size_t, [_i32, Dims]),
    "neat_lanes_pack": (ctypes.c_int, [_P, _i32, Dims, _P, ctypes.c_size_t, _P]),
    "neat_lanes_query": (ctypes.c_int, [_P, ctypes.POINTER(LanesInfo)]),
    "neat_forward_lanes": (ctypes.c_int, [_P, _i32, Dims, _P, _P, ctypes.c_uint32, _P]),
    "neat_lanes_pack_recurrent": (ctypes.c_int, [_P, _i32, Dims, _P, ctypes.c_size_t, _P]),
    "neat_forward_lanes_recurrent": (ctypes.c_int, [_P, _i32, Dims, _P, _i32, _P, ctypes.c_uint32, _i32, _P]),
    "neat_forward_lanes_steps": (ctypes.c_int, [_P, _i32, Dims, _P, _i64, _P, _i64, _i32, ctypes.c_uint32,
                                                ctypes.POINTER(_P), _P]),
    "neat_lanes_cache_destroy": (None, [_P]),
    "neat_lanes_tune": (ctypes.c_int, [_P, _i32, Dims, _P, _i64, _P, _i64, _i32, ctypes.POINTER(ctypes.c_uint32), _P]),
    "neat_forward_fused": (ctypes.c_int, [_P, _i32, Dims, _P, _i64, _i32, _P, _i64, _i32, ctypes.POINTER(Launch), _P]),
    "neat_plan_create": (ctypes.c_int, [ctypes.POINTER(PopDesc), _i32, ctypes.POINTER(PlanOptions), _P,
                                        ctypes.POINTER(_P)]),
    "neat_plan_forward": (ctypes.c_int, [_P, _i32, _P]),
    "neat_plan_forward_steps": (ctypes.c_int, [_P, _i32, _i32, _P]),
    "neat_plan_describe": (ctypes.c_int, [_P, ctypes.c_char_p, _i32]),
    "neat_plan_destroy": (None, [_P]),
    "neat_forward_multi_noalloc": (ctypes.c_int, [ctypes.POINTER(PopDesc), _i32, _i32, _P]),
    "neat_cppn_query": (ctypes.c_int, [_P, _i32, Dims, Substrate, ctypes.c_float, _P, _P]),
    "neat_serve_create": (ctypes.c_int, [ctypes.POINTER(ServeCfg), ctypes.POINTER(_P)]),
    "neat_serve_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "neat_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "neat_serve_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _i32, ctypes.POINTER(Result)]),
    "neat_serve_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "neat_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServeStats)]),
    "neat_serve_destroy": (None, [_P]),
    "neat_fill_normal": (ctypes.c_int, [ctypes.c_uint64, _i32, _i64, _P, _P]),
    "neat_last_error": (ctypes.c_char_p, []),
    "neat_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class NeatError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where} failed with {code}: {last_error()}")
        self.code = code


def last_error() -> str:
    return _lib.neat_last_error().decode()


def version() -> str:
    return _lib.neat_version().decode()


def _check(code: int, where: str) -> None:
    if code != NEAT_OK:
        raise NeatError(code, where)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def dims(num_inputs: int, num_outputs: int, max_nodes: int, max_conns: int) -> Dims:
    return Dims(num_inputs, num_outputs, max_nodes, max_conns)


def neat_record_stride(d: Dims) -> int:
    return _lib.neat_record_stride(d)


def neat_transformed_bytes(pop: int, d: Dims) -> int:
    return _lib.neat_transformed_bytes(pop, d)


def neat_default_launch(pop: int, d: Dims, batch: int) -> Launch:
    L = Launch()
    _check(_lib.neat_default_launch(pop, d, batch, ctypes.byref(L)), "neat_default_launch")
    return L


def neat_schedule(transformed, pop: int, d: Dims, order=None, stream=None):
    """Depth-descending genome order (int32 [pop], device) for Launch(order=...)."""
    import torch
    if order is None:
        order = torch.empty(max(pop, 1), dtype=torch.int32, device=transformed.device)
    _check(_lib.neat_schedule(_ptr(transformed), pop, d, _ptr(order), _stream(stream)), "neat_schedule")
    return order[:pop]


def neat_selftest_bounded_wait(limit_us: int = 20000) -> int:
    r = ctypes.c_uint32(0)
    _check(_lib.neat_selftest_bounded_wait(limit_us, ctypes.byref(r)), "neat_selftest_bounded_wait")
    return r.value


def neat_device_error(clear: bool = True) -> int:
    v = ctypes.c_uint32(0)
    _check(_lib.neat_device_error(int(clear), ctypes.byref(v)), "neat_device_error")
    return v.value


def neat_transform(nodes, conns, d: Dims, transformed=None, status=None, stream=None):
    """Transform a population (torch CUDA tensors f32 [P][Nmax][5], [P][Cmax][4]).

    Returns (transformed uint8 tensor, status int32 tensor [P])."""
    import torch
    pop = nodes.shape[0]
    assert nodes.is_cuda and nodes.dtype == torch.float32 and nodes.is_contiguous()
    assert conns.is_cuda and conns.dtype == torch.float32 and conns.is_contiguous()
    assert tuple(nodes.shape[1:]) == (d.max_nodes, 5) and tuple(conns.shape[1:]) == (d.max_conns, 4)
    nbytes = neat_transformed_bytes(pop, d)
    if transformed is None:
        transformed = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=nodes.device)
    if status is None:
        status = torch.empty(max(pop, 1), dtype=torch.int32, device=nodes.device)
    _check(_lib.neat_transform(_ptr(nodes), _ptr(conns), pop, d, _ptr(transformed),
                               transformed.numel() * transformed.element_size(), _ptr(status),
                               _stream(stream)), "neat_transform")
    return transformed, status[:pop]


def neat_transform_recurrent(nodes, conns, d: Dims, transformed=None, status=None, stream=None):
    """Transform for recurrent networks (cycles allowed); as neat_transform."""
    import torch
    pop = nodes.shape[0]
    assert nodes.is_cuda and conns.is_cuda and nodes.is_contiguous() and conns.is_contiguous()
    nbytes = neat_transformed_bytes(pop, d)
    if transformed is None:
        transformed = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=nodes.device)
    if status is None:
        status = torch.empty(max(pop, 1), dtype=torch.int32, device=nodes.device)
    _check(_lib.neat_transform_recurrent(_ptr(nodes), _ptr(conns), pop, d, _ptr(transformed),
                                         transformed.numel() * transformed.element_size(), _ptr(status),
                                         _stream(stream)), "neat_transform_recurrent")
    return transformed, status[:pop]


def neat_default_launch_recurrent(pop: int, d: Dims, batch: int) -> Launch:
    L = Launch()
    _check(_lib.neat_default_launch_recurrent(pop, d, batch, ctypes.byref(L)), "neat_default_launch_recurrent")
    return L


def neat_forward_recurrent(transformed, pop: int, d: Dims, inputs, iterations: int, outputs=None,
                           launch: Launch | None = None, stream=None):
    """Recurrent forward: f32 [P][B][O] after `iterations` synchronous iterations."""
    import torch
    assert inputs.dtype == torch.float32 and inputs.is_contiguous()
    assert inputs.shape[0] == pop and inputs.shape[2] == d.num_inputs
    batch = inputs.shape[1]
    if outputs is None:
        outputs = torch.empty((pop, batch, d.num_outputs), dtype=torch.float32, device=inputs.device)
    _check(_lib.neat_forward_recurrent_ex(_ptr(transformed), pop, d, _ptr(inputs), batch, iterations, _ptr(outputs),
                                          ctypes.byref(launch) if launch is not None else None, _stream(stream)),
           "neat_forward_recurrent")
    return outputs


def neat_gene_stride(d: Dims) -> int:
    return int(_lib.neat_gene_stride(d))


def neat_distance_prepare(nodes, conns, d: Dims, genes=None, status=None, stream=None):
    """Gene records (sorted keys + attributes) of a population for
    neat_distance.  Returns (genes uint8 tensor, status int32 tensor [P])."""
    import torch
    pop = nodes.shape[0]
    assert nodes.is_cuda and conns.is_cuda and nodes.is_contiguous() and conns.is_contiguous()
    assert tuple(nodes.shape[1:]) == (d.max_nodes, 5) and tuple(conns.shape[1:]) == (d.max_conns, 4)
    nbytes = neat_gene_stride(d) * pop
    if genes is None:
        genes = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=nodes.device)
    if status is None:
        status = torch.empty(max(pop, 1), dtype=torch.int32, device=nodes.device)
    _check(_lib.neat_distance_prepare(_ptr(nodes), _ptr(conns), pop, d, _ptr(genes),
                                      genes.numel() * genes.element_size(), _ptr(status), _stream(stream)),
           "neat_distance_prepare")
    return genes, status[:pop]


def neat_distance(genes_a, pop_a: int, genes_b, pop_b: int, d: Dims, c_disjoint: float, c_homologous: float,
                  out=None, stream=None):
    """Distance matrix f32 [pop_a][pop_b] between two prepared populations."""
    import torch
    if out is None:
        out = torch.empty((pop_a, pop_b), dtype=torch.float32, device=genes_a.device)
    ld = out.stride(0) if out.dim() == 2 and pop_a > 0 else max(pop_b, 1)
    assert out.dtype == torch.float32 and (out.dim() != 2 or out.stride(1) == 1)
    _check(_lib.neat_distance(_ptr(genes_a), pop_a, _ptr(genes_b), pop_b, d, c_disjoint, c_homologous, _ptr(out),
                              max(ld, pop_b), _stream(stream)), "neat_distance")
    return out


def neat_speciate(distances, threshold: float, n_reps: int | None = None, species=None, stream=None):
    """Nearest representative under the threshold per row (int32 [pop], -1 = none)."""
    import torch
    pop = distances.shape[0]
    reps = distances.shape[1] if n_reps is None else n_reps
    assert distances.dtype == torch.float32 and distances.stride(1) == 1
    if species is None:
        species = torch.empty(max(pop, 1), dtype=torch.int32, device=distances.device)
    _check(_lib.neat_speciate(_ptr(distances), pop, reps, distances.stride(0), threshold, _ptr(species),
                              _stream(stream)), "neat_speciate")
    return species[:pop]


def neat_mutation_sizes(d: Dims) -> tuple[int, int]:
    """(uint32 words, float normals) of random input per genome for neat_mutate."""
    w, z = _i64(), _i64()
    _check(_lib.neat_mutation_sizes(d, ctypes.byref(w), ctypes.byref(z)), "neat_mutation_sizes")
    return w.value, z.value


def neat_mutate(nodes, conns, d: Dims, m: Mutation, words, normals, new_keys, stream=None):
    """Mutate a population in place (torch CUDA tensors f32 [P][Nmax][5],
    [P][Cmax][4]); words uint32 (int32 tensor) [P][W], normals f32 [P][Z],
    new_keys int32 [P]."""
    import torch
    pop = nodes.shape[0]
    W, Z = neat_mutation_sizes(d)
    assert nodes.is_contiguous() and conns.is_contiguous() and words.is_contiguous() and normals.is_contiguous()
    assert words.numel() >= pop * W and normals.numel() >= pop * Z and new_keys.numel() >= pop
    assert words.dtype in (torch.int32, torch.uint32) and normals.dtype == torch.float32
    assert new_keys.dtype == torch.int32
    _check(_lib.neat_mutate(_ptr(nodes), _ptr(conns), pop, d, ctypes.byref(m), _ptr(words), _ptr(normals),
                            _ptr(new_keys), _stream(stream)), "neat_mutate")
    return nodes, conns


def neat_crossover(nodes, conns, d: Dims, parents, words, nodes_out=None, conns_out=None, stream=None):
    """Children of parent pairs (int32 [K][2], the first the fitter); words
    uint32 (int32 tensor) [K][Nmax + Cmax].  Returns (nodes_out, conns_out)."""
    import torch
    K = parents.shape[0]
    if nodes_out is None:
        nodes_out = torch.empty((K, d.max_nodes, 5), dtype=torch.float32, device=nodes.device)
    if conns_out is None:
        conns_out = torch.empty((K, d.max_conns, 4), dtype=torch.float32, device=nodes.device)
    assert parents.dtype == torch.int32 and parents.is_contiguous() and words.is_contiguous()
    assert words.numel() >= K * (d.max_nodes + d.max_conns)
    _check(_lib.neat_crossover(_ptr(nodes), _ptr(conns), nodes.shape[0], d, _ptr(parents), K, _ptr(words),
                               _ptr(nodes_out), _ptr(conns_out), _stream(stream)), "neat_crossover")
    return nodes_out, conns_out


def neat_substrate_forward(weights, inputs, resolution: int = 16, layers: int = 3, hidden_act: int = 1,
                           output_act: int = 1, outputs=None, stream=None):
    """HyperNEAT substrate outputs f32 [P][B][R] from CPPN weight blocks
    f32 [P][layers-1][R][R] and inputs f32 [P][B][R]."""
    import torch
    P, B, R = inputs.shape
    assert R == resolution * resolution and weights.shape == (P, layers - 1, R, R)
    assert weights.is_contiguous() and inputs.is_contiguous() and inputs.dtype == torch.float32
    if outputs is None:
        outputs = torch.empty((P, B, R), dtype=torch.float32, device=inputs.device)
    _check(_lib.neat_substrate_forward(_ptr(weights), P, Substrate(resolution, layers), _ptr(inputs), B, hidden_act,
                                       output_act, _ptr(outputs), _stream(stream)), "neat_substrate_forward")
    return outputs


def neat_fill_words(seed: int, stream_id: int, out, stream=None):
    """Fill an int32/uint32 tensor with Philox words (see include/neat.h)."""
    _check(_lib.neat_fill_words(seed, stream_id, _ptr(out), out.numel(), _stream(stream)), "neat_fill_words")
    return out


def neat_forward(transformed, pop: int, d: Dims, inputs, outputs=None, launch: Launch | None = None,
                 stream=None):
    """Outputs f32 [P][B][O] of a transformed population on inputs f32 [P][B][I]."""
    import torch
    assert inputs.dtype == torch.float32 and inputs.is_contiguous()
    batch = inputs.shape[1]
    assert inputs.shape[0] == pop and inputs.shape[2] == d.num_inputs
    if outputs is None:
        outputs = torch.empty((pop, batch, d.num_outputs), dtype=torch.float32, device=inputs.device)
    code = _lib.neat_forward_ex(_ptr(transformed), pop, d, _ptr(inputs), batch, _ptr(outputs),
                                ctypes.byref(launch) if launch is not None else None, _stream(stream))
    _check(code, "neat_forward")
    return outputs


def neat_cppn_query(transformed, pop: int, d: Dims, resolution: int = 16, layers: int = 3,
                    threshold: float = 0.2, weights=None, stream=None):
    """Substrate weights f32 [pop][layers-1][res^2][res^2] of CPPN genomes."""
    import torch
    r2 = resolution * resolution
    if weights is None:
        weights = torch.empty((pop, layers - 1, r2, r2), dtype=torch.float32, device=transformed.device)
    _check(_lib.neat_cppn_query(_ptr(transformed), pop, d, Substrate(resolution, layers), threshold,
                                _ptr(weights), _stream(stream)), "neat_cppn_query")
    return weights


class StepsCache:
    """Owner of the CUDA graph that neat_forward_steps builds and replays."""

    def __init__(self):
        self.handle = _P(None)

    def close(self):
        if self.handle.value:
            _lib.neat_steps_cache_destroy(self.handle)
            self.handle = _P(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neat_forward_fused(transformed, pop: int, d: Dims, inputs, outputs, launch: Launch | None = None,
                       stream=None):
    """``steps`` forwards in one launch, the records held in shared memory
    across steps: inputs f32 [S][P][B][I] known in advance -> outputs
    f32 [S][P][B][O]."""
    steps, P, B = inputs.shape[0], inputs.shape[1], inputs.shape[2]
    assert P == pop and outputs.shape[:3] == (steps, pop, B)
    assert inputs.is_contiguous() and outputs.is_contiguous()
    _check(_lib.neat_forward_fused(_ptr(transformed), pop, d, _ptr(inputs), P * B * d.num_inputs, B, _ptr(outputs),
                                   P * B * d.num_outputs, steps, ctypes.byref(launch) if launch is not None else None,
                                   _stream(stream)), "neat_forward_fused")
    return outputs


def neat_forward_steps(transformed, pop: int, d: Dims, inputs, outputs, cache: StepsCache,
                       launch: Launch | None = None, stream=None):
    """Run ``steps`` forwards as one CUDA graph: inputs f32 [S][P][B][I] ->
    outputs f32 [S][P][B][O] (step s reads inputs[s], writes outputs[s])."""
    steps, P, B = inputs.shape[0], inputs.shape[1], inputs.shape[2]
    assert P == pop and outputs.shape[:3] == (steps, pop, B)
    assert inputs.is_contiguous() and outputs.is_contiguous()
    code = _lib.neat_forward_steps(_ptr(transformed), pop, d, _ptr(inputs), P * B * d.num_inputs, B,
                                   _ptr(outputs), P * B * d.num_outputs, steps,
                                   ctypes.byref(launch) if launch is not None else None,
                                   ctypes.byref(cache.handle), _stream(stream))
    _check(code, "neat_forward_steps")
    return outputs


def neat_lanes_bytes(pop: int, d: Dims) -> int:
    return int(_lib.neat_lanes_bytes(pop, d))


def neat_lanes_pack(transformed, pop: int, d: Dims, lanes=None, stream=None):
    """Compile lane programs (two threads per genome) of a transformed
    population; returns the lanes buffer (uint8 CUDA tensor)."""
    import torch
    nbytes = neat_lanes_bytes(pop, d)
    if nbytes == 0:
        raise NeatError(NEAT_EINVAL, "neat_lanes_bytes (dims not supported by lane programs)")
    if lanes is None:
        lanes = torch.empty(nbytes, dtype=torch.uint8, device=transformed.device)
    _check(_lib.neat_lanes_pack(_ptr(transformed), pop, d, _ptr(lanes), lanes.numel() * lanes.element_size(),
                                _stream(stream)), "neat_lanes_pack")
    return lanes


def neat_lanes_pack_recurrent(transformed, pop: int, d: Dims, lanes=None, stream=None):
    """Compile recurrent lane programs from records of
    neat_transform_recurrent; returns the lanes buffer (uint8 CUDA tensor)."""
    import torch
    nbytes = neat_lanes_bytes(pop, d)
    if nbytes == 0:
        raise NeatError(NEAT_EINVAL, "neat_lanes_bytes (dims not supported by lane programs)")
    if lanes is None:
        lanes = torch.empty(nbytes, dtype=torch.uint8, device=transformed.device)
    _check(_lib.neat_lanes_pack_recurrent(_ptr(transformed), pop, d, _ptr(lanes),
                                          lanes.numel() * lanes.element_size(), _stream(stream)),
           "neat_lanes_pack_recurrent")
    return lanes


def neat_forward_lanes_recurrent(lanes, pop: int, d: Dims, inputs, iterations: int, outputs=None,
                                 stage_bytes: int = 0, pdl: bool = False, stream=None):
    """`iterations` recurrent iterations from lane programs: inputs f32 [P][I]
    (or [P][1][I]) -> outputs f32 with the same leading shape and O last."""
    import torch
    assert inputs.is_contiguous() and inputs.numel() == pop * d.num_inputs
    if outputs is None:
        outputs = torch.empty(tuple(inputs.shape[:-1]) + (d.num_outputs,), dtype=torch.float32, device=inputs.device)
    _check(_lib.neat_forward_lanes_recurrent(_ptr(lanes), pop, d, _ptr(inputs), iterations, _ptr(outputs),
                                             stage_bytes, int(pdl), _stream(stream)), "neat_forward_lanes_recurrent")
    return outputs


def neat_lanes_query(lanes) -> LanesInfo:
    info = LanesInfo()
    _check(_lib.neat_lanes_query(_ptr(lanes), ctypes.byref(info)), "neat_lanes_query")
    return info


def neat_forward_lanes(lanes, pop: int, d: Dims, inputs, outputs=None, stage_bytes: int = 0, stream=None):
    """One forward from lane programs: inputs f32 [P][I] (or [P][1][I]) ->
    outputs f32 with the same leading shape and O last."""
    import torch
    assert inputs.is_contiguous() and inputs.numel() == pop * d.num_inputs
    if outputs is None:
        outputs = torch.empty(tuple(inputs.shape[:-1]) + (d.num_outputs,), dtype=torch.float32, device=inputs.device)
    _check(_lib.neat_forward_lanes(_ptr(lanes), pop, d, _ptr(inputs), _ptr(outputs), stage_bytes, _stream(stream)),
           "neat_forward_lanes")
    return outputs


class LanesCache:
    """Owner of the CUDA graph that neat_forward_lanes_steps builds and replays."""

    def __init__(self):
        self.handle = _P(None)

    def close(self):
        if self.handle.value:
            _lib.neat_lanes_cache_destroy(self.handle)
            self.handle = _P(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neat_forward_lanes_steps(lanes, pop: int, d: Dims, inputs, outputs, cache: LanesCache, stage_bytes: int = 0,
                             stream=None):
    """``steps`` forwards from lane programs as one CUDA graph: inputs f32
    [S][P][1][I] (or [S][P][I]) -> outputs f32 [S][P][1][O] (or [S][P][O])."""
    steps = inputs.shape[0]
    assert inputs.shape[1] == pop and outputs.shape[0] == steps and outputs.shape[1] == pop
    assert inputs.is_contiguous() and outputs.is_contiguous()
    _check(_lib.neat_forward_lanes_steps(_ptr(lanes), pop, d, _ptr(inputs), pop * d.num_inputs, _ptr(outputs),
                                         pop * d.num_outputs, steps, stage_bytes, ctypes.byref(cache.handle),
                                         _stream(stream)), "neat_forward_lanes_steps")
    return outputs


def neat_lanes_tune(lanes, pop: int, d: Dims, inputs, outputs, stream=None) -> int:
    """stage_bytes for neat_forward_lanes_steps, timed on these arrays
    (inputs [S][P][...][I], outputs [S][P][...][O]; writes outputs)."""
    steps = inputs.shape[0]
    assert inputs.shape[1] == pop and outputs.shape[0] == steps and outputs.shape[1] == pop
    assert inputs.is_contiguous() and outputs.is_contiguous()
    sb = ctypes.c_uint32(0)
    _check(_lib.neat_lanes_tune(_ptr(lanes), pop, d, _ptr(inputs), pop * d.num_inputs, _ptr(outputs),
                                pop * d.num_outputs, steps, ctypes.byref(sb), _stream(stream)), "neat_lanes_tune")
    return int(sb.value)


class Plan:
    """neat_plan_*: several transformed populations, one persistent launch per step.

    pops: sequence of dicts with keys transformed, pop, dims, inputs, outputs
    (torch CUDA tensors; inputs [S][pop][batch][I] or [pop][batch][I],
    outputs likewise), the step strides being taken from the leading
    dimension when the tensors are 4-D."""

    def __init__(self, pops, autotune: bool = False, size_buckets: bool = True, block_threads: int = 0,
                 pdl: bool = True, stream=None):
        descs = (PopDesc * len(pops))()
        self._keep = []
        for i, p in enumerate(pops):
            x, y = p["inputs"], p["outputs"]
            batch = x.shape[-2]
            d = p["dims"]
            in_step = x.shape[-3] * batch * d.num_inputs if x.dim() == 4 else 0
            out_step = y.shape[-3] * batch * d.num_outputs if y.dim() == 4 else 0
            descs[i] = PopDesc(_ptr(p["transformed"]), p["pop"], d, batch, _ptr(x), in_step, _ptr(y), out_step)
            self._keep.append((p["transformed"], x, y))
        opt = PlanOptions(int(autotune), int(size_buckets), block_threads, int(pdl))
        self.handle = _P(None)
        _check(_lib.neat_plan_create(descs, len(pops), ctypes.byref(opt), _stream(stream), ctypes.byref(self.handle)),
               "neat_plan_create")

    def forward(self, step: int = 0, stream=None):
        _check(_lib.neat_plan_forward(self.handle, step, _stream(stream)), "neat_plan_forward")

    def forward_steps(self, first_step: int, steps: int, stream=None):
        _check(_lib.neat_plan_forward_steps(self.handle, first_step, steps, _stream(stream)),
               "neat_plan_forward_steps")

    def describe(self) -> dict:
        import json
        n = _lib.neat_plan_describe(self.handle, None, 0)
        buf = ctypes.create_string_buffer(n)
        _lib.neat_plan_describe(self.handle, buf, n)
        return json.loads(buf.value.decode())

    def close(self):
        if self.handle.value:
            _lib.neat_plan_destroy(self.handle)
            self.handle = _P(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """neat_serve_*: continuous batching of evaluation requests under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 256):
        self.handle = _P(None)
        cfg = ServeCfg(hbm_budget_bytes, max_active, 0)
        _check(_lib.neat_serve_create(ctypes.byref(cfg), ctypes.byref(self.handle)), "neat_serve_create")

    def submit(self, nodes: np.ndarray, conns: np.ndarray, d: Dims, batch: int, steps: int, obs_seed: int,
               outputs, out_step_stride: int = 0, borrow: bool = False) -> int:
        """Queue a request; with borrow=True the host arrays must stay alive
        (and unchanged) until the request is done."""
        nodes = np.ascontiguousarray(nodes, dtype=np.float32)
        conns = np.ascontiguousarray(conns, dtype=np.float32)
        req = Request(nodes.ctypes.data, conns.ctypes.data, nodes.shape[0], d, batch, steps,
                      REQ_BORROW_HOST if borrow else 0, obs_seed, _ptr(outputs), out_step_stride)
        t = ctypes.c_uint64(0)
        _check(_lib.neat_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)), "neat_serve_submit")
        return t.value

    def poll(self, ticket: int):
        r = Result()
        code = _lib.neat_serve_poll(self.handle, ticket, ctypes.byref(r))
        return code, r

    def wait(self, ticket: int, timeout_ms: int = 60000):
        r = Result()
        code = _lib.neat_serve_wait(self.handle, ticket, timeout_ms, ctypes.byref(r))
        return code, r

    def cancel(self, ticket: int):
        _check(_lib.neat_serve_cancel(self.handle, ticket), "neat_serve_cancel")

    def stats(self) -> ServeStats:
        st = ServeStats()
        _check(_lib.neat_serve_stats(self.handle, ctypes.byref(st)), "neat_serve_stats")
        return st

    def close(self):
        if self.handle.value:
            _lib.neat_serve_destroy(self.handle)
            self.handle = _P(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neat_fill_normal(seed: int, step: int, out, stream=None):
    _check(_lib.neat_fill_normal(seed, step, out.numel(), _ptr(out), _stream(stream)), "neat_fill_normal")
    return out


def pop_descs(pops):
    """neat_pop_desc array for dicts as taken by Plan (kept alive by the caller)."""
    descs = (PopDesc * len(pops))()
    for i, p in enumerate(pops):
        x, y = p["inputs"], p["outputs"]
        batch = x.shape[-2]
        d = p["dims"]
        in_step = x.shape[-3] * batch * d.num_inputs if x.dim() == 4 else 0
        out_step = y.shape[-3] * batch * d.num_outputs if y.dim() == 4 else 0
        descs[i] = PopDesc(_ptr(p["transformed"]), p["pop"], d, batch, _ptr(x), in_step, _ptr(y), out_step)
    return descs


def neat_forward_multi_noalloc(pops, step: int = 0, stream=None):
    """One step of several populations through the allocation-free entry point."""
    descs = pop_descs(pops)
    _check(_lib.neat_forward_multi_noalloc(descs, len(pops), step, _stream(stream)), "neat_forward_multi_noalloc")


# ----------------------------------------------------------- record decoding

@dataclass
class Decoded:
    """Host view of transformed records, in the oracle's terms (node rows)."""
    n_nodes: np.ndarray      # [P]
    n_levels: np.ndarray     # [P]
    n_edges: np.ndarray      # [P]
    status: np.ndarray       # [P] uint32
    order: np.ndarray        # [P][Nmax] node row per position, -1 pad
    level_ptr: np.ndarray    # [P][Nmax+1] (padded with n_nodes)
    in_ptr: np.ndarray       # [P][Nmax+1] by position (padded with n_edges)
    in_src: np.ndarray       # [P][Cmax] source node row, -1 pad
    in_w: np.ndarray         # [P][Cmax] float32 weights, 0 pad
    in_pos: np.ndarray       # [P][I]
    out_pos: np.ndarray      # [P][O]
    uniform_activation: np.ndarray = None   # [P] id or 255
    uniform_aggregation: np.ndarray = None  # [P] id or 255


def decode_records(buf: np.ndarray, pop: int, d: Dims) -> Decoded:
    """Unpack ``pop`` records (a host uint8 copy of the transformed buffer)
    following the layout documented in include/neat.h."""
    stride = neat_record_stride(d)
    N, C, I, O = d.max_nodes, d.max_conns, d.num_inputs, d.num_outputs
    buf = np.ascontiguousarray(buf[: stride * pop]).reshape(pop, stride)
    hdr = buf[:, :32].copy().view(np.uint32).reshape(pop, 8)
    out = Decoded(n_nodes=(hdr[:, 0] & 0xFFFF).astype(np.int32), n_levels=(hdr[:, 0] >> 16).astype(np.int32),
                  n_edges=hdr[:, 1].astype(np.int32), status=hdr[:, 2].copy(),
                  uniform_activation=(hdr[:, 3] & 0xFF).astype(np.int32),
                  uniform_aggregation=((hdr[:, 3] >> 8) & 0xFF).astype(np.int32),
                  order=np.full((pop, N), -1, np.int32), level_ptr=np.zeros((pop, N + 1), np.int32),
                  in_ptr=np.zeros((pop, N + 1), np.int32), in_src=np.full((pop, C), -1, np.int32),
                  in_w=np.zeros((pop, C), np.float32), in_pos=np.zeros((pop, I), np.int32),
                  out_pos=np.zeros((pop, O), np.int32))
    for g in range(pop):
        n, nl, E = int(hdr[g, 0] & 0xFFFF), int(hdr[g, 0] >> 16), int(hdr[g, 1])
        if hdr[g, 2] & G_ERROR_MASK:
            continue
        off_edge, off_level, off_io = int(hdr[g, 5]), int(hdr[g, 6]), int(hdr[g, 7])
        nodes = buf[g, 32:32 + 16 * n].copy()
        rows = nodes.view(np.uint16).reshape(n, 8)[:, 7].astype(np.int32)
        ebeg = nodes.view(np.uint16).reshape(n, 8)[:, 4].astype(np.int32)
        ecnt = nodes.view(np.uint16).reshape(n, 8)[:, 5].astype(np.int32)
        out.order[g, :n] = rows
        lev = buf[g, off_level:off_level + 2 * (nl + 1)].copy().view(np.uint16).astype(np.int32)
        out.level_ptr[g, :nl + 1] = lev
        out.level_ptr[g, nl + 1:] = n
        starts = np.concatenate([[0], np.cumsum(ecnt)])
        out.in_ptr[g, :n] = starts[:-1]
        out.in_ptr[g, n:] = E
        assert np.all(ebeg[ecnt > 0] + ecnt[ecnt > 0] <= E)
        edges = buf[g, off_edge:off_edge + 8 * E].copy()
        out.in_w[g, :E] = edges.view(np.float32).reshape(E, 2)[:, 0]
        src_pos = edges.view(np.uint32).reshape(E, 2)[:, 1].astype(np.int64)
        out.in_src[g, :E] = rows[src_pos]
        io = buf[g, off_io:off_io + 2 * (I + O)].copy().view(np.uint16).astype(np.int32)
        out.in_pos[g] = io[:I]
        out.out_pos[g] = io[I:]
        # edge_begin/edge_count must tile [0, E) in position order
        assert starts[-1] == E and np.array_equal(starts[:-1][ecnt > 0], ebeg[ecnt > 0])
    return out
