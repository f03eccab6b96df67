"""Mutation and crossover through the C ABI (neat_mutate, neat_crossover,
neat_fill_words) against the FP64 oracle, on the same random inputs.

Structure must match exactly: which rows are present, keys, connection
endpoints, enabled flags, activation and aggregation ids (the decisions are
integer comparisons of the same words).  Bias, response and weight values
pass within |gpu - ref| <= 1e-5 max(1, |ref|) (one float rounding of a
multiply-add against double).  Crossover copies values, so it must match bit
for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome
from tests.parity import assert_outputs_close

pytestmark = pytest.mark.gpu

FIELDS = ("node_add", "node_delete", "conn_add", "conn_delete", "bias_init_mean", "bias_init_std",
          "bias_mutate_power", "bias_mutate_rate", "bias_replace_rate", "response_init_mean", "response_init_std",
          "response_mutate_power", "response_mutate_rate", "response_replace_rate", "weight_init_mean",
          "weight_init_std", "weight_mutate_power", "weight_mutate_rate", "weight_replace_rate",
          "activation_replace_rate", "aggregation_replace_rate", "enabled_mutate_rate", "activation_default",
          "aggregation_default", "feedforward")

# the appendix's Brax settings (node_add 0.2, conn_add 0.4, bias / weight
# mutate 0.5 power at rates 0.7 / 0.8, replace 0.1, response fixed)
PAPER = dict(node_add=0.2, conn_add=0.4, bias_init_std=1.0, bias_mutate_power=0.5, bias_mutate_rate=0.7,
             bias_replace_rate=0.1, response_init_mean=1.0, weight_init_std=1.0, weight_mutate_power=0.5,
             weight_mutate_rate=0.8, weight_replace_rate=0.1)
BUSY = dict(node_add=0.6, node_delete=0.3, conn_add=0.7, conn_delete=0.3, bias_init_mean=0.1, bias_init_std=1.5,
            bias_mutate_power=0.5, bias_mutate_rate=0.5, bias_replace_rate=0.3, response_init_mean=1.0,
            response_init_std=0.2, response_mutate_power=0.1, response_mutate_rate=0.4, response_replace_rate=0.2,
            weight_init_mean=-0.2, weight_init_std=2.0, weight_mutate_power=0.7, weight_mutate_rate=0.6,
            weight_replace_rate=0.3, activation_replace_rate=0.3, aggregation_replace_rate=0.2,
            enabled_mutate_rate=0.05, activation_options=[0, 1, 2, 4, 5], aggregation_options=[0, 2, 3])


@pytest.fixture(scope="module")
def neat():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2404_01817_gb300 import neat as N
    return N


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _configs(neat, **kw):
    kw = dict(kw)
    g = neat.mutation(**kw)
    o = oracle.mutation_config(**kw)
    for f in FIELDS:
        assert getattr(g, f) == getattr(o, f)
    return g, o


def _random_inputs(seed, P, N, C):
    Wn, Zn = oracle.mutation_words(N, C)
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2**32, size=(P, Wn), dtype=np.uint64).astype(np.uint32)
    z = rng.standard_normal((P, Zn)).astype(np.float32)
    return u, z


def _gpu_mutate(neat, pop, cfg, u, z, keys):
    d = neat.dims(pop.num_inputs, pop.num_outputs, pop.max_nodes, pop.max_conns)
    nodes, conns = _dev(pop.nodes), _dev(pop.conns)
    neat.neat_mutate(nodes, conns, d, cfg, _dev(u.view(np.int32)), _dev(z), _dev(np.asarray(keys, np.int32)))
    return nodes.cpu().numpy(), conns.cpu().numpy()


def _compare(gn, gc, on, oc, what):
    # structure exactly
    np.testing.assert_array_equal(np.isnan(gn), np.isnan(on), err_msg=f"{what}: node rows")
    np.testing.assert_array_equal(np.isnan(gc), np.isnan(oc), err_msg=f"{what}: connection rows")
    for col in (0, 3, 4):
        np.testing.assert_array_equal(np.nan_to_num(gn[..., col]), np.nan_to_num(on[..., col]),
                                      err_msg=f"{what}: node column {col}")
    for col in (0, 1, 2):
        np.testing.assert_array_equal(np.nan_to_num(gc[..., col]), np.nan_to_num(oc[..., col]),
                                      err_msg=f"{what}: connection column {col}")
    # values within the tolerance
    assert_outputs_close(gn[..., 1:3], on[..., 1:3], what=f"{what}: bias/response")
    assert_outputs_close(gc[..., 3], oc[..., 3], what=f"{what}: weights")


def _dag(seed, pop, nmax=24, cmax=60):
    return W.random_dag_population(seed, pop, 3, 2, nmax, cmax, hidden=lambda r: int(r.integers(0, 12)),
                                   edges=lambda r, n: int(r.integers(n // 2, 2 * n)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.2)


@pytest.mark.parametrize("name,kw", [("paper", PAPER), ("busy", BUSY), ("busy-recurrent", dict(BUSY, feedforward=0))])
def test_mutation_matches_oracle_over_generations(neat, name, kw):
    g_cfg, o_cfg = _configs(neat, **kw)
    p = _dag(11, 300)
    gpu = (p.nodes, p.conns)
    ref = (p.nodes, p.conns)
    for gen in range(4):
        u, z = _random_inputs(100 + gen, 300, 24, 60)
        keys = 1000 + 300 * gen + np.arange(300)
        gn, gc = _gpu_mutate(neat, W.Population(*gpu, 3, 2), g_cfg, u, z, keys)
        on, oc = oracle.mutate(*ref, 3, 2, o_cfg, u, z, keys)
        _compare(gn, gc, on, oc, f"{name} generation {gen}")
        gpu = (gn, gc)
        ref = (on.astype(np.float32), oc.astype(np.float32))
    if kw.get("feedforward", 1):
        st = oracle.transform(gpu[0], gpu[1], 3, 2)["status"]
        assert (st & 0xFF == 0).all()                           # still valid and acyclic
    assert (~np.isnan(gpu[0][:, :, 0])).sum() != (~np.isnan(p.nodes[:, :, 0])).sum()   # structure changed


def test_node_split_preserves_the_function_on_gpu(neat):
    p = W.random_dag_population(12, 200, 3, 2, 30, 80, hidden=lambda r: int(r.integers(0, 10)),
                                edges=lambda r, n: int(r.integers(n, 2 * n)), acts=(W.ACT_IDENTITY,),
                                aggs=(W.AGG_SUM,), p_disabled=0.1)
    cfg = neat.mutation(node_add=1.0, activation_default=0, bias_init_mean=0.0, response_init_mean=1.0)
    u, z = _random_inputs(13, 200, 30, 80)
    u[:, 2:] = 0xFFFFFFFF                                        # nothing but the split
    u[:, 0] = 0
    gn, gc = _gpu_mutate(neat, p, cfg, u, z, 500 + np.arange(200))
    assert ((~np.isnan(gn[:, :, 0])).sum(1) == (~np.isnan(p.nodes[:, :, 0])).sum(1) + 1).all()
    x = W.normal_inputs(14, (200, 4, 3))
    before = oracle.forward(p.nodes, p.conns, 3, 2, x)
    after = oracle.forward(gn, gc, 3, 2, x)
    assert_outputs_close(after, before, what="node split")


def test_mutation_edge_cases(neat):
    import torch
    # full tensors: no free rows, so additions are skipped; an empty genome stays empty
    full = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 1)], [(0, 1, 1, 0.5)], 2, 1)
    empty = genome([None, None], [None], 2, 1)
    nodes = np.concatenate([full[0], empty[0]])
    conns = np.concatenate([full[1], empty[1]])
    g_cfg, o_cfg = _configs(neat, node_add=1.0, conn_add=1.0, weight_mutate_rate=1.0, weight_mutate_power=1.0)
    u, z = _random_inputs(15, 2, 2, 1)
    u[:, [0, 4]] = 0
    gn, gc = _gpu_mutate(neat, W.Population(nodes, conns, 1, 1), g_cfg, u, z, [7, 8])
    on, oc = oracle.mutate(nodes, conns, 1, 1, o_cfg, u, z, [7, 8])
    _compare(gn, gc, on, oc, "edge cases")
    d = neat.dims(1, 1, 2, 1)
    e = torch.empty((0, 2, 5), device="cuda")
    neat.neat_mutate(e, torch.empty((0, 1, 4), device="cuda"), d, g_cfg, torch.zeros(1, dtype=torch.int32,
                     device="cuda"), torch.zeros(1, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))


def test_largest_genomes(neat):
    p = W.related_population(16, 4, 3, 2, 1024, 8192, ancestor_hidden=500, ancestor_edges=5000, new_nodes=200,
                             new_conns=1000, key_pool=300)
    g_cfg, o_cfg = _configs(neat, **dict(BUSY, node_delete=0.0))
    u, z = _random_inputs(17, 4, 1024, 8192)
    u[:, [0, 4]] = 0                                              # a split and a connection addition each
    gn, gc = _gpu_mutate(neat, p, g_cfg, u, z, 5000 + np.arange(4))
    on, oc = oracle.mutate(p.nodes, p.conns, 3, 2, o_cfg, u, z, 5000 + np.arange(4))
    _compare(gn, gc, on, oc, "1024 nodes / 8192 connections")


def test_crossover_matches_oracle_bit_for_bit(neat):
    p = W.related_population(18, 400, 3, 2, 24, 60, ancestor_hidden=6, ancestor_edges=20, new_nodes=6,
                             new_conns=12, key_pool=10)
    rng = np.random.default_rng(19)
    parents = rng.integers(0, 400, size=(500, 2)).astype(np.int32)
    parents[:20, 1] = parents[:20, 0]                             # self-crosses
    words = rng.integers(0, 2**32, size=(500, 84), dtype=np.uint64).astype(np.uint32)
    d = neat.dims(3, 2, 24, 60)
    gn, gc = neat.neat_crossover(_dev(p.nodes), _dev(p.conns), d, _dev(parents), _dev(words.view(np.int32)))
    on, oc = oracle.crossover(p.nodes, p.conns, parents, words)
    np.testing.assert_array_equal(gn.cpu().numpy().view(np.uint32), on.view(np.uint32))
    np.testing.assert_array_equal(gc.cpu().numpy().view(np.uint32), oc.view(np.uint32))
    np.testing.assert_array_equal(gn.cpu().numpy()[:20].view(np.uint32), p.nodes[parents[:20, 0]].view(np.uint32))


def test_crossover_launch_shapes_and_bad_parents(neat):
    """Genomes of at most 64 node rows and 256 connection rows cross with
    128 threads per child, larger ones with 256: the same parents padded to
    100 node rows (words moved with the rows) give the same children, bit
    for bit with the oracle.  A parent index outside [0, pop) gives an empty
    child; the other children are unaffected."""
    p = W.related_population(20, 300, 3, 2, 24, 60, ancestor_hidden=6, ancestor_edges=20, new_nodes=6,
                             new_conns=12, key_pool=10)
    rng = np.random.default_rng(21)
    parents = rng.integers(0, 300, size=(333, 2)).astype(np.int32)
    words = rng.integers(0, 2**32, size=(333, 84), dtype=np.uint64).astype(np.uint32)
    on, oc = oracle.crossover(p.nodes, p.conns, parents, words)
    bad = parents.copy()
    bad[5, 0], bad[6, 1], bad[7, 1] = 300, -1, 1 << 30
    for nmax in (24, 100):
        nodes = np.full((300, nmax, 5), np.nan, np.float32)
        nodes[:, :24] = p.nodes
        pw = np.zeros((333, nmax + 60), np.uint32)
        pw[:, :24], pw[:, nmax:] = words[:, :24], words[:, 24:]
        d = neat.dims(3, 2, nmax, 60)
        gn, gc = neat.neat_crossover(_dev(nodes), _dev(p.conns), d, _dev(parents), _dev(pw.view(np.int32)))
        gn = gn.cpu().numpy()
        assert np.isnan(gn[:, 24:]).all()
        np.testing.assert_array_equal(gn[:, :24].view(np.uint32), on.view(np.uint32), err_msg=f"nmax={nmax}")
        np.testing.assert_array_equal(gc.cpu().numpy().view(np.uint32), oc.view(np.uint32), err_msg=f"nmax={nmax}")
        bn, bc = neat.neat_crossover(_dev(nodes), _dev(p.conns), d, _dev(bad), _dev(pw.view(np.int32)))
        bn, bc = bn.cpu().numpy(), bc.cpu().numpy()
        assert np.isnan(bn[5:8]).all() and np.isnan(bc[5:8]).all()
        keep = np.r_[0:5, 8:333]
        np.testing.assert_array_equal(bn[keep, :24].view(np.uint32), on[keep].view(np.uint32))
        np.testing.assert_array_equal(bc[keep].view(np.uint32), oc[keep].view(np.uint32))


def test_random_words(neat):
    import torch
    a = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    b = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    neat.neat_fill_words(7, 3, a)
    neat.neat_fill_words(7, 3, b)
    assert torch.equal(a, b)                                      # a function of (seed, stream, index)
    neat.neat_fill_words(7, 4, b)
    assert (a != b).float().mean().item() > 0.99
    odd = torch.empty(1001, dtype=torch.int32, device="cuda")
    neat.neat_fill_words(7, 3, odd)
    assert torch.equal(odd, a[:1001])                             # prefix property, ragged tail
    v = a.cpu().numpy().view(np.uint32).astype(np.float64)
    assert abs(v.mean() / 2**32 - 0.5) < 0.002
    bits = np.unpackbits(a.cpu().numpy().view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.001


def test_full_generation_at_bench_size_sampled(neat):
    """The evolve workload as bench.py runs it: 10 000 Ant-shaped genomes in
    mid-evolution, random parent pairs, device-generated Philox words and
    normals, crossover, mutation with the appendix's settings, transform.
    Sampled children against the oracle's crossover and mutation on the same
    words; every child valid and acyclic."""
    import torch
    P = 10000
    p = W.ant_related_population(0, P, acyclic=True)
    d = neat.dims(27, 8, 50, 200)
    nodes, conns = _dev(p.nodes), _dev(p.conns)
    parents = np.random.default_rng(5).integers(0, P, size=(P, 2)).astype(np.int32)
    Wn, Zn = neat.neat_mutation_sizes(d)
    xw = neat.neat_fill_words(11, 0, torch.empty((P, 250), dtype=torch.int32, device="cuda"))
    mw = neat.neat_fill_words(11, 1, torch.empty((P, Wn), dtype=torch.int32, device="cuda"))
    z = neat.neat_fill_normal(11, 0, torch.empty((P, Zn), device="cuda"))
    keys = np.arange(1000, 1000 + P, dtype=np.int32)
    g_cfg, o_cfg = _configs(neat, **PAPER)
    cn, cc = neat.neat_crossover(nodes, conns, d, _dev(parents), xw)
    neat.neat_mutate(cn, cc, d, g_cfg, mw, z, _dev(keys))
    rec, status = neat.neat_transform(cn, cc, d)
    assert (status.cpu().numpy() & 0xFF == 0).all()
    idx = np.arange(0, P, 97)
    on, oc = oracle.crossover(p.nodes, p.conns, parents[idx], xw.cpu().numpy().view(np.uint32)[idx])
    on, oc = oracle.mutate(on, oc, 27, 8, o_cfg, mw.cpu().numpy().view(np.uint32)[idx], z.cpu().numpy()[idx], keys[idx])
    _compare(cn.cpu().numpy()[idx], cc.cpu().numpy()[idx], on, oc, "full generation sample")
