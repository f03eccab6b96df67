"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Transform outputs (order, levels, incoming edge lists, status) must match the
oracle exactly; forward outputs within |gpu - ref| <= 1e-5 max(1, |ref|).
"""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome, stack
from tests.parity import assert_outputs_close, assert_topology_equal, compare_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def neat():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2404_01817_gb300 import neat as N
    return N


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _transform(neat, pop):
    d = neat.dims(pop.num_inputs, pop.num_outputs, pop.max_nodes, pop.max_conns)
    rec, st = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    return d, rec, st


def _decode(neat, rec, pop, d):
    return neat.decode_records(rec.cpu().numpy(), pop, d)


def _check_transform(neat, pop, what):
    d, rec, st = _transform(neat, pop)
    ref = oracle.transform(pop.nodes, pop.conns, pop.num_inputs, pop.num_outputs)
    dec = _decode(neat, rec, pop.pop, d)
    assert_topology_equal(dec, ref, pop.pop, what)
    np.testing.assert_array_equal(st.cpu().numpy().astype(np.uint32), ref["status"])
    return d, rec


# ------------------------------------------------------------- transform

def test_transform_xor(neat):
    _check_transform(neat, W.xor_population(0, 100), "xor")


def test_transform_ant_full_population(neat):
    _check_transform(neat, W.ant_population(0, 10000), "ant")


@pytest.mark.parametrize("bucket", range(4))
def test_transform_batched_buckets(neat, bucket):
    pops = W.batched_populations(0, pop=512)
    _check_transform(neat, pops[bucket], f"batched Nmax={pops[bucket].max_nodes}")


def test_transform_cppn(neat):
    _check_transform(neat, W.cppn_population(0, 1000), "cppn")


def _malformed_population(seed, n):
    """Random small genomes with planted defects of every kind."""
    base = W.random_dag_population(seed, n, 3, 2, 16, 48, hidden=lambda r: int(r.integers(0, 10)),
                                   edges=lambda r, k: int(r.integers(k, 3 * k)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.2)
    rng = np.random.default_rng(seed)
    nodes, conns = base.nodes.copy(), base.conns.copy()
    for g in range(n):
        kind = g % 12
        nv = np.nonzero(~np.isnan(nodes[g, :, 0]))[0]
        cv = np.nonzero(~np.isnan(conns[g, :, 0]))[0]
        free_c = np.nonzero(np.isnan(conns[g, :, 0]))[0]
        if kind == 1 and len(cv):                      # cycle through an enabled back edge
            c = cv[rng.integers(len(cv))]
            if free_c.size:
                conns[g, free_c[0]] = (conns[g, c, 1], conns[g, c, 0], 1, 0.5)
                conns[g, c, 2] = 1
        elif kind == 2:                                # duplicate key
            nodes[g, nv[-1], 0] = nodes[g, nv[-2], 0]
        elif kind == 3:                                # fractional key
            nodes[g, nv[-1], 0] += 0.5
        elif kind == 4:                                # bad enum
            nodes[g, nv[-1], 4] = 7
        elif kind == 5 and len(cv) and free_c.size:    # duplicate connection
            conns[g, free_c[0]] = conns[g, cv[0]]
        elif kind == 6 and len(cv):                    # NaN weight
            conns[g, cv[0], 2] = 1
            conns[g, cv[0], 3] = np.nan
        elif kind == 7:                                # missing output
            rows = nv[nodes[g, nv, 0] == 3]
            nodes[g, rows, :] = np.nan
        elif kind == 8 and free_c.size:                # dangling
            conns[g, free_c[0]] = (1, 999, 1, 1.0)
        elif kind == 9 and free_c.size:                # into input
            conns[g, free_c[0]] = (4, 0, 1, 1.0)
        elif kind == 10:                               # permuted rows and interior holes
            nodes[g] = nodes[g][rng.permutation(16)]
            conns[g] = conns[g][rng.permutation(48)]
        elif kind == 11 and len(cv):                   # NaN bias
            nodes[g, nv[-1], 1] = np.nan
    return W.Population(nodes, conns, 3, 2)


def test_transform_status_bits_fuzz(neat):
    pop = _malformed_population(7, 600)
    _check_transform(neat, pop, "malformed")
    ref = oracle.transform(pop.nodes, pop.conns, 3, 2)
    seen = np.bitwise_or.reduce(ref["status"])
    assert seen & 0xFF == 0x7F and seen & 0x300 == 0x300     # every bit exercised


def test_transform_max_sizes(neat):
    """Nmax = 1024 and Cmax = 8192: a dense random DAG at the limits."""
    pop = W.random_dag_population(3, 6, 16, 8, 1024, 8192, hidden=lambda r: 1000,
                                  edges=lambda r, n: 8192, acts=W.ALL_ACTS, aggs=W.ALL_AGGS)
    d, rec = _check_transform(neat, pop, "max")
    x = W.normal_inputs(3, (6, 5, 16))
    y = neat.neat_forward(rec, 6, d, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 16, 8, x), what="max sizes")


def test_forward_max_sizes_with_64_inputs(neat):
    """Nmax 1024, Cmax 8192, 64 input vectors per genome: a 32-column value
    tile would not fit one block beside the 84 KB record, so the default
    launch halves the tile; the outputs match the oracle."""
    pop = W.random_dag_population(4, 6, 16, 8, 1024, 8192, hidden=lambda r: 1000,
                                  edges=lambda r, n: 8192, acts=W.ALL_ACTS, aggs=W.ALL_AGGS)
    d, rec = _check_transform(neat, pop, "max, 64 inputs")
    L = neat.neat_default_launch(6, d, 64)
    assert L.tile == 16 and L.group == 256
    x = W.normal_inputs(4, (6, 64, 16))
    y = neat.neat_forward(rec, 6, d, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 16, 8, x), what="max sizes, 64 inputs")


# --------------------------------------------------------------- forward

def test_forward_xor(neat):
    pop = W.xor_population(0, 100)
    d, rec = _check_transform(neat, pop, "xor")
    x = W.xor_inputs(100)
    y = neat.neat_forward(rec, 100, d, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 3, 1, x), what="xor")


def test_forward_xor_handworked(neat):
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "xor_handworked.json")))
    gs = [genome([tuple(r) for r in fx[k]["nodes"]], [tuple(r) for r in fx[k]["conns"]], 10, 20)
          for k in ("encoding_bias_in_nodes", "encoding_bias_input")]
    nodes, conns = stack(gs)
    pop = W.Population(nodes, conns, 3, 1)
    d, rec = _check_transform(neat, pop, "xor golden")
    x = np.broadcast_to(np.asarray(fx["inputs"], np.float32), (2, 4, 3)).copy()
    y = neat.neat_forward(rec, 2, d, _dev(x)).cpu().numpy()[:, :, 0]
    want = np.array([float(v) for v in fx["expected_y"]])
    assert np.all(np.abs(y - want) <= 1e-5 * np.maximum(1, np.abs(want)))


def test_forward_ant_small(neat):
    pop = W.ant_population(0, 997)                           # not a multiple of any tile
    d, rec = _check_transform(neat, pop, "ant")
    x = W.normal_inputs(1, (997, 3, 27))
    y = neat.neat_forward(rec, 997, d, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 27, 8, x), what="ant")


@pytest.mark.parametrize("bucket", range(4))
def test_forward_batched_buckets(neat, bucket):
    pops = W.batched_populations(0, pop=96)
    pop = pops[bucket]
    d, rec = _check_transform(neat, pop, "batched")
    x = W.normal_inputs(2, (96, 64, 8))
    y = neat.neat_forward(rec, 96, d, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 8, 4, x), what=f"Nmax={pop.max_nodes}")


def test_forward_error_genomes_give_nan(neat):
    pop = _malformed_population(11, 240)
    d, rec = _check_transform(neat, pop, "malformed")
    x = W.normal_inputs(3, (240, 5, 3))
    y = neat.neat_forward(rec, 240, d, _dev(x)).cpu().numpy()
    ref = oracle.forward(pop.nodes, pop.conns, 3, 2, x)
    assert np.isnan(ref).any() and np.isfinite(ref).any()
    assert_outputs_close(y, ref, what="malformed")


def test_forward_is_independent_of_launch_shape(neat):
    """Bit-identical outputs whatever the group/tile/block shape."""
    for pop, B in [(W.ant_population(1, 300), 1), (W.ant_population(1, 300), 7),
                   (W.batched_populations(1, pop=40)[2], 64)]:
        d, rec = _check_transform(neat, pop, "shape")
        x = _dev(W.normal_inputs(4, (pop.pop, B, pop.num_inputs)))
        outs = []
        for group, tile, gpb, split in [(2, 1, 1, 1), (8, 1, 16, 2), (32, 1, 4, 4), (4, 1, 32, 1), (16, 1, 8, 4),
                                        (64, 1, 2, 2), (128, 1, 1, 1), (1, 1, 40, 1), (32, 32, 2, 1),
                                        (64, 8, 3, 1), (256, 32, 1, 1), (16, 16, 8, 1), (4, 4, 64, 1),
                                        (8, 8, 5, 1)]:
            if tile > 1 and B == 1:
                continue
            L = neat.Launch(group, tile, gpb, 0, split)
            smem = gpb * (neat.neat_record_stride(d) + 4 * pop.max_nodes * tile)
            if smem > 200 * 1024:
                continue                      # beyond the shared memory of one block
            outs.append(neat.neat_forward(rec, pop.pop, d, x, launch=L).cpu().numpy())
        assert len(outs) >= 4
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])
        ref = oracle.forward(pop.nodes, pop.conns, pop.num_inputs, pop.num_outputs, x.cpu().numpy())
        assert_outputs_close(outs[0], ref, what="shape")


def test_forward_edge_cases(neat):
    import torch
    pop = W.ant_population(2, 5)
    d, rec = _check_transform(neat, pop, "edge")
    # batch 0 and pop 0 are no-ops
    y = neat.neat_forward(rec, 5, d, torch.empty((5, 0, 27), device="cuda"))
    assert y.shape == (5, 0, 8)
    neat.neat_forward(rec, 0, d, torch.empty((0, 3, 27), device="cuda"))
    # a genome with no inputs at all, and one whose outputs have no incoming edges
    g0 = genome([(0, 0.5, 1, 0, 1), (1, -0.25, 2, 1, 2)], [None], 4, 2)
    pop0 = W.Population(*g0, 0, 2)
    d0, rec0 = _check_transform(neat, pop0, "no inputs")
    y = neat.neat_forward(rec0, 1, d0, torch.empty((1, 3, 0), device="cuda")).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop0.nodes, pop0.conns, 0, 2, np.zeros((1, 3, 0), np.float32)))
    # max_conns = 0: no connection rows at all (the empty tensor's pointer is NULL)
    ant = W.ant_population(3, 20)
    popc = W.Population(ant.nodes, np.zeros((20, 0, 4), np.float32), 27, 8)
    dc, recc = _check_transform(neat, popc, "no connection rows")
    x = W.normal_inputs(4, (20, 2, 27))
    y = neat.neat_forward(recc, 20, dc, _dev(x)).cpu().numpy()
    assert_outputs_close(y, oracle.forward(popc.nodes, popc.conns, 27, 8, x))


def test_steps_graph_matches_per_step_forward(neat):
    import torch
    pop = W.ant_population(5, 1000)
    d, rec = _check_transform(neat, pop, "steps")
    S = 12
    x = _dev(W.normal_inputs(5, (S, 1000, 1, 27)))
    y_graph = torch.empty((S, 1000, 1, 8), device="cuda")
    cache = neat.StepsCache()
    neat.neat_forward_steps(rec, 1000, d, x, y_graph, cache)
    neat.neat_forward_steps(rec, 1000, d, x, y_graph, cache)       # replay of the cached graph
    torch.cuda.synchronize()
    for s in range(S):
        y = neat.neat_forward(rec, 1000, d, x[s]).cpu().numpy()
        np.testing.assert_array_equal(y_graph[s].cpu().numpy(), y)
    cache.close()


def test_ant_full_size_sampled_steps(neat):
    """The bench workload: 10 000 genomes x 1000 steps in the CUDA graph, the
    launch shape bench.py times; sampled steps against the oracle."""
    import torch
    pop = W.ant_population(0, 10000)
    d, rec = _check_transform(neat, pop, "ant full")
    S = 1000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    x = torch.randn((S, 10000, 1, 27), device="cuda", generator=gen)
    y = torch.empty((S, 10000, 1, 8), device="cuda")
    cache = neat.StepsCache()
    L = neat.neat_default_launch(10000, d, 1)       # the batched launch bench.py times
    L.pdl = 1
    order = neat.neat_schedule(rec, 10000, d)
    L.order_dev = order.data_ptr()
    neat.neat_forward_steps(rec, 10000, d, x, y, cache, launch=L)
    torch.cuda.synchronize()
    worst = 0.0
    for s in (0, 1, 499, 998, 999):
        xs = x[s].cpu().numpy()
        ref = oracle.forward(pop.nodes, pop.conns, 27, 8, xs)
        bad, mabs, mscaled, n = compare_outputs(y[s].cpu().numpy(), ref)
        assert bad == 0, f"step {s}: {bad} bad, max scaled {mscaled}"
        worst = max(worst, mscaled)
    cache.close()
    print(f"ant full-size max scaled error {worst:.3g}")


def _assert_node_count_tiebreak(rec, pop, d, o):
    """Within a level count (up to 63), the order puts genomes with more
    non-input nodes (the nodes after the leading inputs, in 64 bins over
    max_nodes) first."""
    hdr = rec.view(pop, -1)[:, :16].cpu().numpy().view(np.uint32)
    n = (hdr[:, 0] & 0xFFFF).astype(np.int64)
    lv = np.minimum(hdr[:, 0] >> 16, 63).astype(np.int64)
    lead = np.minimum(hdr[:, 3] >> 16, n).astype(np.int64)
    shift = 0
    while (d.max_nodes >> shift) > 64:
        shift += 1
    nb = np.minimum((n - lead) >> shift, 63)
    key = lv * 64 + nb
    assert np.all(np.diff(key[o]) <= 0), "order is not (levels, non-input nodes) descending"


def test_schedule_order_is_a_permutation_and_changes_nothing(neat):
    import torch
    for pop, B in [(W.ant_population(8, 2000), 1), (W.batched_populations(8, pop=100)[3], 16)]:
        d, rec = _check_transform(neat, pop, "schedule")
        order = neat.neat_schedule(rec, pop.pop, d)
        torch.cuda.synchronize()
        o = order.cpu().numpy()
        assert sorted(o.tolist()) == list(range(pop.pop))
        dec = _decode(neat, rec, pop.pop, d)
        assert np.all(np.diff(dec.n_levels[o]) <= 0)            # deepest first
        _assert_node_count_tiebreak(rec, pop.pop, d, o)
        x = _dev(W.normal_inputs(9, (pop.pop, B, pop.num_inputs)))
        L0 = neat.neat_default_launch(pop.pop, d, B)
        y0 = neat.neat_forward(rec, pop.pop, d, x, launch=L0).cpu().numpy()
        L1 = neat.neat_default_launch(pop.pop, d, B)
        L1.order_dev = order.data_ptr()
        y1 = neat.neat_forward(rec, pop.pop, d, x, launch=L1).cpu().numpy()
        np.testing.assert_array_equal(y0, y1)
        if B == 1:
            S = 4
            xs = _dev(W.normal_inputs(10, (S, pop.pop, 1, pop.num_inputs)))
            ys = torch.empty((S, pop.pop, 1, pop.num_outputs), device="cuda")
            L1.pdl = 1
            cache = neat.StepsCache()
            neat.neat_forward_steps(rec, pop.pop, d, xs, ys, cache, launch=L1)
            torch.cuda.synchronize()
            for s in range(S):
                np.testing.assert_array_equal(ys[s].cpu().numpy(),
                                              neat.neat_forward(rec, pop.pop, d, xs[s].contiguous()).cpu().numpy())
            cache.close()


def test_node_tanh_error_bound(neat):
    """The nodes' tanh (1 - 2 / (exp(2z) + 1) on the hardware exponential and
    reciprocal) through the public path: one tanh node y = tanh(x), against
    numpy's double tanh; absolute error <= 5e-7, limits and NaN exact."""
    nodes, conns = genome([(0, 0, 1, 0, 0), (1, 0, 1, 0, 1)], [(0, 1, 1, 1.0)])
    x = np.concatenate([np.linspace(-12, 12, 200001), np.linspace(-1e-3, 1e-3, 2001), 10.0 ** np.arange(-30, 3),
                        -(10.0 ** np.arange(-30, 3)), [0.0, 40.0, -40.0, 1e30, -1e30, np.inf, -np.inf]])
    x = x.astype(np.float32)
    X = x.reshape(1, -1, 1)
    d = neat.dims(1, 1, 2, 1)
    rec, st = neat.neat_transform(_dev(nodes), _dev(conns), d)
    y = neat.neat_forward(rec, 1, d, _dev(X)).cpu().numpy().ravel()
    ref = np.tanh(x.astype(np.float64))
    assert np.max(np.abs(y - ref)) <= 5e-7
    assert (y[x >= 20] == 1.0).all() and (y[x <= -20] == -1.0).all()
    xn = np.array([[[np.nan]]], np.float32)
    assert np.isnan(neat.neat_forward(rec, 1, d, _dev(xn)).cpu().numpy()).all()
