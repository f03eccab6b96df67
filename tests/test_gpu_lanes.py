"""Lane programs (neat_lanes_pack / neat_forward_lanes[_steps]) through the C ABI.

Outputs must be bit-identical to neat_forward with one input vector per
genome (same node rule and aggregation order; the padding edges of a lane
program change no bit of any partial), and within the float tolerance of
the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome, stack
from tests.parity import assert_outputs_close, compare_outputs

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


def _prepare(neat, pop):
    d = neat.dims(pop.num_inputs, pop.num_outputs, pop.max_nodes, pop.max_conns)
    rec, st = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    lanes = neat.neat_lanes_pack(rec, pop.pop, d)
    return d, rec, lanes


def _check_one_step(neat, pop, seed, what, stage_bytes=0):
    d, rec, lanes = _prepare(neat, pop)
    x = W.normal_inputs(seed, (pop.pop, 1, pop.num_inputs))
    xd = _dev(x)
    y_lanes = neat.neat_forward_lanes(lanes, pop.pop, d, xd, stage_bytes=stage_bytes).cpu().numpy()
    y_plain = neat.neat_forward(rec, pop.pop, d, xd).cpu().numpy()
    np.testing.assert_array_equal(y_lanes, y_plain, err_msg=f"{what}: lanes vs neat_forward")
    ref = oracle.forward(pop.nodes, pop.conns, pop.num_inputs, pop.num_outputs, x)
    mabs, mscaled = assert_outputs_close(y_lanes, ref, what=what)
    print(f"{what}: max abs {mabs:.3g}, max scaled {mscaled:.3g}")
    return d, rec, lanes


def test_lanes_ant_partial_warp(neat):
    """997 Ant genomes (the last warp holds 5 of its 16): bit-equal to neat_forward, oracle parity."""
    d, rec, lanes = _check_one_step(neat, W.ant_population(0, 997), 1, "ant 997")
    info = neat.neat_lanes_query(lanes)
    assert info.pop == 997 and info.warps == (997 + 15) // 16 and info.unordered == 0
    assert 0 < info.max_warp_bytes <= info.warp_stride


def test_lanes_xor(neat):
    _check_one_step(neat, W.xor_population(0, 100), 2, "xor")


@pytest.mark.parametrize("bucket", [0, 1])
def test_lanes_every_aggregation_and_activation(neat, bucket):
    """Mixed activations and aggregations (all 7 x 4) at Nmax 16 and 64: the
    general walk and the per-aggregation padding edges."""
    pop = W.batched_populations(3, pop=200)[bucket]
    _check_one_step(neat, pop, 3 + bucket, f"mixed Nmax={pop.max_nodes}")


def test_lanes_nmax_128_dense(neat):
    """The largest genomes lane programs take: Nmax 128, many edges per node."""
    pop = W.random_dag_population(5, 70, 8, 4, 128, 1024, hidden=lambda r: int(r.integers(60, 116)),
                                  edges=lambda r, n: int(r.integers(4 * n, 8 * n)), acts=W.ALL_ACTS,
                                  aggs=W.ALL_AGGS)
    _check_one_step(neat, pop, 5, "Nmax 128")


def test_lanes_program_from_device_memory(neat):
    """stage_bytes smaller than every warp program: the programs are read from
    device memory instead of shared memory, with the same bits."""
    pop = W.ant_population(4, 300)
    d, rec, lanes = _check_one_step(neat, pop, 6, "ant 300 staged")
    x = _dev(W.normal_inputs(6, (300, 1, 27)))
    y_staged = neat.neat_forward_lanes(lanes, 300, d, x).cpu().numpy()
    y_global = neat.neat_forward_lanes(lanes, 300, d, x, stage_bytes=16).cpu().numpy()
    np.testing.assert_array_equal(y_staged, y_global)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_lanes_inputs_not_16_byte_aligned(neat, shift):
    """Inputs and outputs that start 4, 8 or 12 bytes past a 16-byte
    boundary: the input chunks that cover the first and last rows reach
    outside the array and are read word by word, the outputs are stored word
    by word; the outputs keep their bits."""
    import torch
    pop = W.ant_population(6, 203)
    d, rec, lanes = _prepare(neat, pop)
    x = W.normal_inputs(9, (203, 27))
    buf = torch.zeros(203 * 27 + 8, device="cuda")
    view = buf[shift:shift + 203 * 27].view(203, 27)
    view.copy_(_dev(x))
    assert view.data_ptr() % 16 == 4 * shift
    y = neat.neat_forward_lanes(lanes, 203, d, view).cpu().numpy()
    ybuf = torch.full((203 * 8 + 4,), float("inf"), device="cuda")
    yview = ybuf[shift:shift + 203 * 8].view(203, 8)
    neat.neat_forward_lanes(lanes, 203, d, view, outputs=yview)
    np.testing.assert_array_equal(yview.cpu().numpy(), y)
    assert np.isinf(ybuf[:shift].cpu().numpy()).all() and np.isinf(ybuf[shift + 203 * 8:].cpu().numpy()).all()
    y_plain = neat.neat_forward(rec, 203, d, _dev(x[:, None, :])).cpu().numpy().reshape(203, 8)
    np.testing.assert_array_equal(y, y_plain)
    for i in (0, 202):                         # the array's first and last rows
        ref = oracle.forward(pop.nodes[i:i + 1], pop.conns[i:i + 1], 27, 8, x[i:i + 1, None, :])
        assert_outputs_close(y[i:i + 1], ref[:, 0], what=f"row {i}")


def _malformed(seed, n):
    """Small genomes, every fourth with a planted error (cycle, duplicate key,
    missing output), the rest valid with warnings (dangling, into-input)."""
    base = W.random_dag_population(seed, n, 3, 2, 16, 48, hidden=lambda r: int(r.integers(0, 10)),
                                   edges=lambda r, k: int(r.integers(k, 3 * k)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.2)
    rng = np.random.default_rng(seed)
    nodes, conns = base.nodes.copy(), base.conns.copy()
    for g in range(n):
        nv = np.nonzero(~np.isnan(nodes[g, :, 0]))[0]
        cv = np.nonzero(~np.isnan(conns[g, :, 0]))[0]
        free_c = np.nonzero(np.isnan(conns[g, :, 0]))[0]
        kind = g % 8
        if kind == 0 and len(cv) and free_c.size:
            c = cv[rng.integers(len(cv))]
            conns[g, free_c[0]] = (conns[g, c, 1], conns[g, c, 0], 1, 0.5)
            conns[g, c, 2] = 1
        elif kind == 2:
            nodes[g, nv[-1], 0] = nodes[g, nv[-2], 0]
        elif kind == 4:
            nodes[g, nv[nodes[g, nv, 0] == 3], :] = np.nan
        elif kind == 5 and free_c.size:
            conns[g, free_c[0]] = (1, 999, 1, 1.0)
        elif kind == 6 and free_c.size:
            conns[g, free_c[0]] = (4, 0, 1, 1.0)
        elif kind == 7:
            nodes[g] = nodes[g][rng.permutation(16)]
            conns[g] = conns[g][rng.permutation(48)]
    return W.Population(nodes, conns, 3, 2)


def test_lanes_error_genomes_give_nan(neat):
    pop = _malformed(12, 160)
    d, rec, lanes = _prepare(neat, pop)
    x = W.normal_inputs(7, (160, 1, 3))
    y = neat.neat_forward_lanes(lanes, 160, d, _dev(x)).cpu().numpy()
    ref = oracle.forward(pop.nodes, pop.conns, 3, 2, x)
    assert np.isnan(ref).any() and np.isfinite(ref).any()
    assert_outputs_close(y, ref, what="malformed")
    np.testing.assert_array_equal(y, neat.neat_forward(rec, 160, d, _dev(x)).cpu().numpy())


def test_lanes_cyclic_records_give_nan(neat):
    """Records of neat_transform_recurrent with a cycle have no feedforward
    schedule: NaN outputs, counted as unordered; acyclic genomes beside them
    are unaffected."""
    cyc = genome([(0, 0, 1, 0, 0), (1, 0.1, 1, 0, 1), (2, 0.2, 1, 0, 1)],
                 [(0, 2, 1, 0.5), (2, 1, 1, 0.7), (1, 2, 1, -0.3)], 3, 3)
    dag = genome([(0, 0, 1, 0, 0), (1, 0.1, 1, 0, 1), (2, 0.2, 1, 0, 1)],
                 [(0, 2, 1, 0.5), (2, 1, 1, 0.7), None], 3, 3)
    nodes, conns = stack([cyc, dag, cyc])
    d = neat.dims(1, 1, 3, 3)
    rec, st = neat.neat_transform_recurrent(_dev(nodes), _dev(conns), d)
    lanes = neat.neat_lanes_pack(rec, 3, d)
    x = np.array([[[0.3]], [[0.3]], [[-1.0]]], np.float32)
    y = neat.neat_forward_lanes(lanes, 3, d, _dev(x)).cpu().numpy().ravel()
    info = neat.neat_lanes_query(lanes)
    assert info.unordered == 2
    assert np.isnan(y[0]) and np.isnan(y[2]) and np.isfinite(y[1])
    ref = oracle.forward(nodes[1:2], conns[1:2], 1, 1, x[1:2])
    assert_outputs_close(y[1:2], ref.ravel())


def test_lanes_edge_cases(neat):
    import torch
    pop = W.ant_population(2, 5)
    d, rec, lanes = _prepare(neat, pop)
    neat.neat_forward_lanes(lanes, 0, d, torch.empty((0, 27), device="cuda"))
    y = neat.neat_forward_lanes(lanes, 5, d, _dev(W.normal_inputs(8, (5, 27)))).cpu().numpy()
    assert y.shape == (5, 8) and np.isfinite(y).all()
    # no inputs at all; outputs without incoming edges (act(bias))
    g0 = genome([(0, 0.5, 1, 0, 1), (1, -0.25, 2, 1, 2)], [None], 4, 2)
    pop0 = W.Population(*g0, 0, 2)
    d0, rec0, lanes0 = _prepare(neat, pop0)
    y0 = neat.neat_forward_lanes(lanes0, 1, d0, torch.empty((1, 0), device="cuda")).cpu().numpy()
    assert_outputs_close(y0, oracle.forward(pop0.nodes, pop0.conns, 0, 2, np.zeros((1, 1, 0), np.float32))[:, 0])
    # no connection rows at all (max_conns = 0, the empty tensor's pointer is NULL)
    ant = W.ant_population(3, 40)
    popc = W.Population(ant.nodes, np.zeros((40, 0, 4), np.float32), 27, 8)
    dc, recc, lanesc = _prepare(neat, popc)
    xc = W.normal_inputs(4, (40, 27))
    yc = neat.neat_forward_lanes(lanesc, 40, dc, _dev(xc)).cpu().numpy()
    assert_outputs_close(yc, oracle.forward(popc.nodes, popc.conns, 27, 8, xc[:, None, :])[:, 0])
    # an empty population packs and runs
    dz = neat.dims(27, 8, 50, 200)
    lz = torch.empty(max(neat.neat_lanes_bytes(0, dz), 256), dtype=torch.uint8, device="cuda")
    neat.neat_lanes_pack(rec, 0, dz, lanes=lz)
    assert neat.neat_lanes_query(lz).warps == 0


def test_lanes_repack_is_deterministic(neat):
    pop = W.ant_population(9, 2000)
    d, rec, lanes = _prepare(neat, pop)
    a = neat.neat_lanes_query(lanes)
    neat.neat_lanes_pack(rec, 2000, d, lanes=lanes)
    b = neat.neat_lanes_query(lanes)
    assert a.max_warp_bytes == b.max_warp_bytes and a.warps == b.warps


def test_lanes_steps_graph_matches_per_step(neat):
    import torch
    pop = W.ant_population(5, 1000)
    d, rec, lanes = _prepare(neat, pop)
    S = 12
    x = _dev(W.normal_inputs(5, (S, 1000, 1, 27)))
    y = torch.empty((S, 1000, 1, 8), device="cuda")
    cache = neat.LanesCache()
    neat.neat_forward_lanes_steps(lanes, 1000, d, x, y, cache)
    neat.neat_forward_lanes_steps(lanes, 1000, d, x, y, cache)        # replay of the cached graph
    torch.cuda.synchronize()
    for s in range(S):
        np.testing.assert_array_equal(y[s].cpu().numpy(), neat.neat_forward(rec, 1000, d, x[s]).cpu().numpy())
    cache.close()


def test_lanes_tune_picks_a_staging_capacity(neat):
    """neat_lanes_tune returns a stage_bytes that stages every program; the
    graph at that capacity gives the same bits."""
    import torch
    pop = W.ant_population(7, 3000)
    d, rec, lanes = _prepare(neat, pop)
    info = neat.neat_lanes_query(lanes)
    S = 16
    x = _dev(W.normal_inputs(10, (S, 3000, 1, 27)))
    y = torch.empty((S, 3000, 1, 8), device="cuda")
    sb = neat.neat_lanes_tune(lanes, 3000, d, x, y)
    assert sb % 16 == 0 and info.max_warp_bytes <= sb <= info.warp_stride
    y2 = torch.empty_like(y)
    cache = neat.LanesCache()
    neat.neat_forward_lanes_steps(lanes, 3000, d, x, y2, cache, stage_bytes=sb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y2.cpu().numpy(), y.cpu().numpy())
    np.testing.assert_array_equal(y2[S - 1].cpu().numpy(), neat.neat_forward(rec, 3000, d, x[S - 1]).cpu().numpy())
    cache.close()


def test_lanes_full_size_sampled_steps(neat):
    """The bench workload and launch: 10 000 Ant genomes x 1000 steps in the
    lane-program graph, stage_bytes from the pack; sampled steps against the
    oracle and against neat_forward."""
    import torch
    pop = W.ant_population(0, 10000)
    d, rec, lanes = _prepare(neat, pop)
    info = neat.neat_lanes_query(lanes)
    S = 1000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    x = torch.randn((S, 10000, 1, 27), device="cuda", generator=gen)
    y = torch.empty((S, 10000, 1, 8), device="cuda")
    cache = neat.LanesCache()
    neat.neat_forward_lanes_steps(lanes, 10000, d, x, y, cache, stage_bytes=info.max_warp_bytes)
    torch.cuda.synchronize()
    worst = 0.0
    for s in (0, 1, 499, 998, 999):
        xs = x[s].cpu().numpy()
        ref = oracle.forward(pop.nodes, pop.conns, 27, 8, xs)
        bad, mabs, mscaled, n = compare_outputs(y[s].cpu().numpy(), ref)
        assert bad == 0, f"step {s}: {bad} bad, max scaled {mscaled}"
        worst = max(worst, mscaled)
    np.testing.assert_array_equal(y[999].cpu().numpy(), neat.neat_forward(rec, 10000, d, x[999]).cpu().numpy())
    cache.close()
    print(f"lanes ant full-size max scaled error {worst:.3g}")
