"""Fused multi-step forward (neat_forward_fused): bit-identical to per-step
forwards with the same records, and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome, stack
from tests.parity import assert_outputs_close

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


def test_fused_equals_graph_steps_on_the_ant_population(neat):
    import torch
    pop = W.ant_population(0, 10000)
    d = neat.dims(27, 8, 50, 200)
    rec, _ = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    order = neat.neat_schedule(rec, 10000, d)
    S = 12
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    x = torch.randn((S, 10000, 1, 27), device="cuda", generator=g)
    y_graph = torch.empty((S, 10000, 1, 8), device="cuda")
    L = neat.neat_default_launch(10000, d, 1)
    L.pdl = 1
    L.order_dev = order.data_ptr()
    cache = neat.StepsCache()
    neat.neat_forward_steps(rec, 10000, d, x, y_graph, cache, launch=L)
    y_fused = neat.neat_forward_fused(rec, 10000, d, x, torch.empty_like(y_graph), launch=L)
    assert torch.equal(y_fused, y_graph)
    y_default = neat.neat_forward_fused(rec, 10000, d, x, torch.empty_like(y_graph))
    assert torch.equal(y_default, y_graph)
    idx = np.arange(0, 10000, 97)
    sub = pop.subset(idx)
    ref = oracle.forward(sub.nodes, sub.conns, 27, 8, x[S - 1, idx].cpu().numpy())
    assert_outputs_close(y_fused[S - 1, idx].cpu().numpy(), ref, what="fused last step")


@pytest.mark.parametrize("batch", [1, 5, 40])
def test_fused_tiles_and_mixed_genomes(neat, batch):
    import torch
    pop = W.random_dag_population(3, 150, 4, 3, 40, 120, hidden=lambda r: int(r.integers(0, 30)),
                                  edges=lambda r, n: int(r.integers(n, 3 * n)), acts=W.ALL_ACTS, aggs=W.ALL_AGGS,
                                  p_disabled=0.2)
    d = neat.dims(4, 3, 40, 120)
    rec, _ = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    S = 4
    x = _dev(W.normal_inputs(5, (S, 150, batch, 4)))
    y = neat.neat_forward_fused(rec, 150, d, x, torch.empty((S, 150, batch, 3), device="cuda"))
    for s in range(S):
        ys = neat.neat_forward(rec, 150, d, x[s].contiguous())
        assert torch.equal(y[s], ys)


def test_fused_invalid_genomes_and_arguments(neat):
    import torch
    ok = genome([(0, 0, 1, 0, 0), (1, 0.5, 1, 0, 1)], [(0, 1, 1, 2.0)])
    cyc = genome([(0, 0, 1, 0, 0), (1, 0.5, 1, 0, 1)], [(1, 1, 1, 2.0)])
    nodes, conns = stack([ok, cyc])
    d = neat.dims(1, 1, 2, 1)
    rec, st = neat.neat_transform(_dev(nodes), _dev(conns), d)
    x = torch.ones((3, 2, 1, 1), device="cuda")
    y = neat.neat_forward_fused(rec, 2, d, x, torch.empty((3, 2, 1, 1), device="cuda")).cpu().numpy()
    assert np.isfinite(y[:, 0]).all() and np.isnan(y[:, 1]).all()
    assert np.allclose(y[:, 0], np.tanh(0.5 + 2.0))
    with pytest.raises(neat.NeatError):
        neat._check(neat._lib.neat_forward_fused(neat._ptr(rec), 2, d, neat._ptr(x), 1, 1, neat._ptr(x), 2, 3, None,
                                                 None), "neat_forward_fused")
