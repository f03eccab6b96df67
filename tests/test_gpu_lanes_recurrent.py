"""Recurrent lane programs (neat_lanes_pack_recurrent /
neat_forward_lanes_recurrent) through the C ABI.

Outputs must be bit-identical to neat_forward_recurrent with one input
vector per genome: the same node rule and aggregation order, the same
synchronous iteration (every non-input node from the previous iteration's
values, non-input nodes starting at 0), and padding edges that change no bit
of any partial.  neat_forward_recurrent is itself checked against the FP64
oracle in test_gpu_recurrent.py; one case here is checked against the oracle
directly as well.
"""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.parity import TOL

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
    rec, st = neat.neat_transform_recurrent(_dev(pop.nodes), _dev(pop.conns), d)
    lanes = neat.neat_lanes_pack_recurrent(rec, pop.pop, d)
    return d, rec, st, lanes


def _both(neat, pop, d, rec, lanes, x, K, **kw):
    xd = _dev(x)
    y_lanes = neat.neat_forward_lanes_recurrent(lanes, pop.pop, d, xd, K, **kw).cpu().numpy()
    y_plain = neat.neat_forward_recurrent(rec, pop.pop, d, xd.view(pop.pop, 1, pop.num_inputs), K)
    return y_lanes, y_plain.view(pop.pop, pop.num_outputs).cpu().numpy()


def test_recurrent_lanes_ant_bit_equal(neat):
    """3000 Ant-shaped recurrent genomes (the last warp partly filled), K = 0,
    1, 2, 8 and 9 iterations (both tile parities at the end)."""
    pop = W.ant_recurrent_population(5, 3000)
    d, rec, st, lanes = _prepare(neat, pop)
    info = neat.neat_lanes_query(lanes)
    assert info.recurrent == 1 and info.pop == 3000 and info.warps == (3000 + 15) // 16 and info.unordered == 0
    x = W.normal_inputs(6, (3000, 27))
    for K in (0, 1, 2, 8, 9):
        y_lanes, y_plain = _both(neat, pop, d, rec, lanes, x, K)
        np.testing.assert_array_equal(y_lanes, y_plain, err_msg=f"K={K}")
        if K == 0:
            assert np.all(y_lanes == 0.0)                # outputs start at 0
        else:
            assert np.isfinite(y_lanes).all()


def test_recurrent_lanes_against_the_oracle(neat):
    """Every 7th of 700 Ant-shaped recurrent genomes after 4 iterations,
    against the FP64 oracle at the float tolerance."""
    pop = W.ant_recurrent_population(8, 700)
    d, rec, st, lanes = _prepare(neat, pop)
    x = W.normal_inputs(9, (700, 27))
    y = neat.neat_forward_lanes_recurrent(lanes, 700, d, _dev(x), 4).cpu().numpy()
    idx = np.arange(0, 700, 7)
    sub = pop.subset(idx)
    ref, ref_st = oracle.forward_recurrent(sub.nodes, sub.conns, 27, 8, x[idx].reshape(idx.size, 1, 27), 4)
    ref = ref.reshape(idx.size, 8)
    err = np.abs(y[idx].astype(np.float64) - ref) / np.maximum(1.0, np.abs(ref))
    print(f"recurrent lanes vs oracle (K = 4): max scaled error {err.max():.3g}")
    assert err.max() <= TOL


@pytest.mark.parametrize("K", [1, 3, 5])
def test_recurrent_lanes_all_activations_and_aggregations(neat, K):
    """Every activation and aggregation (the general walk, not the sum + tanh
    path); the program staged in shared memory and read from device memory;
    with and without programmatic dependent launch."""
    pop = W.random_recurrent_population(40 + K, 211, 4, 3, 40, 160, hidden=lambda r: int(r.integers(0, 26)),
                                        edges=lambda r, n: int(r.integers(n, 4 * n + 1)), acts=W.ALL_ACTS,
                                        aggs=W.ALL_AGGS, p_disabled=0.1)
    d, rec, st, lanes = _prepare(neat, pop)
    x = W.normal_inputs(50 + K, (211, 4))
    y_plain = None
    for kw in ({}, {"stage_bytes": 16}, {"pdl": True}):
        y_lanes, y_plain = _both(neat, pop, d, rec, lanes, x, K, **kw)
        np.testing.assert_array_equal(y_lanes, y_plain, err_msg=f"K={K} {kw}")


def test_recurrent_lanes_large_genomes(neat):
    """max_nodes 128 with up to 100 hidden nodes and 1024 connections: long
    beats (more than 8 quads in a lane) and long programs, sum + tanh and
    mixed activations."""
    for acts in ((W.ACT_TANH,), (W.ACT_TANH, W.ACT_SIGMOID, W.ACT_SIN, W.ACT_GAUSS)):
        pop = W.random_recurrent_population(60, 64, 8, 4, 128, 1024, hidden=lambda r: int(r.integers(60, 101)),
                                            edges=lambda r, n: int(r.integers(4 * n, 8 * n + 1)), acts=acts,
                                            aggs=(W.AGG_SUM,), p_disabled=0.1)
        d, rec, st, lanes = _prepare(neat, pop)
        x = W.normal_inputs(61, (64, 8))
        y_lanes, y_plain = _both(neat, pop, d, rec, lanes, x, 3)
        np.testing.assert_array_equal(y_lanes, y_plain, err_msg=f"acts={acts}")


def test_recurrent_lanes_errors_and_mismatched_buffers(neat):
    """A genome with an error bit gets NaN outputs (the others are
    unchanged); a buffer packed for the other forward gives NaN everywhere;
    negative iteration counts are refused."""
    pop = W.ant_recurrent_population(70, 40)
    pop.nodes[3, 40, 0] = pop.nodes[3, 0, 0]             # a duplicated key: an error genome
    d, rec, st, lanes = _prepare(neat, pop)
    assert st.cpu().numpy()[3] & 0xFF
    x = W.normal_inputs(71, (40, 27))
    y_lanes, y_plain = _both(neat, pop, d, rec, lanes, x, 2)
    assert np.isnan(y_lanes[3]).all()
    np.testing.assert_array_equal(y_lanes, y_plain)
    ff = W.ant_population(72, 40)
    rec_ff, _ = neat.neat_transform(_dev(ff.nodes), _dev(ff.conns), d)
    lanes_ff = neat.neat_lanes_pack(rec_ff, 40, d)
    assert np.isnan(neat.neat_forward_lanes_recurrent(lanes_ff, 40, d, _dev(x), 2).cpu().numpy()).all()
    assert np.isnan(neat.neat_forward_lanes(lanes, 40, d, _dev(x)).cpu().numpy()).all()
    with pytest.raises(neat.NeatError):
        neat.neat_forward_lanes_recurrent(lanes, 40, d, _dev(x), -1)
