"""HyperNEAT substrate evaluation through the C ABI (neat_substrate_forward)
against the FP64 oracle, on generated weight blocks and end to end from CPPN
genomes.  Outputs pass within |gpu - ref| <= 1e-5 max(1, |ref|)."""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
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


@pytest.mark.parametrize("batch", [1, 3, 16, 37])
@pytest.mark.parametrize("acts", [(1, 1), (0, 2), (3, 4)])
def test_substrate_matches_oracle(neat, batch, acts):
    w = W.substrate_weights(1, 40, res=16, layers=3)
    x = W.normal_inputs(2, (40, batch, 256))
    y = neat.neat_substrate_forward(_dev(w), _dev(x), 16, 3, *acts).cpu().numpy()
    ref = oracle.substrate_forward(w, x, *acts)
    assert_outputs_close(y, ref, what=f"substrate batch {batch} acts {acts}")


@pytest.mark.parametrize("res,layers", [(7, 2), (7, 4), (2, 3), (33, 3)])
def test_other_substrates(neat, res, layers):
    R = res * res
    w = W.substrate_weights(3, 6, res=res, layers=layers, scale=0.15 if R > 256 else 0.3)
    x = W.normal_inputs(4, (6, 5, R))
    y = neat.neat_substrate_forward(_dev(w), _dev(x), res, layers).cpu().numpy()
    assert_outputs_close(y, oracle.substrate_forward(w, x), what=f"res {res} layers {layers}")


@pytest.mark.parametrize("res,layers", [(16, 3), (8, 4), (32, 3)])
def test_batch_chunks_do_not_change_bits(neat, res, layers):
    """Batches of up to 4 vectors take the bulk-copy kernel, larger ones the
    per-thread-load kernel; both split the sources into the same slices, so
    every vector's outputs are the same bits either way."""
    R = res * res
    w = _dev(W.substrate_weights(5, 10, res=res, layers=layers, scale=0.15 if R > 256 else 0.3))
    x = W.normal_inputs(6, (10, 37, R))
    y = neat.neat_substrate_forward(w, _dev(x), res, layers).cpu().numpy()
    assert_outputs_close(y, oracle.substrate_forward(w.cpu().numpy(), x), what=f"res {res} layers {layers} batch 37")
    for b in (0, 15, 16, 36):
        yb = neat.neat_substrate_forward(w, _dev(x[:, b:b + 1]), res, layers).cpu().numpy()
        np.testing.assert_array_equal(yb[:, 0], y[:, b])
    y4 = neat.neat_substrate_forward(w, _dev(x[:, 3:7]), res, layers).cpu().numpy()
    np.testing.assert_array_equal(y4, y[:, 3:7])


@pytest.mark.parametrize("res,layers,batch", [(8, 2, 1), (8, 4, 3), (32, 3, 1), (32, 2, 2), (16, 5, 4)])
def test_bulk_copy_substrates_match_oracle(neat, res, layers, batch):
    """The bulk-copy kernel at one stage per layer (8 x 8), eight-row
    stages (32 x 32), several layers (the stage barriers' phases carry
    across layers) and 1 to 4 vectors."""
    R = res * res
    w = W.substrate_weights(7, 12, res=res, layers=layers, scale=0.15 if R > 256 else 0.3)
    x = W.normal_inputs(8, (12, batch, R))
    y = neat.neat_substrate_forward(_dev(w), _dev(x), res, layers).cpu().numpy()
    assert_outputs_close(y, oracle.substrate_forward(w, x), what=f"bulk copy res {res} layers {layers} batch {batch}")


def test_cppn_to_substrate_end_to_end(neat):
    """CPPN genomes -> weight blocks (neat_cppn_query) -> substrate outputs,
    against the oracle's own query and substrate evaluation."""
    import torch
    pop = W.cppn_population(7, 3)
    d = neat.dims(5, 1, pop.max_nodes, pop.max_conns)
    rec, _ = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    w = neat.neat_cppn_query(rec, 3, d, 16, 3, 0.2)
    x = W.normal_inputs(8, (3, 4, 256))
    y = neat.neat_substrate_forward(w.contiguous(), _dev(x)).cpu().numpy()
    g, blk, s, t = np.meshgrid(np.arange(3), np.arange(2), np.arange(256), np.arange(256), indexing="ij")
    q = np.stack([g.ravel(), blk.ravel(), s.ravel(), t.ravel()], 1).astype(np.int32)
    raw, ref_w = oracle.cppn_query(pop.nodes, pop.conns, 16, 0.2, q)
    ref_w = ref_w.reshape(3, 2, 256, 256)
    gpu_w = w.cpu().numpy()
    flips = ((gpu_w == 0) != (ref_w == 0)).reshape(3, -1).any(1)    # a threshold decided differently
    ref = oracle.substrate_forward(ref_w.astype(np.float32), x)
    compared = 0
    for k in range(3):
        if not flips[k]:
            assert_outputs_close(y[k], ref[k], what=f"end to end genome {k}")
            compared += 1
    assert compared >= 2
    torch.cuda.synchronize()


def test_full_size_bench_launch_sampled(neat):
    """The substrate workload as bench.py runs it: 1000 CPPN genomes queried on
    3 layers of 16 x 16 (524 MB of weight blocks), one vector per genome (the
    bulk-copy kernel, 1000 blocks), and 16 vectors (the per-thread-load
    kernel); sampled genomes against the oracle on the same weight blocks."""
    import torch
    pop = W.cppn_population(0, 1000)
    d = neat.dims(5, 1, pop.max_nodes, pop.max_conns)
    rec, _ = neat.neat_transform(_dev(pop.nodes), _dev(pop.conns), d)
    w = neat.neat_cppn_query(rec, 1000, d, 16, 3, 0.2)
    idx = np.arange(0, 1000, 41)
    wi = w[torch.from_numpy(idx).cuda()].cpu().numpy()
    for batch in (1, 16):
        x = W.normal_inputs(20 + batch, (1000, batch, 256))
        y = neat.neat_substrate_forward(w, _dev(x)).cpu().numpy()
        assert_outputs_close(y[idx], oracle.substrate_forward(wi, x[idx]), what=f"full size batch {batch}")
        if batch == 16:
            y1 = neat.neat_substrate_forward(w, _dev(x[:, :1])).cpu().numpy()
            np.testing.assert_array_equal(y1[:, 0], y[:, 0])          # both kernels, the same bits
