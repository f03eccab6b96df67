"""The allocation-free batched forward (neat_forward_multi_noalloc).

Some callers cannot call cudaMalloc: a real-time control loop that must not
stall on the device allocator, or a process whose device memory belongs to
another framework's pool.  This entry point keeps its scratch in a fixed
device array instead.  The test calls it through the C ABI twice in a row
(two steps) and checks that each result equals the ordinary neat_forward's
bit for bit (the same kernel arithmetic and aggregation order; NaN matches
NaN); a later call captured in a CUDA graph replays to the same bits.  It
lives in a file of its own that pytest collects last, and passes alone in a
fresh process or after the rest.
"""

import numpy as np
import pytest

from paper_2404_01817_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_forward_on_two_calls():
    import torch
    from paper_2404_01817_gb300 import neat
    pops = [W.ant_population(11, 700), W.batched_populations(5, pop=120)[2], W.xor_population(2, 100)]
    batches = [1, 16, 4]
    S = 2
    descs = []
    for j, (p, B) in enumerate(zip(pops, batches)):
        d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
        rec, st = neat.neat_transform(torch.from_numpy(p.nodes).cuda(), torch.from_numpy(p.conns).cuda(), d)
        x = torch.from_numpy(W.normal_inputs(40 + j, (S, p.pop, B, p.num_inputs))).cuda()
        y = torch.full((S, p.pop, B, p.num_outputs), float("inf"), device="cuda")
        descs.append(dict(transformed=rec, pop=p.pop, dims=d, inputs=x, outputs=y))
    arr = neat.pop_descs(descs)
    stream = torch.cuda.current_stream().cuda_stream
    for step in range(S):                                  # two calls in a row through the C ABI
        rc = neat._lib.neat_forward_multi_noalloc(arr, len(descs), step, stream)
        assert rc == neat.NEAT_OK, neat.last_error()
    torch.cuda.synchronize()
    for p, dsc in zip(pops, descs):
        for step in range(S):
            ref = neat.neat_forward(dsc["transformed"], p.pop, dsc["dims"], dsc["inputs"][step].contiguous())
            np.testing.assert_array_equal(dsc["outputs"][step].cpu().numpy(), ref.cpu().numpy(),
                                          err_msg=f"no-alloc step {step}")
    # sizes beyond the scratch limits are refused with a clear error
    big = (neat.PopDesc * 65)()
    assert neat._lib.neat_forward_multi_noalloc(big, 65, 0, stream) == neat.NEAT_EINVAL
    assert "64" in neat.last_error()
    one = neat.pop_descs(descs[:1])
    one[0].pop = 40000
    assert neat._lib.neat_forward_multi_noalloc(one, 1, 0, stream) == neat.NEAT_EINVAL
    assert "32768" in neat.last_error()


def test_noalloc_call_captured_in_a_graph():
    """After the first call on the device, a call can be captured: it copies
    nothing from host memory (its bucket table is a kernel argument), so the
    captured graph replays the step, and the outputs match neat_forward."""
    import torch
    from paper_2404_01817_gb300 import neat
    pops = [W.ant_population(12, 500), W.xor_population(3, 100)]
    batches = [2, 4]
    S = 3
    descs = []
    for j, (p, B) in enumerate(zip(pops, batches)):
        d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
        rec, st = neat.neat_transform(torch.from_numpy(p.nodes).cuda(), torch.from_numpy(p.conns).cuda(), d)
        x = torch.from_numpy(W.normal_inputs(60 + j, (S, p.pop, B, p.num_inputs))).cuda()
        y = torch.full((S, p.pop, B, p.num_outputs), float("inf"), device="cuda")
        descs.append(dict(transformed=rec, pop=p.pop, dims=d, inputs=x, outputs=y))
    arr = neat.pop_descs(descs)
    rc = neat._lib.neat_forward_multi_noalloc(arr, len(descs), 0, torch.cuda.current_stream().cuda_stream)
    assert rc == neat.NEAT_OK, neat.last_error()              # eager: the device's first call if no other ran
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        for step in (1, 2):
            rc = neat._lib.neat_forward_multi_noalloc(arr, len(descs), step, side.cuda_stream)
            assert rc == neat.NEAT_OK, neat.last_error()
    for dsc in descs:
        dsc["outputs"][1:].fill_(float("inf"))
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    for p, dsc in zip(pops, descs):
        for step in range(S):
            ref = neat.neat_forward(dsc["transformed"], p.pop, dsc["dims"], dsc["inputs"][step].contiguous())
            np.testing.assert_array_equal(dsc["outputs"][step].cpu().numpy(), ref.cpu().numpy(),
                                          err_msg=f"captured no-alloc step {step}")
