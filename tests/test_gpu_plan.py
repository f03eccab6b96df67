"""Batched multi-population plans (one persistent launch per step) against
the single-population forward and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.parity import assert_outputs_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def neat():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_01817_gb300 import neat as N
    return N


def _setup(neat, pops, batch, steps=None, seed=0):
    import torch
    out = []
    for j, p in enumerate(pops):
        d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
        rec, st = neat.neat_transform(torch.from_numpy(p.nodes).cuda(), torch.from_numpy(p.conns).cuda(), d)
        shape = (p.pop, batch, p.num_inputs) if steps is None else (steps, p.pop, batch, p.num_inputs)
        x = torch.from_numpy(W.normal_inputs(seed + j, shape)).cuda()
        y = torch.full(shape[:-1] + (p.num_outputs,), float("inf"), device="cuda")
        out.append(dict(transformed=rec, pop=p.pop, dims=d, inputs=x, outputs=y))
    return out


@pytest.mark.parametrize("size_buckets,autotune,block_threads",
                         [(True, False, 0), (False, False, 0), (True, True, 0), (True, False, 512),
                          (True, False, 1024), (False, True, 1024)])
def test_plan_matches_forward_batched_uneven(neat, size_buckets, autotune, block_threads):
    import torch
    pops = W.batched_populations(0, pop=160)
    descs = _setup(neat, pops, 64)
    plan = neat.Plan(descs, autotune=autotune, size_buckets=size_buckets, block_threads=block_threads)
    info = plan.describe()
    assert len(info["buckets"]) >= 4
    if block_threads:
        assert info["block_threads"] == block_threads
    assert all(b["G"] <= info["block_threads"] and b["G"] & (b["G"] - 1) == 0 for b in info["buckets"])
    plan.forward(0)
    torch.cuda.synchronize()
    for p, dsc in zip(pops, descs):
        ref = neat.neat_forward(dsc["transformed"], p.pop, dsc["dims"], dsc["inputs"]).cpu().numpy()
        np.testing.assert_array_equal(dsc["outputs"].cpu().numpy(), ref)
    # sampled against the oracle
    for p, dsc in zip(pops, descs):
        idx = np.arange(0, p.pop, 7)
        sub = p.subset(idx)
        x = dsc["inputs"].cpu().numpy()[idx]
        assert_outputs_close(dsc["outputs"].cpu().numpy()[idx],
                             oracle.forward(sub.nodes, sub.conns, sub.num_inputs, sub.num_outputs, x),
                             what=f"plan Nmax={p.max_nodes}")
    plan.close()


def test_plan_single_input_population(neat):
    import torch
    pops = [W.ant_population(3, 1500), W.xor_population(1, 100)]
    descs = _setup(neat, pops[:1], 1) + _setup(neat, pops[1:], 4)
    plan = neat.Plan(descs)
    plan.forward(0)
    torch.cuda.synchronize()
    for p, dsc in zip(pops, descs):
        ref = neat.neat_forward(dsc["transformed"], p.pop, dsc["dims"], dsc["inputs"]).cpu().numpy()
        np.testing.assert_array_equal(dsc["outputs"].cpu().numpy(), ref)
    plan.close()


def test_plan_steps_graph(neat):
    import torch
    pops = W.batched_populations(2, pop=64)[:3] + [W.ant_population(4, 500)]
    S = 6
    descs = _setup(neat, pops[:3], 16, steps=S) + _setup(neat, pops[3:], 1, steps=S)
    plan = neat.Plan(descs)
    plan.forward_steps(0, S)
    plan.forward_steps(0, S)          # replay
    torch.cuda.synchronize()
    graph_out = [d["outputs"].clone() for d in descs]
    for d in descs:
        d["outputs"].fill_(float("inf"))
    for s in range(S):
        plan.forward(s)
    torch.cuda.synchronize()
    for a, d in zip(graph_out, descs):
        np.testing.assert_array_equal(a.cpu().numpy(), d["outputs"].cpu().numpy())
    for p, d in zip(pops, descs):
        for s in (0, S - 1):
            ref = neat.neat_forward(d["transformed"], p.pop, d["dims"], d["inputs"][s].contiguous()).cpu().numpy()
            np.testing.assert_array_equal(d["outputs"][s].cpu().numpy(), ref)
    assert neat.neat_device_error() == 0
    plan.close()


def test_plan_full_size_uneven_batch_sampled(neat):
    """The uneven-batch workload at full size (4 x 2048 genomes, 64 inputs
    each) through the autotuned plan bench.py times; sampled genomes against
    the oracle."""
    import torch
    pops = W.batched_populations(0, pop=2048)
    descs = _setup(neat, pops, 64, seed=77)
    plan = neat.Plan(descs, autotune=True)
    plan.forward(0)
    torch.cuda.synchronize()
    desc = plan.describe()
    assert desc["block_threads"] in (256, 512, 1024)                  # tuned, the block size too
    assert {"block_threads": desc["block_threads"]}.items() <= desc["autotune"][-1].items()
    assert all(b["G"] <= desc["block_threads"] for b in desc["buckets"])
    worst = 0.0
    for j, (p, dsc) in enumerate(zip(pops, descs)):
        idx = np.random.default_rng(j).choice(p.pop, 48, replace=False)
        sub = p.subset(idx)
        x = dsc["inputs"].cpu().numpy()[idx]
        ref = oracle.forward(sub.nodes, sub.conns, sub.num_inputs, sub.num_outputs, x)
        mabs, mscaled = assert_outputs_close(dsc["outputs"].cpu().numpy()[idx], ref, what=f"full Nmax={p.max_nodes}")
        worst = max(worst, mscaled)
    print(f"uneven batch full-size max scaled error {worst:.3g}")
    plan.close()
