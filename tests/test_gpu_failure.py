"""Failure detection without a GPU fault: a bounded on-device wait that
nothing satisfies gives up, reports through the device error word, and the
context keeps working."""
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.parity import assert_outputs_close

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    import time

    import torch
    from paper_2404_01817_gb300 import neat
    neat.neat_device_error(clear=True)
    t0 = time.perf_counter()
    r = neat.neat_selftest_bounded_wait(20000)          # 20 ms bound
    dt = time.perf_counter() - t0
    assert r == 2                                        # the wait gave up
    assert dt < 5.0
    assert neat.neat_device_error(clear=True) & 1
    assert neat.neat_device_error(clear=True) == 0       # cleared
    # the context is still usable: a normal transform + forward is correct
    pop = W.xor_population(3, 50)
    d = neat.dims(3, 1, 10, 20)
    rec, st = neat.neat_transform(torch.from_numpy(pop.nodes).cuda(), torch.from_numpy(pop.conns).cuda(), d)
    x = W.xor_inputs(50)
    y = neat.neat_forward(rec, 50, d, torch.from_numpy(x).cuda()).cpu().numpy()
    assert_outputs_close(y, oracle.forward(pop.nodes, pop.conns, 3, 1, x))


def test_argument_errors_are_reported_not_faulted():
    import torch
    from paper_2404_01817_gb300 import neat
    d = neat.dims(3, 1, 10, 20)
    bad = torch.zeros(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(neat.NeatError) as ei:
        neat.neat_forward(bad[1:], 1, d, torch.zeros((1, 1, 3), device="cuda"))   # misaligned records
    assert ei.value.code == neat.NEAT_EINVAL
    assert neat.neat_selftest_bounded_wait.__name__
    assert neat._lib.neat_selftest_bounded_wait(0, None) == neat.NEAT_EINVAL
