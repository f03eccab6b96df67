"""The multi-rank (N > 1) path of the benchmark on CPU: two gloo ranks.

Each rank evaluates its own population (no collective in the data path);
only the timing is combined as the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_2404_01817_gb300 import shard
    from paper_2404_01817_gb300 import workloads as W
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = shard.rank_env()
    pop = W.ant_population(shard.population_seed(r), 20)
    x = W.normal_inputs(r, (20, 2, 27))
    y = oracle.forward(pop.nodes, pop.conns, 27, 8, x)      # this rank's shard of the work
    t = 1.0 + 0.5 * r                                        # a per-rank elapsed time
    slowest = shard.max_over_ranks(t)
    dist.barrier()
    out[r] = (r, lr, w, float(np.abs(pop.nodes[~np.isnan(pop.nodes)]).sum()), slowest,
              shard.job_throughput(20 * 2, w, slowest), float(np.nansum(y)))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_populations_and_combine_timing():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    (r0, lr0, w0, s0, slow0, thr0, y0), (r1, lr1, w1, s1, slow1, thr1, y1) = res[0], res[1]
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 != s1 and y0 != y1                             # distinct populations per rank
    assert slow0 == slow1 == pytest.approx(1.5)              # max over ranks
    assert thr0 == thr1 == pytest.approx(2 * 40 / 1.5)       # all ranks' units over the slowest time
