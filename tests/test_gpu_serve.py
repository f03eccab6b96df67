"""Serving: continuous batching under an HBM budget (neat_serve_*)."""
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


def _request(seed, pop, nmax, batch):
    req = dict(id=seed, pop=pop, max_nodes=nmax, max_conns=4 * nmax, num_inputs=min(27, nmax // 2),
               num_outputs=min(8, max(1, nmax // 4)), batch=batch, steps=5, seed=1000 + seed)
    return req, W.request_population(req)


def _direct(neat, p, batch, steps, seed):
    """The same evaluation without the server: transform, observations from
    the serving generator, neat_forward per step."""
    import torch
    d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
    rec, st = neat.neat_transform(torch.from_numpy(p.nodes).cuda(), torch.from_numpy(p.conns).cuda(), d)
    outs, obs = [], []
    for s in range(steps):
        x = torch.empty((p.pop, batch, p.num_inputs), device="cuda")
        neat.neat_fill_normal(seed, s, x)
        outs.append(neat.neat_forward(rec, p.pop, d, x).cpu().numpy())
        obs.append(x.cpu().numpy())
    return np.stack(outs), np.stack(obs)


def _submit(neat, srv, req, p):
    import torch
    d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
    y = torch.full((req["steps"], p.pop, req["batch"], p.num_outputs), float("inf"), device="cuda")
    t = srv.submit(p.nodes, p.conns, d, req["batch"], req["steps"], req["seed"], y,
                   out_step_stride=p.pop * req["batch"] * p.num_outputs)
    return t, y


def test_serve_matches_direct_and_oracle(neat):
    srv = neat.Server(1 << 30)
    req, p = _request(1, 300, 64, 8)
    t, y = _submit(neat, srv, req, p)
    code, res = srv.wait(t, 60000)
    assert code == neat.NEAT_OK and res.status == neat.NEAT_OK
    assert res.genome_forwards == 300 * 8 * 5
    direct, obs = _direct(neat, p, 8, 5, req["seed"])
    np.testing.assert_array_equal(y.cpu().numpy(), direct)
    # sampled genomes against the FP64 oracle, on the generated observations
    idx = np.arange(0, 300, 11)
    sub = p.subset(idx)
    for s in (0, 4):
        ref = oracle.forward(sub.nodes, sub.conns, sub.num_inputs, sub.num_outputs, obs[s][idx])
        assert_outputs_close(y[s].cpu().numpy()[idx], ref, what=f"serve step {s}")
    x = obs[0].ravel()
    assert abs(float(x.mean())) < 0.05 and abs(float(x.std()) - 1.0) < 0.05     # N(0,1)
    srv.close()


def test_serve_alone_equals_mixed(neat):
    """A request's outputs are bit-identical alone and among other requests
    whose work is on the device at the same time (their admit..done
    intervals overlap the request's)."""
    req, p = _request(2, 257, 50, 3)
    srv = neat.Server(1 << 30)
    t, y_alone = _submit(neat, srv, req, p)
    assert srv.wait(t)[0] == neat.NEAT_OK
    srv.close()
    srv = neat.Server(1 << 30, max_active=16)
    others = [_request(10 + k, 64 + 97 * k, [8, 30, 120, 300, 16][k % 5], [1, 5, 17, 2, 64][k % 5]) for k in range(8)]
    others = [(dict(r, steps=50), q) for r, q in others]       # long enough to run beside the request
    tickets = [_submit(neat, srv, r, q) for r, q in others[:4]]
    t, y_mixed = _submit(neat, srv, req, p)
    tickets += [_submit(neat, srv, r, q) for r, q in others[4:]]
    code, res = srv.wait(t)
    assert code == neat.NEAT_OK
    spans = []
    for tk, _ in tickets:
        c, r = srv.wait(tk)
        assert c == neat.NEAT_OK
        spans.append((r.admit_ms, r.done_ms))
    overlapping = sum(1 for a, b in spans if a < res.done_ms and b > res.admit_ms)
    assert overlapping >= 2, f"only {overlapping} requests were active beside the request"
    np.testing.assert_array_equal(y_alone.cpu().numpy(), y_mixed.cpu().numpy())
    for (r, q), (tk, y) in zip(others, tickets):
        direct, _ = _direct(neat, q, r["batch"], r["steps"], r["seed"])
        np.testing.assert_array_equal(y.cpu().numpy(), direct)
    st = srv.stats()
    assert st.completed == 9 and st.latency_p99_ms >= st.latency_p50_ms > 0 and st.genome_forwards_per_s > 0
    srv.close()


def test_serve_budget_queueing_cancel_and_timeouts(neat):
    req, p = _request(3, 400, 128, 4)
    srv = neat.Server(10 << 20, max_active=8)        # one request (~7 MB) fits, two do not
    # a request that can never fit is refused at submit
    big_req, big = _request(4, 4096, 512, 8)
    with pytest.raises(neat.NeatError) as ei:
        _submit(neat, srv, big_req, big)
    assert ei.value.code == neat.NEAT_EBUDGET
    # two requests that do not fit together: the second is admitted after the first is done
    t1, y1 = _submit(neat, srv, req, p)
    t2, y2 = _submit(neat, srv, req, p)
    t3, y3 = _submit(neat, srv, req, p)
    srv.cancel(t3)
    c1, r1 = srv.wait(t1)
    c2, r2 = srv.wait(t2)
    c3, r3 = srv.wait(t3)
    assert c1 == neat.NEAT_OK and c2 == neat.NEAT_OK
    assert r2.admit_ms >= r1.done_ms - 1e-6
    assert c3 == neat.NEAT_ECANCELLED
    np.testing.assert_array_equal(y1.cpu().numpy(), y2.cpu().numpy())
    # a bounded host wait on a request that cannot be done yet (20 000 steps,
    # each at least one kernel launch) expires with NEAT_ETIMEOUT; cancelling
    # it then stops it
    import torch
    d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
    y4 = torch.empty((p.pop, req["batch"], p.num_outputs), device="cuda")     # every step overwrites it
    t4 = srv.submit(p.nodes, p.conns, d, req["batch"], 20000, req["seed"], y4)
    code, _ = srv.wait(t4, 1)
    assert code == neat.NEAT_ETIMEOUT
    assert srv.poll(t4)[0] == neat.NEAT_EAGAIN
    srv.cancel(t4)
    code, r4 = srv.wait(t4, 60000)
    assert code == neat.NEAT_ECANCELLED and r4.genome_forwards < 400 * 4 * 20000
    srv.close()
