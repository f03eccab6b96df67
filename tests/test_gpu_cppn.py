"""CPPN substrate queries against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome
from tests.parity import compare_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def neat():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_01817_gb300 import neat as N
    return N


def _run(neat, pop, res=16, layers=3, thr=0.2):
    import torch
    d = neat.dims(5, 1, pop.max_nodes, pop.max_conns)
    rec, st = neat.neat_transform(torch.from_numpy(pop.nodes).cuda(), torch.from_numpy(pop.conns).cuda(), d)
    w = neat.neat_cppn_query(rec, pop.pop, d, res, layers, thr)
    torch.cuda.synchronize()
    return w.cpu().numpy()


def _check(w, pop, queries, res, thr=0.2):
    raw, ref = oracle.cppn_query(pop.nodes, pop.conns, res, thr, queries)
    got = w[queries[:, 0], queries[:, 1], queries[:, 2], queries[:, 3]].astype(np.float64)
    # where the float32 threshold decision differs, the raw value must sit at the threshold
    flip = (got == 0) != (ref == 0)
    assert np.all(np.abs(np.abs(raw[flip]) - thr) <= 1e-5 * np.maximum(1, np.abs(raw[flip])))
    bad, mabs, mscaled, n = compare_outputs(got[~flip], ref[~flip])
    assert bad == 0, f"{bad} queries outside tolerance (max scaled {mscaled})"
    return mscaled


def test_cppn_identity_grid(neat):
    """A CPPN that outputs x_s exposes the coordinate grid and the threshold."""
    nodes, conns = genome([(k, 0, 1, 0, 0) for k in range(5)] + [(5, 0, 1, 0, 0)], [(0, 5, 1, 1.0)], 8, 8)
    pop = W.Population(nodes, conns, 5, 1)
    w = _run(neat, pop, res=16, layers=3)
    lin = np.linspace(-1, 1, 16).astype(np.float32)
    xs = lin[np.arange(256) % 16]
    want = np.where(np.abs(xs) < np.float32(0.2), 0, xs)
    for blk in range(2):
        np.testing.assert_array_equal(w[0, blk], np.broadcast_to(want[:, None], (256, 256)))


def test_cppn_population_sampled(neat):
    pop = W.cppn_population(0, 1000)
    w = _run(neat, pop)
    rng = np.random.default_rng(0)
    Q = 20000
    q = np.stack([rng.integers(0, 1000, Q), rng.integers(0, 2, Q), rng.integers(0, 256, Q),
                  rng.integers(0, 256, Q)], 1).astype(np.int32)
    q = q[np.argsort(q[:, 0], kind="stable")]
    err = _check(w, pop, q, 16)
    print(f"cppn max scaled error {err:.3g}")
    # both blocks see identical inputs (no layer coordinate), so they agree bit for bit
    np.testing.assert_array_equal(w[:, 0], w[:, 1])


def test_cppn_full_genomes_and_other_substrate(neat):
    pop = W.cppn_population(7, 12)
    w = _run(neat, pop, res=5, layers=4, thr=0.05)
    g, b, s, t = np.meshgrid(np.arange(12), np.arange(3), np.arange(25), np.arange(25), indexing="ij")
    q = np.stack([g.ravel(), b.ravel(), s.ravel(), t.ravel()], 1).astype(np.int32)
    _check(w, pop, q, 5, thr=0.05)


def test_cppn_shared_memory_at_the_default_limit(neat):
    """Nmax 41: the dynamic shared memory (about 45.6 KB) is under 48 KB but
    with the kernel's static shared memory over it, so the launch needs the
    raised limit."""
    pop = W.random_dag_population(9, 40, 5, 1, 41, 120, hidden=lambda r: int(r.integers(0, 36)),
                                  edges=lambda r, n: int(r.integers(n, 3 * n)),
                                  acts=(W.ACT_SIN, W.ACT_GAUSS, W.ACT_TANH, W.ACT_IDENTITY), aggs=(W.AGG_SUM,))
    w = _run(neat, pop)
    rng = np.random.default_rng(3)
    q = np.stack([rng.integers(0, 40, 4000), rng.integers(0, 2, 4000), rng.integers(0, 256, 4000),
                  rng.integers(0, 256, 4000)], 1).astype(np.int32)
    _check(w, pop, q[np.argsort(q[:, 0], kind="stable")], 16)


@pytest.mark.parametrize("nmax,cmax", [(32, 96), (64, 200), (150, 400)])
def test_cppn_equals_forward_bit_for_bit(neat, nmax, cmax):
    """Over genomes with every activation and aggregation and value tiles of
    32 to 150 rows, the query kernel's raw outputs equal neat_forward's on
    the same coordinate inputs bit for bit, including the ragged last chunk
    (625 queries per block), and match the oracle."""
    import torch
    res, P = 5, 24
    pop = W.random_dag_population(11, P, 5, 1, nmax, cmax, hidden=lambda r: int(r.integers(0, nmax - 5)),
                                  edges=lambda r, n: int(r.integers(n, 2 * n + 1)), acts=W.ALL_ACTS,
                                  aggs=W.ALL_AGGS, p_disabled=0.1)
    d = neat.dims(5, 1, nmax, cmax)
    rec, st = neat.neat_transform(torch.from_numpy(pop.nodes).cuda(), torch.from_numpy(pop.conns).cuda(), d)
    w = neat.neat_cppn_query(rec, P, d, res, 2, 0.0).cpu().numpy()          # threshold 0: raw outputs
    coord = (-1.0 + 2.0 * np.arange(res) / (res - 1)).astype(np.float32)
    node = np.arange(res * res)
    xs, ys = coord[node % res], coord[node // res]
    s, t = np.meshgrid(node, node, indexing="ij")
    x = np.stack([xs[s.ravel()], ys[s.ravel()], xs[t.ravel()], ys[t.ravel()], np.ones(s.size, np.float32)], 1)
    xb = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(x, (P,) + x.shape))).cuda()
    y = neat.neat_forward(rec, P, d, xb).cpu().numpy()[:, :, 0]
    np.testing.assert_array_equal(w[:, 0].reshape(P, -1), y)
    g, b, ss, tt = np.meshgrid(np.arange(P), [0], np.arange(0, 25, 3), np.arange(25), indexing="ij")
    q = np.stack([g.ravel(), b.ravel(), ss.ravel(), tt.ravel()], 1).astype(np.int32)
    _check(w, pop, q, res, thr=0.0)
