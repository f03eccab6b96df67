"""Genome distance and species assignment through the C ABI
(neat_distance_prepare, neat_distance, neat_speciate) against the FP64
oracle.

Distances pass within |gpu - ref| <= 1e-5 max(1, |ref|), NaN where the
oracle has NaN; status words and species indices must match exactly (the
species rule is applied by the oracle to the GPU's own float32 distances and
threshold, so both sides decide in the same precision).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2404_01817_gb300 import workloads as W
from tests.genome_helpers import genome, stack
from tests.parity import assert_outputs_close

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "distance_handworked.json")


@pytest.fixture(scope="module")
def neat():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2404_01817_gb300 import neat as N
    return N


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _prepare(neat, nodes, conns, I=3, O=2):
    d = neat.dims(I, O, nodes.shape[1], conns.shape[1])
    genes, st = neat.neat_distance_prepare(_dev(nodes), _dev(conns), d)
    return d, genes, st.cpu().numpy().astype(np.uint32)


def _distance(neat, a, b, cd=1.0, ch=0.5, I=3, O=2):
    d, ga, sa = _prepare(neat, a[0], a[1], I, O)
    _, gb, sb = _prepare(neat, b[0], b[1], I, O)
    out = neat.neat_distance(ga, a[0].shape[0], gb, b[0].shape[0], d, cd, ch).cpu().numpy()
    return out, sa, sb


def _related(seed, pop, nmax=24, cmax=60):
    return W.related_population(seed, pop, 3, 2, nmax, cmax, ancestor_hidden=6, ancestor_edges=20, new_nodes=6,
                                new_conns=12, key_pool=10)


def test_handworked_example(neat):
    g = json.load(open(GOLD))
    a = genome(g["a"]["nodes"], g["a"]["conns"], 6, 6)
    b = genome(g["b"]["nodes"], g["b"]["conns"], 6, 6)
    out, sa, sb = _distance(neat, a, b, g["c_disjoint"], g["c_homologous"])
    assert sa[0] == 0 and sb[0] == 0
    assert out[0, 0] == np.float32(g["distance"])             # dyadic values: exact in float32 too


def test_gene_records(neat):
    p = _related(1, 40)
    d, genes, st = _prepare(neat, p.nodes, p.conns)
    assert (st == 0).all()
    stride = neat.neat_gene_stride(d)
    raw = genes.cpu().numpy()[: 40 * stride].reshape(40, stride)
    for g in range(40):
        hdr = raw[g, :16].view(np.uint32)
        keys = np.sort(p.nodes[g, ~np.isnan(p.nodes[g, :, 0]), 0]).astype(np.uint32)
        present = ~np.isnan(p.conns[g, :, 0])
        pairs = np.sort(p.conns[g, present, 0].astype(np.uint64) << np.uint64(24) |
                        p.conns[g, present, 1].astype(np.uint64))
        n, m = int(hdr[0]), int(hdr[1])
        assert (n, m, int(hdr[2])) == (len(keys), len(pairs), 0)
        np.testing.assert_array_equal(raw[g, 16:16 + 4 * n].view(np.uint32), keys)
        off = 16 + ((4 * n + 15) // 16) * 16 + 16 * n
        np.testing.assert_array_equal(raw[g, off:off + 8 * m].view(np.uint64), pairs)


def _records(neat, nodes, conns, I, O):
    d = neat.dims(I, O, nodes.shape[1], conns.shape[1])
    genes, st = neat.neat_distance_prepare(_dev(nodes), _dev(conns), d)
    stride = neat.neat_gene_stride(d)
    return genes.cpu().numpy()[: nodes.shape[0] * stride].reshape(nodes.shape[0], stride), st.cpu().numpy()


def _written(rec):
    """The bytes a gene record defines: the header, then for a valid record
    the node keys with their padding, node attributes, pair keys and
    connection attributes (the last few bytes of alignment are unwritten)."""
    n, m, status = (int(x) for x in rec[:12].view(np.uint32))
    if status:
        return rec[:16]
    return rec[:16 + (4 * n + 15) // 16 * 16 + 16 * n + 16 * m]


def test_gene_record_forms_agree(neat):
    """Genomes of at most 64 node rows and 256 connection rows are prepared
    one warp each (keys sorted in registers), larger ones one block each
    (keys sorted in shared memory): the same genomes padded past those
    limits give the same record bytes and statuses.  Error genomes (a
    duplicated key, a duplicated pair, a bad key), an empty genome and full
    64 x 256 genomes included, with keys below 2^12 (32-bit sort keys in the
    warp form) and above (64-bit ones)."""
    p = _related(12, 90)
    nodes, conns = p.nodes.copy(), p.conns.copy()
    rn = np.flatnonzero(~np.isnan(nodes[5, :, 0]))
    nodes[5, rn[1]] = nodes[5, rn[0]]
    rc = np.flatnonzero(~np.isnan(conns[9, :, 0]))
    conns[9, rc[1]] = conns[9, rc[0]]
    nodes[13, rn[2], 0] = 1.5
    nodes[20] = np.nan
    conns[20] = np.nan
    conns[21] = np.nan                                      # nodes only
    full = W.random_dag_population(13, 40, 3, 2, 64, 256, hidden=lambda r: 59,
                                   edges=lambda r, n: int(r.integers(200, 257)), acts=W.ALL_ACTS,
                                   aggs=W.ALL_AGGS, p_disabled=0.3)
    wide_n, wide_c = full.nodes.copy(), full.conns.copy()    # keys past 2^12: 64-bit sort keys
    wide_n[:, :, 0] += 5000.0
    wide_c[:, :, :2] += 5000.0
    for (nd, cn, nmax, cmax) in ((nodes, conns, 100, 60), (wide_n, wide_c, 65, 256),
                                 (full.nodes, full.conns, 65, 256), (full.nodes, full.conns, 64, 300)):
        warp, st_w = _records(neat, nd, cn, 3, 2)
        block, st_b = _records(neat, _pad(nd, nmax), _pad(cn, cmax), 3, 2)
        np.testing.assert_array_equal(st_w, st_b)
        for g in range(nd.shape[0]):
            np.testing.assert_array_equal(_written(warp[g]), _written(block[g]), err_msg=f"genome {g}")
    assert (st_w == 0).all()
    _, st = _records(neat, nodes, conns, 3, 2)
    assert np.flatnonzero(st).tolist() == [5, 9, 13]
    n_full = (~np.isnan(full.nodes[:, :, 0])).sum(1)
    assert n_full.max() == 64 and (~np.isnan(full.conns[:, :, 0])).sum(1).max() > 200


@pytest.mark.parametrize("cd,ch", [(1.0, 0.5), (2.0, 3.0)])
def test_distances_match_oracle(neat, cd, ch):
    a = _related(2, 70)
    b = _related(3, 37)                          # another ancestor: mostly disjoint genes
    mixed = (np.concatenate([a.nodes[:20], b.nodes[:17]]), np.concatenate([a.conns[:20], b.conns[:17]]))
    out, sa, sb = _distance(neat, (a.nodes, a.conns), mixed, cd, ch)
    ref, ra, rb = oracle.distance(a.nodes, a.conns, *mixed, cd, ch)
    np.testing.assert_array_equal(sa, ra)
    np.testing.assert_array_equal(sb, rb)
    assert_outputs_close(out, ref, what=f"distance cd={cd} ch={ch}")
    assert out[:, 20:].mean() > out[:, :20].mean()          # the other lineage is farther away


def test_random_dag_populations_and_wide_genomes(neat):
    p = W.random_dag_population(4, 30, 3, 2, 40, 120, hidden=lambda r: int(r.integers(0, 30)),
                                edges=lambda r, n: int(r.integers(0, 3 * n)), acts=W.ALL_ACTS, aggs=W.ALL_AGGS,
                                p_disabled=0.3)
    out, _, _ = _distance(neat, (p.nodes, p.conns), (p.nodes, p.conns))
    ref, _, _ = oracle.distance(p.nodes, p.conns, p.nodes, p.conns, 1.0, 0.5)
    assert_outputs_close(out, ref, what="random DAGs")
    assert (np.diag(out) == 0).all()
    assert_outputs_close(out, out.T, what="symmetry")
    # the largest genomes (1024 nodes, 8192 connections): one record per block
    w = W.related_population(5, 3, 3, 2, 1024, 8192, ancestor_hidden=600, ancestor_edges=6000, new_nodes=300,
                             new_conns=1500, key_pool=400)
    out, _, _ = _distance(neat, (w.nodes, w.conns), (w.nodes, w.conns))
    ref, _, _ = oracle.distance(w.nodes, w.conns, w.nodes, w.conns, 1.0, 0.5)
    assert_outputs_close(out, ref, what="1024 nodes / 8192 conns")


def test_tiling_does_not_change_bits(neat):
    """A column of the distance matrix has the same bits whichever tile of
    representatives, and whichever block of a-genomes, computes it: 1 to 5
    and 9 representatives (tiles of 1, 2, 4 and 8 records, full and partial)
    against a run over 40."""
    p = _related(6, 300)
    d, genes, _ = _prepare(neat, p.nodes, p.conns)
    full = neat.neat_distance(genes, 300, genes, 40, d, 1.0, 0.5).cpu().numpy()
    stride = neat.neat_gene_stride(d)
    for nb in (1, 2, 3, 4, 5, 9):
        part = neat.neat_distance(genes[7 * stride:], 290, genes[5 * stride:], nb, d, 1.0, 0.5).cpu().numpy()
        np.testing.assert_array_equal(part, full[7:297, 5:5 + nb], err_msg=f"{nb} representatives")


def _pad(a, rows):
    out = np.full((a.shape[0], rows, a.shape[2]), np.nan, np.float32)
    out[:, :a.shape[1]] = a
    return out


def test_table_forms_agree_bit_for_bit(neat):
    """The same genomes through the three ways a block indexes its staged
    records, chosen by the dims alone: union tables over the tile's keys (at
    most 255 genes of each kind), one hash table per record (300 nodes) and
    binary search (1024 nodes / 8192 connections).  Records are compact, so
    the distances must agree bit for bit; 21 representatives leave a partial
    last tile, and two error genomes give NaN rows and columns."""
    p = _related(11, 130)
    nodes, conns = p.nodes.copy(), p.conns.copy()
    rn = np.flatnonzero(~np.isnan(nodes[4, :, 0]))
    nodes[4, rn[1]] = nodes[4, rn[0]]                        # a duplicated node key
    rc = np.flatnonzero(~np.isnan(conns[17, :, 0]))
    conns[17, rc[1]] = conns[17, rc[0]]                      # a duplicated connection pair
    ref, _, _ = oracle.distance(nodes, conns, nodes[:21], conns[:21], 1.0, 0.5)
    outs = []
    for nmax, cmax in ((24, 60), (300, 400), (1024, 8192)):
        d, genes, st = _prepare(neat, _pad(nodes, nmax), _pad(conns, cmax))
        assert st[4] and st[17] and np.count_nonzero(st) == 2
        outs.append(neat.neat_distance(genes, 130, genes, 21, d, 1.0, 0.5).cpu().numpy())
    assert_outputs_close(outs[0], ref, what="union tables")
    assert np.isnan(outs[0][4]).all() and np.isnan(outs[0][:, 17]).all()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_invalid_and_empty_genomes(neat):
    ok = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    dupkey = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1), (1, 0.3, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    dupconn = genome([(0, 0, 1, 0, 0), (1, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), (0, 1, 0, 0.1)], 3, 2)
    badkey = genome([(0, 0, 1, 0, 0), (1.5, 0.2, 1, 0, 1)], [(0, 1, 1, 0.5), None], 3, 2)
    empty = genome([None, None, None], [None, None], 3, 2)
    nodes, conns = stack([ok, dupkey, dupconn, badkey, empty])
    out, sa, _ = _distance(neat, (nodes, conns), (nodes, conns), 1.5, 0.5, I=1, O=1)
    ref, ra, _ = oracle.distance(nodes, conns, nodes, conns, 1.5, 0.5)
    np.testing.assert_array_equal(sa, ra)
    assert_outputs_close(out, ref, what="invalid/empty")
    assert out[4, 4] == 0.0 and out[0, 4] == 3.0


def test_genomes_without_connection_rows(neat):
    """max_conns = 0: genes are nodes only, and the connection term is 0;
    the same genomes with 8 all-NaN connection rows and with 100 node rows
    give the same bits."""
    p = _related(14, 60)
    nodes = p.nodes
    ref, _, _ = oracle.distance(nodes, np.zeros((60, 0, 4), np.float32), nodes[:11],
                                np.zeros((11, 0, 4), np.float32), 1.0, 0.5)
    outs = []
    for nmax, cmax in ((24, 0), (24, 8), (100, 0)):
        nd = _pad(nodes, nmax)
        cn = np.full((60, cmax, 4), np.nan, np.float32)
        d, genes, st = _prepare(neat, nd, cn)
        assert (st == 0).all()
        outs.append(neat.neat_distance(genes, 60, genes, 11, d, 1.0, 0.5).cpu().numpy())
    assert_outputs_close(outs[0], ref, what="nodes only")
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_speciate_matches_oracle(neat):
    import torch
    p = _related(7, 500)
    d, genes, _ = _prepare(neat, p.nodes, p.conns)
    reps = 48
    dist = neat.neat_distance(genes, 500, genes, reps, d, 1.0, 0.5)
    dist[13, :] = float("nan")
    dist[14, 3] = float("nan")
    host = dist.cpu().numpy()
    for thr in (0.0, float(np.median(host[:, :reps][np.isfinite(host)])), 3.0):
        thr32 = float(np.float32(thr))
        sp = neat.neat_speciate(dist, thr32).cpu().numpy()
        np.testing.assert_array_equal(sp, oracle.speciate(host.astype(np.float64), thr32))
    sp = neat.neat_speciate(dist, 3.0).cpu().numpy()
    own = np.arange(reps)
    own[13] = -1                                               # row 13 is all NaN
    np.testing.assert_array_equal(sp[:reps], own)              # a representative is its own nearest
    # ties resolve to the lowest column
    t = torch.tensor([[0.5, 0.25, 0.25, 0.25] * 10], device="cuda")
    assert neat.neat_speciate(t, 1.0).cpu().numpy()[0] == 1
    # a strided view: only the first n_reps columns are representatives
    wide = torch.full((500, 64), 0.0, device="cuda")
    wide[:, :reps] = dist
    sp2 = neat.neat_speciate(wide, 3.0, n_reps=reps).cpu().numpy()
    np.testing.assert_array_equal(sp2, sp)


def test_ant_population_against_representatives(neat):
    """10000 Ant-shaped genomes in mid-evolution against 64 representatives
    (the benchmarked launch); 60 sampled rows against the oracle."""
    p = W.ant_related_population(0, 10000)
    d = neat.dims(27, 8, 50, 200)
    genes, st = neat.neat_distance_prepare(_dev(p.nodes), _dev(p.conns), d)
    reps = np.arange(0, 10000, 157)[:64]
    rg, _ = neat.neat_distance_prepare(_dev(p.nodes[reps]), _dev(p.conns[reps]), d)
    out = neat.neat_distance(genes, 10000, rg, 64, d, 1.0, 0.5).cpu().numpy()
    idx = np.arange(0, 10000, 167)
    ref, _, _ = oracle.distance(p.nodes[idx], p.conns[idx], p.nodes[reps], p.conns[reps], 1.0, 0.5)
    assert_outputs_close(out[idx], ref, what="ant distances")
    assert (st.cpu().numpy() == 0).all() and np.isfinite(out).all()
    np.testing.assert_array_equal(out[reps, np.arange(64)], 0.0)
