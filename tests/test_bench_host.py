"""Host logic of the benchmark (no GPU): the algorithmic bytes behind every
roofline fraction, and the source-hash gate on the recorded ncu
instruction counts behind the issue rooflines."""
import numpy as np

import bench
from paper_2404_01817_gb300 import workloads as W

NAN = np.nan


def test_genome_forward_bytes_hand_counted():
    """16 B per present node, 6 B per enabled connection, 4 B per observation
    and per action, counted by hand on two genomes (1 input, 1 output)."""
    nodes = np.full((2, 4, 5), NAN, np.float32)
    nodes[0, 0] = (0, 0, 1, 0, 0)
    nodes[0, 2] = (1, 0.5, 1, 0, 1)
    nodes[0, 3] = (2, -0.5, 1, 0, 1)                 # three present rows, one NaN row between
    nodes[1, 0] = (0, 0, 1, 0, 0)
    nodes[1, 1] = (1, 0.1, 1, 0, 1)                  # two present rows
    conns = np.full((2, 3, 4), NAN, np.float32)
    conns[0, 0] = (0, 2, 1, 0.5)                     # enabled
    conns[0, 1] = (2, 1, 0, 0.25)                    # disabled: no bytes
    conns[0, 2] = (0, 1, NAN, 1.0)                   # enabled flag NaN: absent
    conns[1, 1] = (0, 1, 1, -1.0)                    # enabled
    pop = W.Population(nodes, conns, 1, 1)
    alg, n, e = bench.genome_forward_bytes(pop)
    assert (n, e) == (5, 2)
    assert alg == 16 * 5 + 6 * 2 + 4 * 2 * (1 + 1) == 108


def test_genome_forward_bytes_of_the_ant_population_scale():
    """The benchmarked population: 16.3 MB of algorithmic bytes per step
    (the figure the headline's roofline divides)."""
    pop = W.ant_population(0, 10000)
    alg, n, e = bench.genome_forward_bytes(pop)
    assert alg == 16 * n + 6 * e + 4 * 10000 * (27 + 8)
    assert 16.0e6 < alg < 16.6e6


def test_issue_roofline_needs_matching_sources(tmp_path, monkeypatch):
    """A recorded count is used only while its kernel's sources hash the
    same (any byte changed: no roofline); the fraction is instructions /
    time / (4 schedulers x SMs x clock).  Checked on a scratch tree."""
    import json
    csrc = tmp_path / "paper_2404_01817_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("kernel one")
    (csrc / "k.cuh").write_text("helpers")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    files = ("k.cu", "k.cuh")
    assert bench.source_hash(files) == bench.source_hash(files)
    assert bench.source_hash(files) != bench.source_hash(files[:1])
    rec = {"kernel_hash": bench.source_hash(files), "warp_instructions_per_launch": 5.0e7}
    (tmp_path / "profiles" / "k.json").write_text(json.dumps(rec))
    r = bench.issue_roofline_from_profile("k.json", files, 1e-4, 152, 2070.0)
    assert r is not None and r["bound"] == "issue" and r["instructions_per_launch"] == 5.0e7
    assert abs(r["frac"] - 5.0e7 / 1e-4 / (4 * 152 * 2070.0e6)) < 1e-12
    assert bench.issue_roofline_from_profile("k.json", files[:1], 1e-4, 152, 2070.0) is None
    assert bench.issue_roofline_from_profile("missing.json", files, 1e-4, 152, 2070.0) is None
    (csrc / "k.cu").write_text("kernel two")                 # the kernel changed since the count was taken
    assert bench.issue_roofline_from_profile("k.json", files, 1e-4, 152, 2070.0) is None
