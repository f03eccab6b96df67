"""Benchmark: population-wide NEAT genome evaluation on the Ant-shaped control
workload (10 000 genomes, 27 inputs, 8 outputs, max 50 nodes / 200 conns,
tanh, sum; 1000 sequential steps with one N(0,1) observation per genome per
step).

One bench step = one episode of the hot path: transform the population once,
compile its lane programs, then 1000 sequential forwards (Section 3.3:
transform once, calculate per call).  Two forms are timed on the same data:
  batched  the 1000 forwards from lane programs as one CUDA graph with
           programmatic dependent launch (neat_forward_lanes_steps) -- the
           headline `value`;
  plain    one neat_forward call per step from the host (one population per
           launch, the level-walk kernel).
`e2e` repeats the batched episode through the C ABI with the genome tensors
and observations in pinned host memory and the actions copied back, all
inside the timed region.

The episode's observations (1.08 GB) exceed the 129 MB L2, so every episode
streams its inputs from HBM; the lane programs (~13 MB) stay L2-resident
across the steps of an episode, as they would between environment steps.

`roofline` rates the forward launch by the algorithmic bytes of a genome
forward (per genome 16 B per present node and 6 B per enabled connection,
plus 4 B per observation and per action, counted from the generated tensors)
against the measured HBM bandwidth; the bytes the kernel actually stages
(its lane programs) and the transformed records are reported beside it.
`issue_roofline` rates the same launch against instruction issue.  The
default run also measures the other four workloads (XOR latency, the uneven
batch, the CPPN query and serving) and embeds their results under `configs`.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --workload xor|batched|cppn|serving|recurrent|distance|evolve|substrate
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "genome-forwards/s (Ant-shape, 10k pop) batched vs plain, % HBM peak; p50/p99 ms"
UNIT = "genome-forwards/s"
POP, I, O, NMAX, CMAX, ENV_STEPS = 10000, 27, 8, 50, 200, 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--env-steps", type=int, default=ENV_STEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other four workloads in the default run")
    ap.add_argument("--stage-bytes", type=int, default=0,
                    help="Ant: the lane programs' staging reservation (0: chosen by neat_lanes_tune before the "
                         "warm-up); a fixed value keeps the launch sequence fixed for ncu launch lists")
    ap.add_argument("--profile", action="store_true",
                    help="short case for ncu (ant: transform, lane compile, 4 forwards, an 8-step graph; "
                         "batched: one plan step); no timing")
    ap.add_argument("--workload", choices=["ant", "xor", "batched", "cppn", "serving", "recurrent", "distance",
                                           "evolve", "substrate"],
                    default="ant", help="ant: the headline line; the others: the other shapes")
    return ap.parse_args()


def dist_env():
    from paper_2404_01817_gb300.shard import rank_env
    return rank_env()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(pop, obs_host, seconds_target=15.0, single_seconds=5.0):
    """The FP64 oracle on the host cores over a bounded sample of the workload:
    all genomes and the first S steps of the episode on every core (S sized
    from a probe), and beside it the same oracle on one core over a smaller
    sample (the first genomes, the first steps)."""
    import concurrent.futures as cf

    import oracle
    cores = os.cpu_count() or 1
    xs_all = np.ascontiguousarray(obs_host[:, :, 0, :].transpose(1, 0, 2))   # [P][steps][I]
    t0 = time.perf_counter()
    oracle.forward(pop.nodes[:200], pop.conns[:200], I, O, xs_all[:200, :50])
    per_gf = (time.perf_counter() - t0) / (200 * 50)
    S = int(max(10, min(xs_all.shape[1], seconds_target * cores / max(per_gf, 1e-9) / POP / 4)))
    chunks = np.array_split(np.arange(POP), cores * 4)

    def run(idx):
        oracle.forward(pop.nodes[idx], pop.conns[idx], I, O, xs_all[idx, :S])

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(run, chunks))
    dt = time.perf_counter() - t0
    # one core: the first G genomes x first S1 steps, about single_seconds of work
    G = 1000
    S1 = int(max(5, min(xs_all.shape[1], single_seconds / max(per_gf, 1e-9) / G)))
    t0 = time.perf_counter()
    oracle.forward(pop.nodes[:G], pop.conns[:G], I, O, xs_all[:G, :S1])
    dt1 = time.perf_counter() - t0
    return {"value": POP * S / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {POP} genomes x first {S} of the episode's steps (FP64 C oracle, "
                      f"transform once per genome + forward per step, {cores} threads)",
            "single_core": {"value": G * S1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"the first {G} genomes x first {S1} steps, one thread"}}


WORKLOAD = ("Ant-shaped control: 10000 genomes/GPU, 27 in / 8 out, max 50 nodes / 200 conns, "
            "0-15 hidden, 100-200 conns, 10% disabled, tanh, sum; bench step = transform + lane-program "
            "compile + 1000 sequential forwards (1 obs/genome/step)")


def genome_forward_bytes(pop) -> tuple[int, int, int]:
    """Algorithmic bytes of one forward over the population: per genome 16 B
    per present node (12 B of node parameters and 4 B of its value) and 6 B
    per enabled connection (weight and source), plus 4 B per observation and
    per action; returns (bytes, present nodes, enabled connections)."""
    n = int((~np.isnan(pop.nodes[:, :, 0])).sum())
    c = pop.conns
    present = ~(np.isnan(c[:, :, 0]) | np.isnan(c[:, :, 1]) | np.isnan(c[:, :, 2]))
    e = int((present & (np.nan_to_num(c[:, :, 2]) != 0)).sum())
    P = pop.nodes.shape[0]
    return 16 * n + 6 * e + 4 * P * (pop.num_inputs + pop.num_outputs), n, e


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no code) on the
    same workload, all host cores.  One bench step = one episode of the
    workload (every genome transformed once and evaluated on its 1000
    observations), rank 0 only."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import concurrent.futures as cf

    import oracle
    from paper_2404_01817_gb300 import workloads as W
    S = args.env_steps
    pop = W.ant_population(0, POP)
    xs = W.normal_inputs(0, (POP, S, I))                 # [genome][step][input]
    cores = os.cpu_count() or 1
    chunks = np.array_split(np.arange(POP), cores * 4)

    def episode():
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(lambda idx: oracle.forward(pop.nodes[idx], pop.conns[idx], I, O, xs[idx]), chunks))

    for _ in range(args.warmup):
        episode()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        episode()
    dt = time.perf_counter() - t0
    value = POP * S * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"all {POP} genomes x {S} steps per bench step (the whole episode), "
                                       f"FP64 C oracle, {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_events(fn, reps, stream):
    """Run fn reps times between CUDA events on `stream`; per-rep ms."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_xor(args, reps=1000):
    print(json.dumps(measure_xor(args, reps)), flush=True)


def measure_xor(args, reps=1000):
    """XOR (100 genomes grown from the 3 -> 1 net, the 4 points with a bias
    input): latency-bound, so the line reports microseconds per call (CUDA
    events around each call, p50 / p99 over `reps` calls) for the transform
    and the forward, and host-to-host latency of both through the public API;
    the outputs' largest scaled error against the FP64 oracle beside it."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    pop = W.xor_population(0, 100)
    d = neat.dims(3, 1, pop.max_nodes, pop.max_conns)
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    x = torch.from_numpy(W.xor_inputs(100)).to(dev)
    rec, st = neat.neat_transform(nodes, conns, d)
    y = neat.neat_forward(rec, 100, d, x)
    stream = torch.cuda.current_stream(dev)
    L = neat.neat_default_launch(100, d, 4)

    def per_call(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        t = np.array([a.elapsed_time(b) * 1e3 for a, b in ev])
        return float(np.percentile(t, 50)), float(np.percentile(t, 99))
    for _ in range(args.warmup):
        neat.neat_transform(nodes, conns, d, rec, st, stream=stream)
        neat.neat_forward(rec, 100, d, x, y, launch=L, stream=stream)
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        tr = per_call(lambda: neat.neat_transform(nodes, conns, d, rec, st, stream=stream))
        fw = per_call(lambda: neat.neat_forward(rec, 100, d, x, y, launch=L, stream=stream))
    xh = x.cpu().pin_memory()
    yh = torch.empty(y.shape, pin_memory=True)
    host = []
    for _ in range(200):
        t0 = time.perf_counter()
        x.copy_(xh, non_blocking=True)
        neat.neat_forward(rec, 100, d, x, y, launch=L, stream=stream)
        yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        host.append((time.perf_counter() - t0) * 1e6)
    _, _, err = oracle_error(y.cpu().numpy(), oracle.forward(pop.nodes, pop.conns, 3, 1, W.xor_inputs(100)))
    line = {"metric": "XOR population latency (100 genomes x 4 inputs): microseconds per forward call (p50)",
            "value": fw[0], "unit": "us", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": fw[0] / 1e3, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "XOR", "genomes": 100, "inputs_per_genome": 4},
            "transform_us": {"p50": tr[0], "p99": tr[1]}, "forward_us": {"p50": fw[0], "p99": fw[1]},
            "e2e": {"value": float(np.percentile(host, 50)), "unit": "us", "p99": float(np.percentile(host, 99)),
                    "h2d_bytes_per_step": int(x.numel() * 4), "d2h_bytes_per_step": int(y.numel() * 4)},
            "clocks": clocks.summary(), "gpu_launches": 2 * reps,
            "parity": {"max_scaled_error": err, "compared": "all 100 genomes x 4 points vs the FP64 oracle"}}
    return line


def run_batched(args):
    line = measure_batched(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def measure_batched(args):
    """Uneven batch: 4 populations x 2048 genomes (max nodes 16/64/256/1024,
    conns ~4x nodes, all activations and aggregations), 64 N(0,1) inputs per
    genome per step, 100 steps; the plan (one persistent launch per step, as
    a CUDA graph) against plain per-population launches; step 0's outputs of
    16 genomes per population against the FP64 oracle."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    S, B = (2 if args.profile else 100), 64
    pops = W.batched_populations(0, pop=2048)
    descs = []
    for j, p in enumerate(pops):
        d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
        rec, st = neat.neat_transform(torch.from_numpy(p.nodes).to(dev), torch.from_numpy(p.conns).to(dev), d)
        g = torch.Generator(device=dev)
        g.manual_seed(10 + j)
        x = torch.randn((S, p.pop, B, p.num_inputs), device=dev, generator=g)
        y = torch.empty((S, p.pop, B, p.num_outputs), device=dev)
        descs.append(dict(transformed=rec, pop=p.pop, dims=d, inputs=x, outputs=y))
    stream = torch.cuda.current_stream(dev)
    plan = neat.Plan(descs, autotune=True)
    if args.profile:                       # one step inside an NVTX range, for ncu --nvtx-include neat_step/
        plan.forward(0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("neat_step")
        plan.forward(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps(plan.describe()), flush=True)
        plan.close()
        return
    for _ in range(args.warmup):
        plan.forward_steps(0, S)
    torch.cuda.synchronize()
    errs = []
    for j, (p, dd) in enumerate(zip(pops, descs)):
        idx = np.arange(0, p.pop, p.pop // 16)[:16]
        xs = dd["inputs"][0][idx].cpu().numpy()
        ref = oracle.forward(p.nodes[idx], p.conns[idx], p.num_inputs, p.num_outputs, xs)
        errs.append(oracle_error(dd["outputs"][0][idx].cpu().numpy(), ref)[2])
    with ClockSampler(0) as clocks:
        ms_b = timed_events(lambda: plan.forward_steps(0, S), args.steps, stream)
    launches = [neat.neat_default_launch(p.pop, dd["dims"], B) for p, dd in zip(pops, descs)]

    def plain():
        for s in range(S):
            for p, dd, L in zip(pops, descs, launches):
                neat.neat_forward(dd["transformed"], p.pop, dd["dims"], dd["inputs"][s], dd["outputs"][s],
                                  launch=L, stream=stream)
    plain()
    ms_p = timed_events(plain, max(1, min(args.steps, 5)), stream)
    gf = sum(p.pop for p in pops) * B * S
    # algorithmic bytes of one step: every record once, the step's inputs and outputs
    alg = 0
    for p, dd in zip(pops, descs):
        hdr = dd["transformed"][:p.pop * neat.neat_record_stride(dd["dims"])].view(p.pop, -1)[:, :32].cpu().numpy()
        alg += int(hdr.view(np.uint32)[:, 4].astype(np.int64).sum()) + 4 * p.pop * B * (p.num_inputs + p.num_outputs)
    t_step = statistics.median(ms_b) / 1e3 / S
    peak, src = measured_peaks()
    line = {"metric": "genome-forwards/s (batched uneven: 4 pops x 2048, Nmax 16/64/256/1024, B=64)",
            "value": gf / (statistics.median(ms_b) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.median(ms_b) / S, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched uneven", "steps_per_graph": S, "batch": B},
            "plain": {"value": gf / (statistics.median(ms_p) / 1e3), "ms_per_step": statistics.median(ms_p) / S},
            "plan": plan.describe(), "clocks": clocks.summary(),
            "roofline": {"bound": "hbm", "achieved": alg / t_step / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / t_step / 1e9 / peak, "traffic": None, "peak_source": src,
                         "note": "plan kernel per step; algorithmic bytes = every record once + inputs + outputs. "
                                 "The large buckets are bound by shared-memory gathers (4 B per edge per input "
                                 "vector) and FP32/SFU issue, not HBM"},
            "gpu_launches": args.steps * S,
            "parity": {"max_scaled_error": max(errs), "per_population": errs,
                       "compared": "step 0, 16 genomes x 64 inputs per population vs the FP64 oracle"}}
    plan.close()
    return line


def run_cppn(args):
    print(json.dumps(measure_cppn(args)), flush=True)


def measure_cppn(args):
    """CPPN substrate batch: 1000 CPPNs x 131072 queries (3 layers of 16x16);
    2000 sampled queries against the FP64 oracle (a threshold decision may
    differ only where the raw value sits at 0.2 within the tolerance)."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    pop = W.cppn_population(0, 1000)
    d = neat.dims(5, 1, pop.max_nodes, pop.max_conns)
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    rec, st = neat.neat_transform(nodes, conns, d)
    w = torch.empty((1000, 2, 256, 256), device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        neat.neat_transform(nodes, conns, d, rec, st, stream=stream)
        neat.neat_cppn_query(rec, 1000, d, 16, 3, 0.2, w, stream=stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        ms = timed_events(step, max(args.steps, 50), stream)
        ms_q = timed_events(lambda: neat.neat_cppn_query(rec, 1000, d, 16, 3, 0.2, w, stream=stream),
                            max(args.steps, 50), stream)
    rng = np.random.default_rng(9)
    qs = np.stack([rng.integers(0, 1000, 2000), rng.integers(0, 2, 2000), rng.integers(0, 256, 2000),
                   rng.integers(0, 256, 2000)], axis=1).astype(np.int32)
    raw, ref = oracle.cppn_query(pop.nodes, pop.conns, 16, 0.2, qs)
    got = w[qs[:, 0], qs[:, 1], qs[:, 2], qs[:, 3]].cpu().numpy().astype(np.float64)
    flip = (got == 0) != (ref == 0)
    flips_ok = bool(np.all(np.abs(np.abs(raw[flip]) - 0.2) <= 1e-5 * np.maximum(1, np.abs(raw[flip]))))
    _, _, err = oracle_error(got[~flip], ref[~flip])
    hdr = rec.view(1000, -1)[:, :32].cpu().numpy().view(np.uint32)
    edges = hdr[:, 1].astype(np.int64)
    nonin = (hdr[:, 0] & 0xFFFF).astype(np.int64) - 5
    q = 1000 * 131072
    t = statistics.median(ms) / 1e3
    tq = statistics.median(ms_q) / 1e3
    flops = 131072 * int((2 * edges + 2 * nonin).sum())       # one FMA per edge, bias/response FMA per node
    cs = clocks.summary()
    sm_mhz = cs["sm_mhz"] or cs["sm_max_mhz"] or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12           # TFLOP/s at the sampled clock
    line = {"metric": "CPPN substrate queries/s (1000 CPPNs x 131072 queries, 3 layers of 16x16)",
            "value": q / t, "unit": "queries/s", "n_gpus": 1, "steps": max(args.steps, 50), "warmup": args.warmup,
            "ms_per_step": statistics.median(ms), "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "CPPN", "genomes": 1000, "queries_per_genome": 131072,
                       "l2": "no flush: 524 MB of weights written per step, larger than L2"},
            "query_kernel_ms": tq * 1e3,
            "roofline": {"bound": "alu", "achieved": flops / tq / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": flops / tq / 1e12 / fp32_peak,
                         "note": f"FMA flops of the edges and node rule against {sms} SMs x 128 FP32 lanes x 2 at "
                                 "the sampled clock; the transcendental activations (sin, exp) are not counted"},
            "parity": {"max_scaled_error": err, "threshold_flips_at_boundary_only": flips_ok,
                       "threshold_flips": int(flip.sum()), "compared": "2000 random queries vs the FP64 oracle"},
            "clocks": cs, "gpu_launches": 2 * max(args.steps, 50)}
    issue = issue_roofline_from_profile("cppn_query_traffic.json", ("neat_cppn.cu", "neat_device.cuh",
                                                                   "neat_internal.h", "neat_item.cuh"),
                                        tq, sms, sm_mhz)
    if issue:
        line["issue_roofline"] = issue
    return line


def run_recurrent(args, S=100, K=8):
    """Recurrent Ant-shaped genomes: 10000 genomes (27 in, 8 out, max 50
    nodes / 200 conns, connections in any direction, tanh, sum), one N(0,1)
    observation per genome per step, K = 8 synchronous iterations per
    forward; S = 100 steps captured in one CUDA graph.  The line's value is
    the recurrent lane programs (neat_lanes_pack_recurrent once, then
    neat_forward_lanes_recurrent per step with programmatic dependent
    launch); the recurrent kernel (neat_forward_recurrent) is timed beside
    it, and the two agree bit for bit on every step."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    pop = W.ant_recurrent_population(0, POP)
    d = neat.dims(I, O, NMAX, CMAX)
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    rec, st = neat.neat_transform_recurrent(nodes, conns, d)
    gen = torch.Generator(device=dev)
    gen.manual_seed(77)
    x = torch.randn((S, POP, 1, I), device=dev, generator=gen)
    y = torch.empty((S, POP, 1, O), device=dev)
    side = torch.cuda.Stream(dev)

    L = neat.neat_default_launch_recurrent(POP, d, 1)
    L.pdl = 1                                    # each step's record copy overlaps the previous step
    # genomes ordered by node count (neat_schedule), 8 threads per genome,
    # 16 genomes per block: 21.5 us/step against 24.0 for the default shape
    # (a sweep of 8/16/32 threads per genome and 128-512 threads per block,
    # with and without the order; bit-identical in every shape)
    order = neat.neat_schedule(rec, POP, d)
    L.group, L.groups_per_block = 8, 16
    L.order_dev = order.data_ptr()

    def steps(stream):
        for s in range(S):
            neat.neat_forward_recurrent(rec, POP, d, x[s], K, y[s], launch=L, stream=stream)
    # recurrent lane programs: compiled once, every program staged in shared
    # memory (the largest program as the reservation: five blocks per SM)
    lanes = neat.neat_lanes_pack_recurrent(rec, POP, d)
    info = neat.neat_lanes_query(lanes)
    stage = (info.max_warp_bytes + 15) // 16 * 16
    y_l = torch.empty((S, POP, O), device=dev)

    def lane_steps(stream):
        for s in range(S):
            neat.neat_forward_lanes_recurrent(lanes, POP, d, x[s].view(POP, I), K, y_l[s], stage_bytes=stage,
                                              pdl=s > 0, stream=stream)
    stream = torch.cuda.current_stream(dev)
    graphs = []
    for fn, out in ((steps, y), (lane_steps, y_l)):
        fn(side)                                 # eager once: attributes set, reference outputs
        torch.cuda.synchronize()
        eager = out.clone()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            fn(side)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager), "graph replay differs from eager launches"
        graphs.append(graph)
    assert torch.equal(y.view(S, POP, O), y_l), "lane programs differ from the recurrent kernel"
    with ClockSampler(0) as clocks:
        ms = timed_events(graphs[1].replay, max(args.steps, 50), stream)
        ms_kernel = timed_events(graphs[0].replay, max(args.steps, 50), stream)
    t_step = statistics.median(ms) / 1e3 / S
    t_kernel = statistics.median(ms_kernel) / 1e3 / S
    hdr = rec.view(POP, -1)[:, :32].cpu().numpy().view(np.uint32)
    used = int(hdr[:, 4].astype(np.int64).sum())
    alg, _, _ = genome_forward_bytes(pop)         # genome bytes + observations + actions per step
    peak, src = measured_peaks()
    achieved = alg / t_step / 1e9
    # FP64 oracle on a bounded sample, one host thread
    idx = np.arange(0, POP, 20)
    sub = pop.subset(idx)
    xs = x[:10, idx].cpu().numpy().transpose(1, 0, 2, 3).reshape(idx.size, 10, I)
    t0 = time.perf_counter()
    oracle.forward_recurrent(sub.nodes, sub.conns, I, O, xs, K)
    dt = time.perf_counter() - t0
    dt_all, cores = oracle_cores(lambda c: oracle.forward_recurrent(sub.nodes[c], sub.conns[c], I, O, xs[c], K),
                                 idx.size)
    cs = clocks.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue = issue_roofline_from_profile("recurrent_lanes_traffic.json", ("neat_lanes.cu", "neat_device.cuh",
                                                                        "neat_internal.h", "neat_item.cuh"),
                                        t_step, sms, cs["sm_mhz"] or cs["sm_max_mhz"] or 2070.0)
    issue_kernel = issue_roofline_from_profile("recurrent_ant_traffic.json", ("neat_recurrent.cu", "neat_device.cuh",
                                                                             "neat_internal.h", "neat_item.cuh"),
                                               t_kernel, sms, cs["sm_mhz"] or cs["sm_max_mhz"] or 2070.0)
    line = {"metric": f"recurrent genome-forwards/s (10000 Ant-shaped recurrent genomes, K={K} iterations, B=1)",
            "value": POP / t_step, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Ant-shaped recurrent", "iterations": K, "env_steps_per_graph": S,
                       "form": "recurrent lane programs (two threads per genome, 16 genomes per warp, two "
                               "interleaved value tiles, one warp barrier per iteration), PDL between steps",
                       "launch": {"warps": info.warps, "threads_per_block": 32, "stage_bytes": stage,
                                  "largest_program_bytes": info.max_warp_bytes},
                       "l2": "inputs larger than L2 (108 MB of observations + 32 MB of actions per graph "
                             "replay; the 20 MB of records stay L2-resident across steps, as in a real episode)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "alg_bytes_per_launch": alg, "record_bytes": used,
                         "note": "algorithmic bytes = per genome 16 B x present nodes + 6 B x enabled connections, "
                                 "+ 4 B x (inputs + outputs), per step; each forward makes K passes over its "
                                 "staged edges, so the kernel is bound by shared-memory and instruction issue, "
                                 "not by HBM"},
            "recurrent_kernel": {"value": POP / t_kernel, "unit": UNIT, "ms_per_step": t_kernel * 1e3,
                                 "form": "neat_forward_recurrent: 8 threads per genome, 16 genomes per block, "
                                         "genomes in neat_schedule's node-count order, PDL",
                                 "issue_roofline": issue_kernel,
                                 "bit_identical_to_lanes": True},
            "cpu_baseline": {"value": idx.size * 10 / dt_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{idx.size} genomes x 10 steps, FP64 C oracle, {cores} threads",
                             "single_core": {"value": idx.size * 10 / dt, "unit": UNIT, "cores": 1}},
            "clocks": cs, "gpu_launches": max(args.steps, 50) * S}
    if issue:
        line["issue_roofline"] = issue
    print(json.dumps(line), flush=True)


def run_distance(args, R=64):
    """Speciation distances: 10000 Ant-shaped genomes in mid-evolution (27 in,
    8 out, max 50 nodes / 200 conns; mutated copies of one ancestor) against
    R = 64 representatives; one step = gene records of the population and of
    the representatives (two streams: the two launches are independent), the
    10000 x 64 distance matrix, and the species assignment
    (compatibility_disjoint 1.0, compatibility_homologous 0.5, threshold
    3.0)."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    pop = W.ant_related_population(0, POP)
    d = neat.dims(I, O, NMAX, CMAX)
    reps = np.arange(0, POP, POP // R)[:R]
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    rn = torch.from_numpy(np.ascontiguousarray(pop.nodes[reps])).to(dev)
    rc = torch.from_numpy(np.ascontiguousarray(pop.conns[reps])).to(dev)
    genes, st = neat.neat_distance_prepare(nodes, conns, d)
    rgenes, rst = neat.neat_distance_prepare(rn, rc, d)
    dist = torch.empty((POP, R), device=dev)
    species = torch.empty(POP, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    # the representatives' records (16 blocks: latency-bound) on a second
    # stream, beside the population's; the distance kernel waits for both
    side = torch.cuda.Stream(dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step(record=False):
        if record:
            ev[0].record(stream)
        fork.record(stream)
        side.wait_event(fork)
        neat.neat_distance_prepare(rn, rc, d, rgenes, rst, stream=side)
        join.record(side)
        neat.neat_distance_prepare(nodes, conns, d, genes, st, stream=stream)
        stream.wait_event(join)
        if record:
            ev[1].record(stream)
        neat.neat_distance(genes, POP, rgenes, R, d, 1.0, 0.5, dist, stream=stream)
        if record:
            ev[2].record(stream)
        neat.neat_speciate(dist, 3.0, species=species, stream=stream)
        if record:
            ev[3].record(stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_rep = max(args.steps, 1500)                     # ~0.25 s: a dozen clock samples
    with ClockSampler(0) as clocks:
        ms = timed_events(step, n_rep, stream)
    parts = []
    for _ in range(5):
        step(record=True)
        torch.cuda.synchronize()
        parts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
    prep_ms, dist_ms, spec_ms = (statistics.median(p[i] for p in parts) for i in range(3))
    t = statistics.median(ms) / 1e3
    hdr = genes.view(POP, -1)[:, :16].cpu().numpy().view(np.uint32)
    used_a = int(hdr[:, 3].astype(np.int64).sum())
    rh = rgenes.view(R, -1)[:, :16].cpu().numpy().view(np.uint32)
    used_b = int(rh[:, 3].astype(np.int64).sum())
    alg = used_a + used_b + 4 * POP * R              # gene records read once + the distance matrix written
    peak, src = measured_peaks()
    achieved = alg / (dist_ms / 1e3) / 1e9
    # FP64 oracle on a bounded sample, one host thread
    idx = np.arange(0, POP, 50)
    t0 = time.perf_counter()
    oracle.distance(pop.nodes[idx], pop.conns[idx], pop.nodes[reps], pop.conns[reps], 1.0, 0.5)
    dt = time.perf_counter() - t0
    dt_all, cores = oracle_cores(lambda c: oracle.distance(pop.nodes[idx[c]], pop.conns[idx[c]], pop.nodes[reps],
                                                           pop.conns[reps], 1.0, 0.5), idx.size)
    cs = clocks.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue = issue_roofline_from_profile("distance_traffic.json", ("neat_distance.cu", "neat_device.cuh",
                                                                 "neat_internal.h"),
                                        dist_ms / 1e3, sms, cs["sm_mhz"] or cs["sm_max_mhz"] or 2070.0)
    line = {"metric": "genome-pair distances/s (10000 Ant-shaped genomes x 64 representatives, with gene records "
                      "and species assignment)",
            "value": POP * R / t, "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "speciation distances", "representatives": R,
                       "l2": "no flush: the 42 MB of gene records fit in L2, as between the prepare and distance "
                             "launches of a generation"},
            "components_ms": {"prepare": prep_ms, "distance": dist_ms, "speciate": spec_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "note": "distance kernel; algorithmic bytes = used gene-record bytes of both sides + the "
                                 "f32 distance matrix; the kernel is bound by instruction issue (one union-table "
                                 "probe per gene, per-representative row reads and warp reductions), not by HBM"},
            "cpu_baseline": {"value": idx.size * R / dt_all, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{idx.size} genomes x {R} representatives, FP64 C oracle (all-pairs "
                                       f"gene matching), {cores} threads",
                             "single_core": {"value": idx.size * R / dt, "unit": "pairs/s", "cores": 1}},
            "clocks": cs, "gpu_launches": 4 * n_rep}
    if issue:
        line["issue_roofline"] = issue
    print(json.dumps(line), flush=True)


def run_evolve(args):
    """One generation of variation for 10000 Ant-shaped genomes in
    mid-evolution (27 in, 8 out, max 50 nodes / 200 conns): random words and
    normals (Philox; the mutation's on a second stream beside the
    crossover), 10000 crossovers of random parent pairs, mutation with
    the appendix's Brax settings (node_add 0.2, conn_add 0.4, bias and weight
    perturbation 0.5 at rates 0.7 / 0.8, replacement 0.1; feedforward
    check), and the transform of the children (ready for evaluation)."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    pop = W.ant_related_population(0, POP, acyclic=True)
    d = neat.dims(I, O, NMAX, CMAX)
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    rng = np.random.default_rng(5)
    parents_h = rng.integers(0, POP, size=(POP, 2)).astype(np.int32)
    parents = torch.from_numpy(parents_h).to(dev)
    Wn, Zn = neat.neat_mutation_sizes(d)
    xwords = torch.empty((POP, NMAX + CMAX), dtype=torch.int32, device=dev)
    mwords = torch.empty((POP, Wn), dtype=torch.int32, device=dev)
    normals = torch.empty((POP, Zn), device=dev)
    keys = torch.arange(1000, 1000 + POP, dtype=torch.int32, device=dev)
    child_n = torch.empty_like(nodes)
    child_c = torch.empty_like(conns)
    rec = torch.empty(neat.neat_transformed_bytes(POP, d), dtype=torch.uint8, device=dev)
    status = torch.empty(POP, dtype=torch.int32, device=dev)
    cfg = neat.mutation(node_add=0.2, conn_add=0.4, bias_init_std=1.0, bias_mutate_power=0.5, bias_mutate_rate=0.7,
                        bias_replace_rate=0.1, weight_init_std=1.0, weight_mutate_power=0.5, weight_mutate_rate=0.8,
                        weight_replace_rate=0.1)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    gen = [0]

    # the mutation's random inputs on a second stream, beside the crossover
    # (they do not depend on it); the mutation waits for both
    side = torch.cuda.Stream(dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step(record=False):
        g = gen[0]
        gen[0] += 1
        if record:
            ev[0].record(stream)
        fork.record(stream)
        side.wait_event(fork)
        neat.neat_fill_words(11, 3 * g + 1, mwords, stream=side)
        neat.neat_fill_normal(11, g, normals, stream=side)
        join.record(side)
        neat.neat_fill_words(11, 3 * g, xwords, stream=stream)
        if record:
            ev[1].record(stream)
        neat.neat_crossover(nodes, conns, d, parents, xwords, child_n, child_c, stream=stream)
        stream.wait_event(join)
        if record:
            ev[2].record(stream)
        neat.neat_mutate(child_n, child_c, d, cfg, mwords, normals, keys, stream=stream)
        if record:
            ev[3].record(stream)
        neat.neat_transform(child_n, child_c, d, rec, status, stream=stream)
        if record:
            ev[4].record(stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_rep = max(args.steps, 800)                      # ~0.25 s: a dozen clock samples
    with ClockSampler(0) as clocks:
        ms = timed_events(step, n_rep, stream)
    parts = []
    for _ in range(5):
        step(record=True)
        torch.cuda.synchronize()
        parts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    comp = {k: statistics.median(p[i] for p in parts)
            for i, k in enumerate(("crossover_words", "crossover_and_mutation_inputs", "mutate", "transform"))}
    assert (status.cpu().numpy() & 0xFF == 0).all(), "children must stay valid and acyclic"
    t = statistics.median(ms) / 1e3
    # the mutation kernel's bytes: the children's tensors read and written, its random inputs read
    mut_bytes = 2 * (child_n.numel() + child_c.numel()) * 4 + (mwords.numel() + normals.numel()) * 4
    peak, src = measured_peaks()
    achieved = mut_bytes / (comp["mutate"] / 1e3) / 1e9
    # FP64 oracle on a bounded sample: crossover + mutation, one host thread
    idx = np.arange(0, POP, 20)
    xw = xwords[idx].cpu().numpy().view(np.uint32)
    mw = mwords[idx].cpu().numpy().view(np.uint32)
    zz = normals[idx].cpu().numpy()
    t0 = time.perf_counter()
    cn, cc = oracle.crossover(pop.nodes, pop.conns, parents_h[idx], xw)
    oracle.mutate(cn, cc, I, O, oracle.mutation_config(node_add=0.2, conn_add=0.4, bias_init_std=1.0,
                                                       bias_mutate_power=0.5, bias_mutate_rate=0.7,
                                                       bias_replace_rate=0.1, weight_init_std=1.0,
                                                       weight_mutate_power=0.5, weight_mutate_rate=0.8,
                                                       weight_replace_rate=0.1),
                  mw, zz, np.arange(idx.size) + 1000)
    dt = time.perf_counter() - t0
    mcfg = oracle.mutation_config(node_add=0.2, conn_add=0.4, bias_init_std=1.0, bias_mutate_power=0.5,
                                  bias_mutate_rate=0.7, bias_replace_rate=0.1, weight_init_std=1.0,
                                  weight_mutate_power=0.5, weight_mutate_rate=0.8, weight_replace_rate=0.1)

    def vary(c):
        cn_c, cc_c = oracle.crossover(pop.nodes, pop.conns, parents_h[idx[c]], xw[c])
        oracle.mutate(cn_c, cc_c, I, O, mcfg, mw[c], zz[c], c + 1000)
    dt_all, cores = oracle_cores(vary, idx.size)
    cs = clocks.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue = issue_roofline_from_profile("mutate_traffic.json", ("neat_evolve.cu", "neat_device.cuh",
                                                               "neat_internal.h", "neat_hash.cuh"),
                                        comp["mutate"] / 1e3, sms, cs["sm_mhz"] or cs["sm_max_mhz"] or 2070.0)
    line = {"metric": "genomes/s through one generation of variation (10000 Ant-shaped genomes: random inputs, "
                      "crossover, mutation, transform)",
            "value": POP / t, "unit": "genomes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "evolve", "l2": "no flush: the 2 x 36 MB of parent and child tensors stay "
                                                  "L2-resident within a generation"},
            "components_ms": comp,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "note": "mutation kernel: child tensors read + written and its random inputs read; "
                                 "one block per genome runs the structural steps with block barriers, so it is "
                                 "latency-bound"},
            "cpu_baseline": {"value": idx.size / dt_all, "unit": "genomes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{idx.size} children: crossover + mutation, FP64 C oracle, {cores} threads "
                                       f"(transform not included)",
                             "single_core": {"value": idx.size / dt, "unit": "genomes/s", "cores": 1}},
            "clocks": cs, "gpu_launches": 6 * n_rep}
    if issue:
        line["issue_roofline"] = issue
    print(json.dumps(line), flush=True)


def run_substrate(args, S=50):
    """HyperNEAT substrate control step: 1000 CPPN genomes' weight blocks
    (neat_cppn_query, 3 layers of 16 x 16, threshold 0.2; 524 MB resident)
    evaluated on one N(0,1) input vector per genome per step (tanh hidden and
    output layers), S steps per timed repetition; the same at 16 vectors per
    genome is reported beside it."""
    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    P = 1000
    pop = W.cppn_population(0, P)
    d = neat.dims(5, 1, pop.max_nodes, pop.max_conns)
    rec, _ = neat.neat_transform(torch.from_numpy(pop.nodes).to(dev), torch.from_numpy(pop.conns).to(dev), d)
    w = neat.neat_cppn_query(rec, P, d, 16, 3, 0.2).contiguous()
    gen = torch.Generator(device=dev)
    gen.manual_seed(21)
    x1 = torch.randn((S, P, 1, 256), device=dev, generator=gen)
    y1 = torch.empty_like(x1)
    x16 = torch.randn((P, 16, 256), device=dev, generator=gen)
    y16 = torch.empty_like(x16)
    stream = torch.cuda.current_stream(dev)

    def steps():
        for s in range(S):
            neat.neat_substrate_forward(w, x1[s], outputs=y1[s], stream=stream)
    for _ in range(args.warmup):
        steps()
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        ms = timed_events(steps, args.steps, stream)
    t = statistics.median(ms) / 1e3 / S
    ms16 = timed_events(lambda: neat.neat_substrate_forward(w, x16, outputs=y16, stream=stream), 10, stream)
    t16 = statistics.median(ms16) / 1e3
    wbytes = w.numel() * 4
    alg = wbytes + 2 * P * 256 * 4                   # weight blocks read once + inputs + outputs
    peak, src = measured_peaks()
    achieved = alg / t / 1e9
    idx = np.arange(0, P, 100)
    wh = w[idx].cpu().numpy()
    xh = x1[0, idx].cpu().numpy()
    t0 = time.perf_counter()
    oracle.substrate_forward(wh, xh)
    dt = time.perf_counter() - t0
    line = {"metric": "substrate genome-forwards/s (1000 HyperNEAT substrates, 3 layers of 16 x 16, 1 input "
                      "vector per genome per step)",
            "value": P / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "HyperNEAT substrate", "resolution": 16, "layers": 3, "steps_per_rep": S,
                       "l2": "inputs larger than L2 (524 MB of weight blocks read every step)"},
            "batch16": {"value": P * 16 / t16, "unit": UNIT, "ms": t16 * 1e3,
                        "achieved_gbs": (wbytes + 2 * P * 16 * 256 * 4) / t16 / 1e9},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "note": "algorithmic bytes = the weight blocks (read once per step) + inputs + outputs"},
            "cpu_baseline": {"value": idx.size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{idx.size} substrates x 1 vector, FP64 C oracle, one thread"},
            "clocks": clocks.summary(), "gpu_launches": args.steps * S}
    print(json.dumps(line), flush=True)


def run_serving(args):
    print(json.dumps(measure_serving(args)), flush=True)


def measure_serving(args, n_requests=2000, budgets_mb=(64, 256, 1024, 16384)):
    """Serving: a Poisson stream (200 requests/s) of `n_requests` requests,
    each with its own log-uniform population (64-4096), max nodes (8-512)
    and observation batch (1-256) and its own genomes (drawn per request,
    in parallel threads ahead of the stream), 100 steps each, through
    neat_serve_* at several HBM budgets (small ones make admission wait;
    a request that can never fit a budget is refused and counted).  The last
    step's outputs of three requests are checked against the FP64 oracle
    (16 genomes each, observations regenerated with neat_fill_normal).
    Beside it, the plain form on the same stream: one request at a time in
    arrival order, each a transform and one neat_forward launch per step
    (no request shares a launch), latency from the request's scheduled
    arrival; its outputs equal the served ones bit for bit."""
    import collections
    import concurrent.futures as cf
    import threading

    import torch
    import oracle
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    reqs = W.serving_requests(0, n_requests)
    results = {}
    parity = None
    served_last = {}                     # last-step outputs of a few requests, largest budget
    for budget_mb in budgets_mb:
        budget = int(budget_mb) << 20
        srv = neat.Server(budget, max_active=256)
        warm = W.request_population_fast(dict(reqs[0], pop=64))
        d0 = neat.dims(warm.num_inputs, warm.num_outputs, warm.max_nodes, warm.max_conns)
        y0 = torch.empty((64, reqs[0]["batch"], warm.num_outputs), device=dev)
        srv.wait(srv.submit(warm.nodes, warm.conns, d0, reqs[0]["batch"], 2, 1, y0))
        tickets, outs, refused = [], {}, []
        lag = []
        pool = cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1))
        window = collections.deque()
        ahead = 48

        def client():
            nxt = 0
            t0 = time.perf_counter()
            for i, r in enumerate(reqs):
                while nxt < len(reqs) and nxt < i + ahead:
                    window.append(pool.submit(W.request_population_fast, reqs[nxt]))
                    nxt += 1
                p = window.popleft().result()
                dt = r["arrival_s"] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                else:
                    lag.append(-dt)
                d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
                y = torch.empty((p.pop, r["batch"], p.num_outputs), device=dev)
                try:
                    tk = srv.submit(p.nodes, p.conns, d, r["batch"], r["steps"], r["seed"], y)
                except neat.NeatError as e:
                    if e.code != neat.NEAT_EBUDGET:
                        raise
                    refused.append(i)
                    continue
                tickets.append((i, tk))
                outs[i] = (y, d)
        with ClockSampler(0) as clocks:
            th = threading.Thread(target=client)
            th.start()
            th.join()
            for i, tk in tickets:
                srv.wait(tk, 600000)
        pool.shutdown()
        st = srv.stats()
        results[f"{budget_mb}MB"] = {
            "latency_p50_ms": st.latency_p50_ms, "latency_p99_ms": st.latency_p99_ms,
            "queue_wait_p50_ms": st.queue_wait_p50_ms, "queue_wait_p99_ms": st.queue_wait_p99_ms,
            "completed": st.completed, "refused_never_fit": len(refused),
            "genome_forwards_per_s": st.genome_forwards_per_s, "ticks": st.ticks,
            "arrival_lag_p99_ms": float(np.percentile(lag, 99)) * 1e3 if lag else 0.0,
            "clocks": clocks.summary()}
        if parity is None and tickets:
            errs = []
            for i, _ in tickets[:3]:
                r = reqs[i]
                y, d = outs[i]
                p = W.request_population_fast(r)
                obs = torch.empty(p.pop * r["batch"] * p.num_inputs, device=dev)
                neat.neat_fill_normal(r["seed"], r["steps"] - 1, obs)
                x = obs.view(p.pop, r["batch"], p.num_inputs).cpu().numpy()
                idx = np.arange(0, p.pop, max(1, p.pop // 16))[:16]
                ref = oracle.forward(p.nodes[idx], p.conns[idx], p.num_inputs, p.num_outputs, x[idx])
                errs.append(oracle_error(y[idx].cpu().numpy(), ref)[2])
            parity = {"max_scaled_error": max(errs),
                      "compared": "last step of 3 requests, 16 genomes each, vs the FP64 oracle"}
        if budget_mb == budgets_mb[-1]:
            for i, _ in tickets[:8]:
                served_last[i] = outs[i][0].clone()
        srv.close()
        outs.clear()
    plain = measure_serving_plain(reqs, served_last)
    best = results[f"{budgets_mb[-1]}MB"]
    line = {"metric": "serving: genome-forwards/s and request latency p50/p99 ms (Poisson 200 req/s)",
            "value": best["genome_forwards_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving", "requests": n_requests, "rate_hz": 200, "steps_per_request": 100,
                       "genomes": "drawn per request (random_dag_population_vec, the Ant recipe at the request's "
                                  "size)", "budgets_mb": list(budgets_mb)},
            "latency_ms": {"p50": best["latency_p50_ms"], "p99": best["latency_p99_ms"]},
            "budgets": results, "plain": plain, "parity": parity}
    return line


def measure_serving_plain(reqs, served_last):
    """The plain form of the serving workload: the same request stream served
    one request at a time in arrival order, each a transform and one
    neat_forward launch per step with the server's observations
    (neat_fill_normal), no two requests in one launch.  Latency counts from
    the request's scheduled arrival, so it includes the wait behind earlier
    requests."""
    import collections
    import concurrent.futures as cf

    import torch
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    pool = cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1))
    window = collections.deque()
    nxt, lat, gf, same = 0, [], 0, True
    with ClockSampler(0) as clocks:
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            while nxt < len(reqs) and nxt < i + 48:
                window.append(pool.submit(W.request_population_fast, reqs[nxt]))
                nxt += 1
            p = window.popleft().result()
            dt = r["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            d = neat.dims(p.num_inputs, p.num_outputs, p.max_nodes, p.max_conns)
            rec, _ = neat.neat_transform(torch.from_numpy(p.nodes).to(dev), torch.from_numpy(p.conns).to(dev), d,
                                         stream=stream)
            B = r["batch"]
            obs = torch.empty(p.pop * B * p.num_inputs, device=dev)
            y = torch.empty((p.pop, B, p.num_outputs), device=dev)
            L = neat.neat_default_launch(p.pop, d, B)
            for st in range(r["steps"]):
                neat.neat_fill_normal(r["seed"], st, obs, stream=stream)
                neat.neat_forward(rec, p.pop, d, obs.view(p.pop, B, p.num_inputs), y, launch=L, stream=stream)
            torch.cuda.synchronize(dev)
            lat.append((time.perf_counter() - t0 - r["arrival_s"]) * 1e3)
            gf += p.pop * B * r["steps"]
            if i in served_last:
                same = same and bool(torch.equal(y, served_last[i]))
        wall = time.perf_counter() - t0
    pool.shutdown()
    return {"latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
            "genome_forwards_per_s": gf / wall, "requests": len(reqs), "wall_s": wall,
            "outputs_equal_served": same, "compared_with_served": len(served_last),
            "form": "one request at a time in arrival order: neat_transform, then one neat_forward launch per "
                    "step (observations from neat_fill_normal); latency from the scheduled arrival",
            "clocks": clocks.summary()}


def oracle_cores(fn, n_items, chunks_per_core=4):
    """Time fn(idx) over all host cores (threads; the oracle releases the GIL
    inside its C calls) on index chunks covering range(n_items); returns
    (seconds, cores)."""
    import concurrent.futures as cf
    cores = os.cpu_count() or 1
    chunks = [c for c in np.array_split(np.arange(n_items), cores * chunks_per_core) if c.size]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(fn, chunks))
    return time.perf_counter() - t0, cores


def oracle_error(gpu, ref):
    """(outputs outside the tolerance, max abs error, max scaled error) of
    float outputs against FP64 references (NaN must match NaN)."""
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    nan_ref = np.isnan(ref)
    bad = int(np.sum(nan_ref != np.isnan(gpu)))
    fin = ~nan_ref & np.isfinite(ref)
    err = np.abs(gpu[fin] - ref[fin])
    scaled = err / np.maximum(1.0, np.abs(ref[fin]))
    bad += int(np.sum(~(scaled <= 1e-5)))
    return bad, (float(err.max()) if err.size else 0.0), (float(scaled.max()) if err.size else 0.0)


def issue_roofline_from_profile(fname, sources, launch_s, sms, sm_mhz):
    """The issue roofline of a kernel from a recorded ncu instruction count
    (profiles/<fname>, valid while its sources hash the same)."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    try:
        tj = json.load(open(path))
    except (OSError, ValueError):
        return None
    if tj.get("kernel_hash") != source_hash(sources) or not tj.get("warp_instructions_per_launch"):
        return None
    insts = tj["warp_instructions_per_launch"]
    peak = 4 * sms * sm_mhz * 1e6
    return {"bound": "issue", "achieved": insts / launch_s, "peak": peak, "unit": "warp instructions/s",
            "frac": insts / launch_s / peak, "instructions_per_launch": insts,
            "note": f"ncu smsp__inst_executed.sum per launch (same sources); peak = 4 schedulers x {sms} SMs x the "
                    "sampled SM clock"}


def other_configs(args):
    """The other four workloads, measured after the headline and embedded
    in its line: XOR latency, the uneven batch, the CPPN query, serving."""
    import torch
    out = {}
    small = argparse.Namespace(**vars(args))
    small.steps = max(3, min(args.steps, 10))
    for name, fn in (("xor", lambda: measure_xor(small, reps=1000)), ("batched", lambda: measure_batched(small)),
                     ("cppn", lambda: measure_cppn(small)), ("serving", lambda: measure_serving(small))):
        try:
            out[name] = fn()
        except Exception as e:                      # a failing workload is reported, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "xor":
        run_xor(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "cppn":
        run_cppn(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "recurrent":
        run_recurrent(args)
        return
    if args.workload == "distance":
        run_distance(args)
        return
    if args.workload == "evolve":
        run_evolve(args)
        return
    if args.workload == "substrate":
        run_substrate(args)
        return
    import torch
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W

    S = args.env_steps
    if args.profile:
        profile_ant(args, dev)
        return
    from paper_2404_01817_gb300.shard import job_throughput, max_over_ranks, population_seed
    pop = W.ant_population(population_seed(rank), POP)     # each rank evaluates its own population
    d = neat.dims(I, O, NMAX, CMAX)
    nodes = torch.from_numpy(pop.nodes).to(dev)
    conns = torch.from_numpy(pop.conns).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + rank)
    obs = torch.randn((S, POP, 1, I), device=dev, generator=gen)
    act = torch.empty((S, POP, 1, O), device=dev)
    rec = torch.empty(neat.neat_transformed_bytes(POP, d), dtype=torch.uint8, device=dev)
    status = torch.empty(POP, dtype=torch.int32, device=dev)
    lanes = torch.empty(neat.neat_lanes_bytes(POP, d), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cache = neat.LanesCache()
    L_plain = neat.neat_default_launch(POP, d, 1)

    # the lane programs' shared-memory reservation per block, chosen once
    # before the timed region by neat_lanes_tune (graphs of 64 steps timed at
    # each number of blocks per SM); every later pack of the same genomes
    # gives the same programs
    neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
    neat.neat_lanes_pack(rec, POP, d, lanes=lanes, stream=stream)
    torch.cuda.synchronize(dev)
    info = neat.neat_lanes_query(lanes)
    stage = args.stage_bytes or neat.neat_lanes_tune(lanes, POP, d, obs, act, stream=stream)

    def episode_batched():
        neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
        neat.neat_lanes_pack(rec, POP, d, lanes=lanes, stream=stream)
        neat.neat_forward_lanes_steps(lanes, POP, d, obs, act, cache, stage_bytes=stage, stream=stream)

    def episode_plain(step_events=None):
        neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
        for s in range(S):
            if step_events is not None:
                step_events[s][0].record(stream)
            neat.neat_forward(rec, POP, d, obs[s], act[s], launch=L_plain, stream=stream)
            if step_events is not None:
                step_events[s][1].record(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- warm-up (also builds the CUDA graph)
    for _ in range(args.warmup):
        episode_batched()
    episode_plain()
    barrier()
    assert int((status.cpu() & 0xFF).sum()) == 0

    # ---- batched: the headline
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    fw_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    with ClockSampler(local_rank) as clocks:
        barrier()
        ev0.record(stream)
        for k in range(args.steps):
            ep_events[k][0].record(stream)
            neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
            neat.neat_lanes_pack(rec, POP, d, lanes=lanes, stream=stream)
            fw_events[k][0].record(stream)
            neat.neat_forward_lanes_steps(lanes, POP, d, obs, act, cache, stage_bytes=stage, stream=stream)
            fw_events[k][1].record(stream)
            ep_events[k][1].record(stream)
        ev1.record(stream)
        barrier()
    t_batched = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dev)
    ep_ms = [a.elapsed_time(b) for a, b in ep_events]
    fw_ms = [a.elapsed_time(b) for a, b in fw_events]
    value = job_throughput(POP * S * args.steps, world, t_batched)

    # ---- plain: one launch per step from the host, per-step latency
    n_plain = max(1, min(args.steps, 5))
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(S)]
    step_ms = []
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(n_plain):
        episode_plain(step_ev)
        torch.cuda.synchronize(dev)
        step_ms += [a.elapsed_time(b) for a, b in step_ev]
    p1.record(stream)
    barrier()
    t_plain = max_over_ranks(p0.elapsed_time(p1) / 1e3, dev)
    value_plain = world * POP * S * n_plain / t_plain

    # ---- end to end through the C ABI: host genome tensors and observations
    # in, actions out, every episode.  The episode is cut into chunks (a short
    # first one, so compute starts early).  Uploads run on one copy stream,
    # downloads on another, so that the two directions overlap each other and
    # the compute: chunk c's observations upload as soon as the previous
    # episode's chunk-c forward has read its buffer (uploads keep running
    # ahead, across episodes), chunk c's forward waits for its upload and for
    # the previous episode's download of its action buffer, and chunk c's
    # actions download behind its forward.
    nodes_h = torch.from_numpy(pop.nodes).pin_memory()
    conns_h = torch.from_numpy(pop.conns).pin_memory()
    obs_h = obs.cpu().pin_memory()
    act_h = torch.empty(act.shape, dtype=torch.float32).pin_memory()
    bounds = [0, min(S, 10)] + [b for b in range(100, S, 100) if b > min(S, 10)] + [S]
    bounds = sorted(set(bounds))
    CH = len(bounds) - 1
    chunk_caches = [neat.LanesCache() for _ in range(CH)]
    up_stream = torch.cuda.Stream(dev)
    down_stream = torch.cuda.Stream(dev)
    prev_fwd = [None] * CH       # the previous episode's chunk-c forward (done reading obs chunk c)
    prev_dl = [None] * CH        # the previous episode's chunk-c download (done reading act chunk c)
    prev_tr = [None]             # the previous episode's transform (done reading the genome tensors)

    def episode_e2e():
        ev_gen, ev_tr = torch.cuda.Event(), torch.cuda.Event()
        ev_in = [torch.cuda.Event() for _ in range(CH)]
        ev_done = [torch.cuda.Event() for _ in range(CH)]
        ev_dl = [torch.cuda.Event() for _ in range(CH)]
        with torch.cuda.stream(up_stream):
            # the genomes first, then the observations chunk by chunk
            if prev_tr[0] is not None:
                up_stream.wait_event(prev_tr[0])
            nodes.copy_(nodes_h, non_blocking=True)
            conns.copy_(conns_h, non_blocking=True)
            ev_gen.record(up_stream)
            for c in range(CH):
                if prev_fwd[c] is not None:
                    up_stream.wait_event(prev_fwd[c])
                lo, hi = bounds[c], bounds[c + 1]
                obs[lo:hi].copy_(obs_h[lo:hi], non_blocking=True)
                ev_in[c].record(up_stream)
        stream.wait_event(ev_gen)
        neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
        ev_tr.record(stream)
        prev_tr[0] = ev_tr
        neat.neat_lanes_pack(rec, POP, d, lanes=lanes, stream=stream)
        for c in range(CH):
            lo, hi = bounds[c], bounds[c + 1]
            stream.wait_event(ev_in[c])
            if prev_dl[c] is not None:
                stream.wait_event(prev_dl[c])
            neat.neat_forward_lanes_steps(lanes, POP, d, obs[lo:hi], act[lo:hi], chunk_caches[c], stage_bytes=stage,
                                          stream=stream)
            ev_done[c].record(stream)
        with torch.cuda.stream(down_stream):
            for c in range(CH):
                lo, hi = bounds[c], bounds[c + 1]
                down_stream.wait_event(ev_done[c])
                act_h[lo:hi].copy_(act[lo:hi], non_blocking=True)
                ev_dl[c].record(down_stream)
        for c in range(CH):
            prev_fwd[c] = ev_done[c]
            prev_dl[c] = ev_dl[c]
        return ev_dl[CH - 1]

    last = episode_e2e()
    stream.wait_event(last)
    torch.cuda.synchronize(dev)
    n_e2e = max(1, min(args.steps, 10))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_e2e):
        last = episode_e2e()
    stream.wait_event(last)                  # every action download of every episode is inside
    e1.record(stream)
    barrier()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    for cc in chunk_caches:
        cc.close()
    h2d = nodes_h.numel() * 4 + conns_h.numel() * 4 + obs_h.numel() * 4
    d2h = act_h.numel() * 4

    # the host link on this machine, now: one episode's uploads and its downloads,
    # each direction timed alone (best of 3); the two overlap in the episodes,
    # so the slower one sets the end-to-end floor
    def copy_s(pairs, st):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        with torch.cuda.stream(st):
            for dst, src in pairs:
                dst.copy_(src, non_blocking=True)
        b.record(st)
        b.synchronize()
        return a.elapsed_time(b) / 1e3
    t_up = min(copy_s([(nodes, nodes_h), (conns, conns_h), (obs, obs_h)], up_stream) for _ in range(3))
    t_dn = min(copy_s([(act_h, act)], down_stream) for _ in range(3))
    link_floor = world * POP * S / max(t_up, t_dn)

    # ---- roofline of the forward kernel: algorithmic bytes per launch
    alg_bytes, n_nodes, n_edges = genome_forward_bytes(pop)
    hdr = rec.view(POP, -1)[:, :32].cpu().numpy().view(np.uint32)
    record_bytes = int(hdr[:, 4].astype(np.int64).sum())                  # used bytes of every record
    program_bytes = lane_program_bytes(lanes, info)
    fwd_launch_s = statistics.mean(fw_ms) / 1e3 / S                      # per forward, graph-amortised
    achieved = alg_bytes / fwd_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = l2_traffic = warp_insts = None
    prof = os.path.join(ROOT, "profiles", "lanes_ant_traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            if tj.get("kernel_hash") == kernel_hash():
                traffic = tj.get("dram_bytes_per_launch")
                l2_traffic = tj.get("l2_bytes_per_launch")
                warp_insts = tj.get("warp_instructions_per_launch")
        except (OSError, ValueError):
            pass

    # ---- fused multi-step variant, reported beside the headline (not as it):
    # the synthetic observations do not depend on the actions, so every
    # step's inputs are known in advance and one launch runs the episode
    # with each genome's record held in shared memory
    L_fused = neat.neat_default_launch(POP, d, 1)
    order = neat.neat_schedule(rec, POP, d, stream=stream)
    L_fused.order_dev = order.data_ptr()

    def episode_fused():
        neat.neat_transform(nodes, conns, d, rec, status, stream=stream)
        neat.neat_schedule(rec, POP, d, order, stream=stream)
        neat.neat_forward_fused(rec, POP, d, obs, act, launch=L_fused, stream=stream)

    episode_fused()
    torch.cuda.synchronize(dev)
    n_fused = max(1, min(args.steps, 5))
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(n_fused):
        episode_fused()
    f1.record(stream)
    barrier()
    t_fused = max_over_ranks(f0.elapsed_time(f1) / 1e3, dev)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batched / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "l2": "inputs larger than L2 (1.08 GB of observations per bench step)",
                   "form": "batched: lane programs (neat_lanes_pack once per episode), the 1000 steps as one CUDA "
                           "graph with programmatic dependent launch (neat_forward_lanes_steps)",
                   "launch": {"warps": info.warps, "threads_per_block": 32, "genomes_per_warp": 16,
                              "stage_bytes": stage, "largest_program_bytes": info.max_warp_bytes,
                              "stage_bytes_from": "--stage-bytes" if args.stage_bytes else
                              "neat_lanes_tune (untimed, before the warm-up)"}},
        "plain": {"value": value_plain, "unit": UNIT, "episodes": n_plain,
                  "step_p50_ms": float(np.percentile(step_ms, 50)), "step_p99_ms": float(np.percentile(step_ms, 99)),
                  "form": "one neat_forward launch per step from the host (level-walk kernel)"},
        "latency_ms": {"episode_p50": float(np.percentile(ep_ms, 50)), "episode_p99": float(np.percentile(ep_ms, 99)),
                       "step_mean_batched": statistics.mean(fw_ms) / S},
        "e2e": {"value": world * POP * S * n_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": n_e2e,
                "form": f"pinned host genomes and observations in, actions out, every episode (transform, lane "
                        f"compile, forwards); {CH} chunks (the first {bounds[1]} steps, then up to 100): uploads run "
                        "ahead of the graphs on their own copy stream, across episodes (a chunk's waits for the "
                        "previous episode's forward of it), downloads behind on another; copy-bound: see link",
                "link": {"h2d_gbs": h2d / t_up / 1e9, "d2h_gbs": d2h / t_dn / 1e9, "floor": link_floor,
                         "frac_of_floor": world * POP * S * n_e2e / t_e2e / link_floor,
                         "note": "one episode's uploads and downloads, each direction timed alone on this box right "
                                 "after the e2e episodes (best of 3); floor = genome-forwards per episode over the "
                                 "slower direction's time"}},
        "fused_multistep": {"value": world * POP * S * n_fused / t_fused, "unit": UNIT, "episodes": n_fused,
                            "us_per_step": t_fused / n_fused / S * 1e6,
                            "form": "one launch per episode (neat_forward_fused, level-walk kernel), records read "
                                    "once; valid only because the synthetic observations ignore the actions, so not "
                                    "the headline"},
        "gpu_launches": args.steps * (4 + S),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "l2_traffic": l2_traffic,
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "kernel": "lanes_kernel (batched form, per launch, graph-amortised)",
                     "alg_bytes_per_launch": alg_bytes,
                     "alg_bytes_rule": "per genome 16 B x present nodes + 6 B x enabled connections, + 4 B x "
                                       "(inputs + outputs); counted from the generated tensors",
                     "present_nodes": n_nodes, "enabled_connections": n_edges,
                     "program_bytes_per_launch": program_bytes,
                     "record_bytes": record_bytes,
                     "l2_traffic_over_alg": (l2_traffic / alg_bytes) if l2_traffic else None},
        "clocks": clocks.summary(),
    }
    # the walk is latency-bound: the same launch against the SMs' issue
    # capacity (one warp instruction per cycle per scheduler, four schedulers
    # per SM, at the SM clock sampled during the timed region)
    if warp_insts:
        sm_mhz = line["clocks"].get("sm_mhz") or line["clocks"].get("sm_max_mhz")
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        if sm_mhz:
            issue_peak = 4 * sms * sm_mhz * 1e6
            issue_achieved = warp_insts / fwd_launch_s
            line["issue_roofline"] = {
                "bound": "issue", "achieved": issue_achieved, "peak": issue_peak, "unit": "warp instructions/s",
                "frac": issue_achieved / issue_peak, "instructions_per_launch": warp_insts,
                "note": "warp instructions per launch from ncu (smsp__inst_executed.sum, same kernel source); peak = "
                        f"4 schedulers x {sms} SMs x the sampled SM clock"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pop, obs.cpu().numpy())
    cache.close()
    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = other_configs(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def profile_ant(args, dev):
    """A short Ant case for ncu: transform, lane-program compile, four single
    lane forwards, then an 8-step lane graph (no timing).  Launch order:
    transform, the three compile kernels, lanes_kernel x 4, then the graph's
    eight lanes_kernel launches.  The single forwards read other
    observations than the graph's, and the observations' dirty lines are
    written back (a read of a buffer larger than L2) before any lane forward,
    so that each graph launch reads its inputs from HBM and its DRAM
    counters hold its own traffic only."""
    import torch
    from paper_2404_01817_gb300 import neat
    from paper_2404_01817_gb300 import workloads as W
    pop = W.ant_population(0, POP)
    d = neat.dims(I, O, NMAX, CMAX)
    rec, st = neat.neat_transform(torch.from_numpy(pop.nodes).to(dev), torch.from_numpy(pop.conns).to(dev), d)
    lanes = neat.neat_lanes_pack(rec, POP, d)
    torch.cuda.synchronize(dev)
    info = neat.neat_lanes_query(lanes)
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    flush = torch.ones(96 << 20, device=dev)                  # 384 MB, allocated before the observations
    x = torch.randn((12, POP, 1, I), device=dev, generator=gen)
    y = torch.empty((12, POP, 1, O), device=dev)
    float(flush.sum())                                         # evicts (writes back) the observations' lines
    for s in range(4):
        neat.neat_forward_lanes(lanes, POP, d, x[8 + s], y[8 + s], stage_bytes=info.max_warp_bytes)
    cache = neat.LanesCache()
    neat.neat_forward_lanes_steps(lanes, POP, d, x[:8], y[:8], cache, stage_bytes=info.max_warp_bytes)
    torch.cuda.synchronize(dev)
    cache.close()
    print(json.dumps({"profile": "ant", "warps": info.warps, "stage_bytes": info.max_warp_bytes,
                      "program_bytes": lane_program_bytes(lanes, info)}), flush=True)


def lane_program_bytes(lanes, info) -> int:
    """Bytes of every warp program of a packed lanes buffer (what the forward
    stages per launch)."""
    raw = lanes[:256].cpu().numpy().view(np.uint64)
    base, stride = int(raw[2]), int(raw[3])
    total = 0
    heads = lanes[base:base + stride * info.warps].view(info.warps, stride)[:, :16].cpu().numpy().view(np.uint32)
    total = int(heads[:, 1].astype(np.int64).sum())
    return total


def source_hash(files) -> str:
    import hashlib
    h = hashlib.sha1()
    for fn in files:
        with open(os.path.join(ROOT, "paper_2404_01817_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def kernel_hash() -> str:
    return source_hash(("neat_lanes.cu", "neat_device.cuh", "neat_internal.h", "neat_item.cuh"))


if __name__ == "__main__":
    main()
