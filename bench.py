#!/usr/bin/env python
"""Throughput of the PercIS estimator on GB300 (one JSON line on stdout).

A step is one complete estimate through the library's C ABI -- load the
CSR (validation, in-adjacency, VertexDiamUB), set the states (sort,
Algorithm 2 tables, C_v, lambda), phase 1 (l1 samples), the Theorem 1
bound, phase 2 (l samples) and the final estimate.  The metric is sampled
pairs per second (l1 + l per step over the device time of the step) with
the inputs resident in HBM.

Default workload: directed R-MAT scale 22 (4,194,304 vertices, edge factor
16, a=0.57 b=0.19 c=0.19, self-loops and duplicates removed, ids permuted),
x ~ Beta(0.5, 2), eps = 0.01, delta = 0.1, timed in the bidirectional form
(Section III-B).  Reported beside it: the plain and batched forms on the
same graph, the differentiated step, the end-to-end figure through host
buffers, GTEPS, the roofline of the dominant kernel, the CPU oracle (same
bidirectional algorithm) on a bounded sample, and three more workloads:
Barabasi-Albert n=100,000 with a 10% outbreak (eps = 0.005), Barabasi-Albert
n=200,000 forward + backward (eps = 0.01), and 512 uneven graphs forward +
backward (eps = 0.01 per graph).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

N > 1 runs under torchrun, one rank per GPU, each rank an independent
estimate (its own seeds; weak scaling, no collective on the data path).
--impl reference times the CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat22_beta": {
        "workload": "rmat22_beta",
        "graph": "R-MAT scale 22 (n=4194304), edge factor 16, a=0.57 b=0.19 c=0.19, directed, self-loops and "
                 "duplicates removed, ids permuted; int64 row offsets / int32 columns",
        "states": "x ~ Beta(0.5, 2)", "eps": 0.01, "delta": 0.1},
    "rmat20_beta": {
        "workload": "rmat20_beta",
        "graph": "R-MAT scale 20 (n=1048576), edge factor 16, a=0.57 b=0.19 c=0.19, directed, self-loops and "
                 "duplicates removed, ids permuted; the scale-22 workload's generator at a quarter of its size",
        "states": "x ~ Beta(0.5, 2)", "eps": 0.01, "delta": 0.1},
    "ba100k_outbreak": {
        "workload": "ba100k_m5_outbreak10",
        "graph": "Barabasi-Albert n=100000, m=5, undirected, int64 row offsets / int32 columns",
        "states": "x=0 on 90% of vertices, U[0.5,1] on a seeded random 10%", "eps": 0.005, "delta": 0.1},
    "ba200k_uniform": {
        "workload": "ba200k_m4_uniform",
        "graph": "Barabasi-Albert n=200000, m=4, undirected", "states": "x ~ U[0,1]", "eps": 0.01,
        "delta": 0.1},
}
DEFAULT_WORKLOAD = "rmat22_beta"
# DRAM traffic per launch of the dominant kernel from an ncu capture, valid only
# for the kernel source it was taken on (sha256 of the .cu file) and the workload.
NCU_TRAFFIC = {
    # one phase-2 pass (first pass + heavy pass) of a warm-up estimate: 1.022 GB read + 0.254 GB written
    ("rmat22_beta", "bibfs.cu"): {"sha256": "f0b7f101d1fd218f480f96be6b1301e4e79c9c902a692ce54032a0b89f61ebd2",
                                  "bytes_per_unit": 1.276e9},
}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def _sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.window = None

    def start(self):
        """Starts sampling every 25 ms and returns once the first sample is in."""
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def mark(self, t0: float, t1: float):
        """The timed region in host wall-clock seconds: samples outside it are dropped."""
        self.window = (t0, t1)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                except (ValueError, IndexError):
                    ts = None
                try:
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = rows
        if self.window and all(r[0] is not None for r in rows):
            t0, t1 = self.window
            inside = [r for r in rows if t0 - 0.03 <= r[0] <= t1 + 0.03]
            if not inside:  # a region shorter than the interval: the first sample after it began
                later = [r for r in rows if r[0] >= t0 - 0.03]
                inside = later[:1]
        sm = [r[1] for r in inside]
        smax = [r[2] for r in inside]
        reasons = {nm for r in inside for nm, val in zip(names, r[3]) if val.lower().startswith("active")}
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU oracle arms

def _save_workload(name: str, d: str):
    """The workload's CSR and states as .npy files, so host worker processes
    map them instead of regenerating the graph."""
    import numpy as np

    from paper_2509_11454_gb300 import synth

    g, x, eps, delta = synth.workload(name, 0)
    np.save(os.path.join(d, "rp.npy"), g.row_ptr)
    np.save(os.path.join(d, "col.npy"), g.col)
    np.save(os.path.join(d, "x.npy"), x)
    with open(os.path.join(d, "meta.json"), "w") as f:
        json.dump({"n": g.n, "directed": bool(g.directed)}, f)


def _load_oracle_workload(d: str):
    import numpy as np

    import oracle
    from paper_2509_11454_gb300 import synth

    with open(os.path.join(d, "meta.json")) as f:
        meta = json.load(f)
    g = synth.Graph(n=meta["n"], row_ptr=np.load(os.path.join(d, "rp.npy")),
                    col=np.load(os.path.join(d, "col.npy")), directed=meta["directed"])
    x = np.load(os.path.join(d, "x.npy"))
    return oracle.from_synth(g), oracle.prepare(x)


def _oracle_worker(args):
    """One host process: the oracle on phase-2 samples i0, i0 + stride, ... (in
    chunks) for budget_s seconds; bidir picks the bidirectional RandomSP."""
    d, i0, stride, budget_s, bidir, chunk = args
    sys.path.insert(0, ROOT)
    import oracle

    og, prep = _load_oracle_workload(d)
    done, t_used, k = 0, 0.0, 0
    while t_used < budget_s:
        t0 = time.perf_counter()
        oracle.run_samples(og, prep, 0, 1, 3, (i0 + k * stride) * chunk, chunk, keep_paths=False, bidir=bidir)
        t_used += time.perf_counter() - t0
        done += chunk
        k += 1
    return done, t_used


def cpu_baseline(name: str, bidir: bool, budget_s: float = 10.0) -> dict:
    """The CPU oracle as it stands (Algorithm 2 sampler + RandomSP + estimator)
    on a bounded sample of phase-2 pairs of the same workload and the same
    RandomSP algorithm as the timed GPU form: one host thread, then one
    process per host core (spawned, each mapping the saved graph)."""
    import multiprocessing as mp

    algo = "bidirectional BFS" if bidir else "one-sided truncated sigma-BFS"
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory(prefix="percis_bench_") as d:
        _save_workload(name, d)
        chunk = 20
        done1, t1 = _oracle_worker((d, 0, 1, budget_s, bidir, chunk))
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(d, c, cores, budget_s / 2, bidir, chunk) for c in range(cores)])
    done_all = sum(r[0] for r in res)
    t_all = max(r[1] for r in res)
    return {"value": done_all / t_all, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "algorithm": f"RandomSP by {algo}",
            "sample": f"{done_all} phase-2 pairs of the same workload (Algorithm 2 sampler, RandomSP by {algo}, "
                      f"estimator) split over {cores} processes, {t_all:.1f} s each",
            "single_thread": {"value": done1 / t1, "cores": 1,
                              "sample": f"{done1} pairs, {t1:.1f} s on one host thread"}}


def replica_seed_base(rank: int) -> int:
    """Each replica draws its own Philox streams (seeds far apart per rank)."""
    return 1_000_003 * rank


def job_totals(t_local: float, pairs_local: int, dist, device: str):
    """Whole-job time (max over ranks) and pairs (sum over ranks); replicas
    exchange nothing else."""
    if dist is None:
        return t_local, float(pairs_local)
    import torch

    tt = torch.tensor([t_local, float(pairs_local)], dtype=torch.float64, device=device)
    tmax = tt.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tt[1])


def run_reference(args):
    """The reference arm: the CPU oracle (bidirectional RandomSP, as the timed
    GPU form) on a bounded sample of the workload per step, one host thread."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    bidir = args.form == "bidir"
    with tempfile.TemporaryDirectory(prefix="percis_ref_") as d:
        _save_workload(args.workload, d)
        og, prep = _load_oracle_workload(d)
    per_step = args.ref_pairs
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.run_samples(og, prep, 1000 + k, 1, 3, 0, per_step, keep_paths=False, bidir=bidir)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot
    algo = "bidirectional BFS" if bidir else "one-sided truncated sigma-BFS"
    line = {"impl": "reference", "metric": "sampled pairs/s", "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(WORKLOADS[args.workload]),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} phase-2 pairs per step (RandomSP by {algo}) on one host thread"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU helpers

def _timed(torch, stream, flush, fn):
    """Device time (s) of fn() on `stream`, L2 flushed before it."""
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1000.0, out


def extra_workload(binding, synth, torch, stream, flush, name: str, steps: int, warmup: int, backward: bool,
                   seed_base: int) -> dict:
    """pairs/s of another single-graph workload (bidirectional form), forward
    or forward + backward per step, inputs resident in HBM."""
    g, x, eps, delta = synth.workload(name, 0)
    eng = binding.PercIS(torch.cuda.current_device())
    eng.set_options(form="bidir")
    rp_d = torch.as_tensor(g.row_ptr, dtype=torch.int64, device="cuda")
    col_d = torch.as_tensor(g.col, dtype=torch.int32, device="cuda")
    x_d = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    pc_d = torch.empty(g.n, dtype=torch.float64, device="cuda")
    gvec = torch.randn(g.n, dtype=torch.float64, device="cuda")
    gx = torch.empty(g.n, dtype=torch.float64, device="cuda")

    def step(seed):
        binding.percis_load_csr(eng.ctx, g.n, g.nnz, rp_d, col_d, g.directed, 1)
        binding.percis_set_states(eng.ctx, x_d, 1)
        inf = binding.percis_estimate(eng.ctx, eps, delta, seed, pc_d, 1)
        if backward:
            binding.percis_backward(eng.ctx, gvec, gx, 1)
        return inf

    for k in range(warmup):
        step(seed_base + 50_000 + k)
    ts, pairs = [], 0
    for k in range(steps):
        dt, inf = _timed(torch, stream, flush, lambda: step(seed_base + k))
        ts.append(dt)
        pairs += inf["ell1"] + inf["ell"]
    eng.close()
    return {"workload": WORKLOADS[name]["workload"], "value": pairs / sum(ts), "unit": "pairs/s",
            "ms_per_step": 1000.0 * sum(ts) / len(ts), "steps": steps, "eps": eps,
            "form": "bidirectional" + (" forward + backward (dPC/dx)" if backward else ""),
            "pairs_per_step": pairs / steps}


def extra_uneven(binding, synth, torch, stream, flush, steps: int, seed_base: int) -> dict:
    """512 independent graphs (Watts-Strogatz k=10 p=0.05, Barabasi-Albert m=3,
    grids with 5% of edges deleted; n log-uniform in [1e3, 2e5]), x ~ U[0,1],
    eps = 0.01 per graph, bidirectional form with recorded sampling launches;
    forward + backward per step."""
    sizes = synth.uneven_batch_sizes(512, 1000, 200_000, 0)
    graphs = synth.graph_batch(sizes, 0)
    vptr, rp, col = synth.union_csr(graphs)
    n = int(vptr[-1])
    x = synth.states_uniform(n, 0)
    eng = binding.PercIS(torch.cuda.current_device())
    eng.set_options(form="bidir", cuda_graphs=1)
    eng.load_graphs(vptr, rp, col)
    eng.set_states(x)
    pc = torch.empty(n, dtype=torch.float64, device="cuda")
    gvec = torch.randn(n, dtype=torch.float64, device="cuda")
    gx = torch.empty(n, dtype=torch.float64, device="cuda")

    def step(seed):
        infos = binding.percis_estimate_graphs(eng.ctx, 0.01, 0.1, seed, pc, 1)
        binding.percis_backward(eng.ctx, gvec, gx, 1)
        return infos

    def run():
        step(seed_base + 70_000)  # warm-up (records the sampling graphs)
        ts, pairs = [], 0
        for k in range(steps):
            dt, infos = _timed(torch, stream, flush, lambda: step(seed_base + k))
            ts.append(dt)
            pairs += sum(f["ell1"] + f["ell"] for f in infos)
        return pairs / sum(ts), 1000.0 * sum(ts) / len(ts), pairs / steps

    value, ms, pps = run()
    # the same batch with the options the autotuner picks on probe phases (not timed)
    t0 = time.time()
    o = eng.autotune(probe_samples=65536, seed=seed_base + 90_000)
    tune_s = time.time() - t0
    tv, tms, _ = run()
    eng.close()
    return {"workload": "uneven512_ws_ba_grid", "value": value, "unit": "pairs/s",
            "ms_per_step": ms, "steps": steps, "graphs": 512, "n": n,
            "nnz": int(col.shape[0]), "eps": 0.01,
            "form": "bidirectional, sampling launches in CUDA graphs, forward + backward (dPC/dx)",
            "pairs_per_step": pps,
            "tuned": {"value": tv, "ms_per_step": tms, "tuning_s": tune_s,
                      "options": {k: o[k] for k in ("bi_heavy_edges", "bi_table_log", "bi_blocks_per_sm")}}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--ref-pairs", type=int, default=100)
    ap.add_argument("--no-extras", action="store_true", help="only the headline and its roofline")
    ap.add_argument("--no-other-workloads", action="store_true", help="skip the extra workloads")
    ap.add_argument("--form", default="bidir", choices=["bidir", "batched"],
                    help="form of the timed step: bidirectional BFS per sample, or the batched multi-source BFS")
    ap.add_argument("--lanes", type=int, default=0, help="batched lane width (0 = library default)")
    ap.add_argument("--lane-order", type=int, default=-1, help="0 = by vertex id, 1 = by hub neighbour")
    ap.add_argument("--direction", type=int, default=-1, help="0 = pull, 1 = push, 2 = by work estimate")
    ap.add_argument("--push-alpha", type=float, default=0.0)
    ap.add_argument("--bi-table-log", type=int, default=0, help="bidirectional store (0 = library default)")
    ap.add_argument("--bi-table-max-log", type=int, default=0)
    ap.add_argument("--bi-heavy-edges", type=int, default=0, help="heavy-level threshold (0 = default, <0 = off)")
    ap.add_argument("--bi-scratch-gib", type=int, default=0, help="direct-store budget, GiB (0 = default)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2509_11454_gb300 import binding, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load_library()

    wl = WORKLOADS[args.workload]
    g, x, eps, delta = synth.workload(args.workload, 0)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    eng = binding.PercIS(local)
    eng.set_options(form=args.form)
    if args.lanes:
        eng.set_options(lanes=args.lanes)
    if args.lane_order >= 0:
        eng.set_options(lane_order=args.lane_order)
    if args.direction >= 0:
        eng.set_options(direction=args.direction)
    if args.push_alpha > 0:
        eng.set_options(push_alpha=args.push_alpha)
    eng.set_options(bi_table_log=args.bi_table_log, bi_table_max_log=args.bi_table_max_log,
                    bi_heavy_edges=args.bi_heavy_edges, bi_scratch_gib=args.bi_scratch_gib)
    rp_d = torch.as_tensor(g.row_ptr, dtype=torch.int64, device="cuda")
    col_d = torch.as_tensor(g.col, dtype=torch.int32, device="cuda")
    x_d = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    pc_d = torch.empty(g.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    seed_base = replica_seed_base(rank)

    def step(seed):
        binding.percis_load_csr(eng.ctx, g.n, g.nnz, rp_d, col_d, g.directed, 1)
        binding.percis_set_states(eng.ctx, x_d, 1)
        return binding.percis_estimate(eng.ctx, eps, delta, seed, pc_d, 1)

    for k in range(args.warmup):
        step(seed_base + 10_000 + k)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    infos, times = [], []
    clocks.start()
    launches0 = binding.percis_launch_count(eng.ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for k in range(args.steps):
        dt, inf = _timed(torch, stream, flush, lambda: step(seed_base + k))  # L2 flushed before every step
        times.append(dt)
        infos.append(inf)
    torch.cuda.synchronize()
    clocks.mark(t_wall0, time.time())
    clk = clocks.stop()
    launches = binding.percis_launch_count(eng.ctx) - launches0
    t_total = sum(times)
    pairs = sum(i["ell1"] + i["ell"] for i in infos)
    t_job, pairs_job = job_totals(t_total, pairs, dist, "cuda")
    value = pairs_job / t_job

    extras = {}
    if rank == 0:
        peaks, peak_kind = _peaks()
        replay_steps = min(args.steps, 3)

        # algorithmic work of the same estimates, counted in an untimed instrumented replay
        def replay(form):
            eng.set_options(instrument=1, form=form)
            work = np.zeros((2, 8))
            for k in range(replay_steps):
                inf = step(seed_base + k)
                work += np.array(inf["work"], dtype=np.float64)
            eng.set_options(instrument=0, form=args.form)
            return work

        work = replay(args.form)
        w = work.sum(axis=0)
        wb = w if args.form == "batched" else replay("batched").sum(axis=0)
        step_s_replayed = sum(times[:replay_steps])
        bfs_share = sum(sum(i["bfs_ms"]) for i in infos) / 1000.0 / t_total
        if args.form == "batched":
            kernel, src_name = ("k_msbfs (batched sigma-BFS + backtrack; one persistent launch per phase, "
                                "figures per batch of W lanes)", "msbfs.cu")
            algo_bytes = 8.0 * w[0] + 8.0 * w[1] + 8.0 * w[2] + 4.0 * w[3]
            bfs_ms = sum(sum(i["bfs_ms"]) for i in infos[:replay_steps])
            bfs_launches = sum(sum(i["bfs_launches"]) for i in infos[:replay_steps])
            work_step = {"sigma_dag_reads": w[0], "sigma_writes": w[1], "union_frontier_rows": w[2],
                         "union_frontier_edges": w[3], "truncated_bfs_edges": w[4], "bfs_samples": w[6]}
            scanned = w[3]
        else:
            kernel, src_name = ("k_bibfs (bidirectional sigma-BFS + backtrack, one block per sample; "
                                "figures per phase-2 pass: the first-pass launch and the heavy-pass launch)",
                                "bibfs.cu")
            # Byte model of the per-pair work: per edge scanned the column (4 B); per
            # vertex reached its row offsets (8 B) and its level and count written
            # (12 B); per count addition (an edge into the next level) the count read
            # (8 B).  The store's own model, reported beside it, adds what the kernel
            # must also move: per edge the level word read at the far end (8 B), per
            # vertex the queue entry (4 B) and the count read back by the meeting and
            # the backtrack (8 B).  The unit is the phase-2 pass (one per step, most of
            # the samples): the first-pass launch and, when samples were handed over,
            # the heavy-pass launch, timed together by the library's events.
            w2 = work[1]
            algo_bytes = 4.0 * w2[0] + 20.0 * w2[2] + 8.0 * w2[1]
            store_bytes = 12.0 * w2[0] + 8.0 * w2[1] + 28.0 * w2[2]
            bfs_ms = sum(i["bfs_ms"][1] for i in infos[:replay_steps])
            bfs_launches = sum(i["bfs_launches"][1] for i in infos[:replay_steps])
            work_step = {"edges_scanned": w[0], "count_additions": w[1], "vertices_reached": w[2],
                         "bfs_samples": w[3] % (1 << 32), "meeting_layers_above_256": w[3] // (1 << 32),
                         "handed_over_samples": w[4], "one_sided_bfs_edges": wb[4]}
            scanned = w[0]
        units = bfs_launches if args.form == "batched" else replay_steps
        per_unit_bytes = algo_bytes / max(units, 1)
        per_unit_s = bfs_ms / 1000.0 / max(units, 1)
        achieved = per_unit_bytes / per_unit_s / 1e9
        traffic = None
        ncu = NCU_TRAFFIC.get((args.workload, src_name))
        if ncu and ncu["sha256"] == _sha(os.path.join(ROOT, "paper_2509_11454_gb300", "csrc", src_name)):
            traffic = ncu["bytes_per_unit"]
        extras["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kernel,
                              "peak_source": f"{peak_kind} HBM copy bandwidth",
                              "work_unit": "batch launch" if args.form == "batched" else "phase-2 pass",
                              "algorithmic_bytes_per_unit": per_unit_bytes,
                              "avg_unit_ms": per_unit_s * 1000.0,
                              "launches_per_step": bfs_launches / replay_steps}
        if args.form != "batched":
            sb = store_bytes / max(units, 1)
            extras["roofline"]["store_model"] = {
                "bytes_per_unit": sb, "achieved": sb / per_unit_s / 1e9,
                "frac": sb / per_unit_s / 1e9 / peaks["hbm_gbs"],
                "note": "adds per edge the level word read (8 B), per vertex the queue entry (4 B) and the "
                        "count read back (8 B)"}
        # GTEPS two ways: the edges a one-sided truncated BFS from s_i scans to settle t_i
        # (the paper-independent work measure), and the edges the timed kernel scanned
        extras["gteps"] = wb[4] / step_s_replayed / 1e9 if wb[4] else None
        extras["gteps_scanned"] = scanned / step_s_replayed / 1e9 if scanned else None
        extras["gteps_note"] = ("gteps: one-sided truncated-BFS edges of the same pairs per second (counted in an "
                                "instrumented replay); gteps_scanned: edges the timed kernel actually scanned")
        extras["work_per_step"] = {k: v / replay_steps for k, v in work_step.items()}
        extras["bfs_share_of_step"] = bfs_share

        if not args.no_extras:
            # plain form: one BFS launch + one backtrack launch per sampled pair, on a bounded
            # sample size (l1 = l = 1000; pairs/s does not depend on l)
            eng.set_options(form="plain", ell1=1000, ell=1000)
            t_p, inf_p = _timed(torch, stream, flush, lambda: step(seed_base))
            eng.set_options(form=args.form, ell1=0, ell=0)
            extras["plain"] = {"value": (inf_p["ell1"] + inf_p["ell"]) / t_p, "unit": "pairs/s",
                               "ms_per_step": t_p * 1000.0, "steps": 1,
                               "sample": "l1 = l = 1000 (the plain form takes one launch per pair)"}

            # the other sampling form on the same seeds
            other = "batched" if args.form == "bidir" else "bidir"
            eng.set_options(form=other)
            to, po = [], 0
            for k in range(replay_steps):
                dt, inf = _timed(torch, stream, flush, lambda: step(seed_base + k))
                to.append(dt)
                po += inf["ell1"] + inf["ell"]
            eng.set_options(form=args.form)
            extras["batched" if other == "batched" else "bidirectional"] = {
                "value": po / sum(to), "unit": "pairs/s", "ms_per_step": 1000.0 * sum(to) / len(to),
                "steps": replay_steps}
            b_val = value / world if args.form == "batched" else extras["batched"]["value"]
            extras["batched_over_plain"] = b_val / extras["plain"]["value"]
            extras["headline_over_plain"] = value / world / extras["plain"]["value"]

            # differentiated form: forward + backward (dPC/dx) per step
            gvec = torch.randn(g.n, dtype=torch.float64, device="cuda")
            gx = torch.empty(g.n, dtype=torch.float64, device="cuda")
            tds, npairs = [], 0

            def fwd_bwd(seed):
                inf = step(seed)
                binding.percis_backward(eng.ctx, gvec, gx, 1)
                return inf

            for k in range(args.steps):
                dt, inf = _timed(torch, stream, flush, lambda: fwd_bwd(seed_base + k))
                tds.append(dt)
                npairs += inf["ell1"] + inf["ell"]
            extras["differentiated"] = {"value": npairs / sum(tds), "unit": "pairs/s",
                                        "ms_per_step": 1000.0 * sum(tds) / len(tds)}

            # end to end through the public API with host buffers (pinned), copies inside the timed region
            rp_h = torch.as_tensor(g.row_ptr, dtype=torch.int64).pin_memory()
            col_h = torch.as_tensor(g.col, dtype=torch.int32).pin_memory()
            x_h = torch.as_tensor(x, dtype=torch.float64).pin_memory()
            pc_h = torch.empty(g.n, dtype=torch.float64).pin_memory()
            te, pe = [], 0
            for k in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                binding.percis_load_csr(eng.ctx, g.n, g.nnz, rp_h, col_h, g.directed, 0)
                binding.percis_set_states(eng.ctx, x_h, 0)
                inf = binding.percis_estimate(eng.ctx, eps, delta, seed_base + k, pc_h, 0)
                te.append(time.perf_counter() - t0)
                pe += inf["ell1"] + inf["ell"]
            h2d = rp_h.numel() * 8 + col_h.numel() * 4 + x_h.numel() * 8
            extras["e2e"] = {"value": pe / sum(te), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                             "d2h_bytes_per_step": pc_h.numel() * 8}
            del rp_h, col_h, x_h, pc_h

            # Graph500-style full traversals: 512 sources, every reachable edge each
            src = torch.as_tensor(np.random.default_rng(7).choice(g.n, 512, replace=False).astype(np.int32),
                                  device="cuda")
            binding.percis_msbfs(eng.ctx, 512, src, None, None)
            tf = []
            for k in range(3):
                dt, _ = _timed(torch, stream, flush, lambda: binding.percis_msbfs(eng.ctx, 512, src, None, None))
                tf.append(dt)
            und = 1 if g.directed else 2
            extras["full_bfs_teps"] = {"gteps": 512 * (g.nnz // und) / min(tf) / 1e9, "sources": 512,
                                       "ms": 1000.0 * min(tf),
                                       "note": "sigma-counting BFS from 512 sources to exhaustion in one "
                                               "batched launch; every edge of the graph counted once per source "
                                               "(undirected edges once)"}
            eng.close()
            eng = None
            torch.cuda.empty_cache()

            if not args.no_other_workloads and world == 1:
                others = []
                for nm, bw in (("ba100k_outbreak", False), ("ba200k_uniform", True)):
                    if nm != args.workload:
                        others.append(extra_workload(binding, synth, torch, stream, flush, nm, 5, 3, bw,
                                                     seed_base))
                        torch.cuda.empty_cache()
                others.append(extra_uneven(binding, synth, torch, stream, flush, 2, seed_base))
                torch.cuda.empty_cache()
                extras["other_workloads"] = others
            if world == 1:
                extras["cpu_baseline"] = cpu_baseline(args.workload, bidir=args.form == "bidir")
                extras["cpu_baseline_one_sided"] = cpu_baseline(args.workload, bidir=False, budget_s=4.0)

    if rank == 0:
        i0 = infos[0]
        cfg = dict(wl)
        cfg.update({"n": g.n, "nnz": g.nnz,
                    "form": {"bidir": "bidirectional BFS per sample", "batched": "batched multi-source BFS"}[args.form],
                    "ell1": i0["ell1"],
                    "ell_mean": statistics.mean(i["ell"] for i in infos),
                    "vertex_diam": i0["vertex_diam"], "dhat": i0["dhat"],
                    "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written before every timed step",
                    "parallelism": f"replicas x{world}"})
        if args.form == "batched":
            cfg.update({"lanes": i0["lanes"],
                        "distinct_sources_phase2_mean": statistics.mean(i["sources"][1] for i in infos)})
        line = {"metric": "sampled pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_job / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg, "gpu_launches": launches, "clocks": clk}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if eng is not None:
        eng.close()


if __name__ == "__main__":
    main()
