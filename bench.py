#!/usr/bin/env python
"""Benchmark of the tvcut hot path: a cold-started AAR solve of one grid to
the iteration at which its cut first equals the exact (max-flow) minimum.

One step = cold start + k* AAR iterations (FP32 iterates, one check at the
end) + the cut, with inputs resident in HBM; k* is found once, untimed, by
checking every iteration against the oracle's min-cut value E* (computed in
the CPU-baseline leg).  value = vertices x iterations / time (Mvertex-iter/s),
summed over ranks (replicas: the single-grid path does not shard).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload volume256|seg1024]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1503_01563_gb300 import inputs  # noqa: E402

WORKLOADS = {
    # 3D 6-connected 256^3 blob volume, integer-scaled LLR unary, weights U{1..30}
    "volume256": dict(dims=(256, 256, 256), seed=3, cap=1500),
    # 2D 4-connected 1024^2 blob segmentation, integer-scaled LLR unary and contrast weights
    "seg1024": dict(dims=(1024, 1024), seed=2, cap=3000),
    # the same image on a 2D 8-connected grid (diagonal contrast weights / sqrt(2)): four blocks
    "seg1024c8": dict(dims=(1024, 1024), seed=2, cap=3000, conn=8),
    # 512 independent 2D grids, H ~ U{64..1024} x W ~ U{64..768}, w ~ U{-50..50}, a ~ U{1..20}
    "batch512": dict(grids=512, seed=4, cap=3000),
    # learned warm start: U-Net (4 levels, 32 channels) trained on solver-generated 128^2 problems,
    # evaluated on held-out 2048^2 problems (w ~ U{-50..50}, a ~ U{1..20}), cold vs warm
    "warm2048": dict(dims=(2048, 2048), seed=999, cap=3000, train_n=4096, train_hw=128, train_steps=4000),
    # the warm-start network's inference alone: U-Net (4 levels, 32 channels) on one 2048^2 input,
    # randomly initialised weights; its 3x3 convolutions are the one dense contraction of the path
    "unet2048": dict(dims=(2048, 2048), seed=21, base=32),
}
# (level, Cin, Cout) of the U-Net's 18 convolutions in forward order (level l: resolution / 2^l)
UNET_CONVS = [(0, 16, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 128), (2, 128, 128), (3, 128, 256),
              (3, 256, 256), (2, 256, 128), (2, 256, 128), (2, 128, 128), (1, 128, 64), (1, 128, 64), (1, 64, 64),
              (0, 64, 32), (0, 64, 32), (0, 32, 32), (0, 32, 16)]
FALLBACK_HBM_GBS = 6800.0


def make_problem(name):
    wl = WORKLOADS[name]
    if "grids" in wl:                 # the reference arm times the largest grid of the batch
        dims, probs = batch_problems(wl["grids"], wl["seed"])
        g = max(range(len(dims)), key=lambda i: dims[i][0] * dims[i][1])
        return probs[g]
    if name == "warm2048":
        return inputs.uniform_grid(wl["dims"], wl["seed"])
    if wl.get("conn") == 8:
        return inputs.segmentation_problem8(wl["dims"], wl["seed"])
    if len(wl["dims"]) == 3:
        return inputs.volume_problem(wl["dims"], wl["seed"])
    return inputs.segmentation_problem(wl["dims"], wl["seed"])


def kernel_bytes_per_vertex(ndim, algo="aar"):
    """Algorithmic bytes per vertex of one launch of each kernel kind (FP32
    state and weights; compact weights have dims[k]-1 entries per chain,
    counted as one per vertex).

    AAR and AP: prox (the scan launch, all blocks) reads s_k and a_k and
    writes x_k for every block; update reads w, every s_k and x_k and writes
    every s_k.  A checked iteration's update also writes the primal (+4 B).

    BCD (one block per launch): prox (the scan in projection mode) reads v_k
    and a_k and writes y_k; update (forming v_k = w - sum_{j != k} y_j) reads
    w and ndim-1 duals and writes v_k.

    FISTA: update (extrapolation and gradient step) reads w, every y_k and
    previous y_k and writes every v_k; prox (the scan in projection mode, all
    blocks) reads v_k and a_k and writes the new y_k.

    BCD and FISTA add one update-kind launch per checked iteration that reads
    w and all duals and writes the primal ("eval")."""
    if algo == "bcd":
        return {"prox": 12, "update": 4 * ndim + 4, "eval": 4 * ndim + 8, "check_extra": 0}
    if algo == "fista":
        return {"prox": 12 * ndim, "update": 4 + 12 * ndim, "eval": 4 * ndim + 8, "check_extra": 0}
    return {"prox": 12 * ndim, "update": 4 + 12 * ndim, "eval": None, "check_extra": 4}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def scan_sources_sha256():
    """Hash of the sources of the scan and update kernels (scan.cu, taut_string.cuh)."""
    h = hashlib.sha256()
    for f in ("scan.cu", "taut_string.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1503_01563_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(kind_name, workload):
    """DRAM bytes per launch of a kernel from a committed ncu summary, valid
    only while the iteration kernels' source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(workload, {}).get(kind_name)
    if ent is None or d.get("scan_sources_sha256") != scan_sources_sha256():
        return None
    return ent


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        """Start sampling every 50 ms; returns once the first sample is written
        (nvidia-smi takes a moment to start), and only samples written after
        that count, so that the median covers the timed region."""
        self.skip = 0
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0:
            with open(self.path) as f:
                n = sum(1 for _ in f)
            if n > 0:
                self.skip = n
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        if len(lines) > self.skip:
            lines = lines[self.skip:]          # samples taken during the timed region
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


ALGOS = {"aar": 0, "ap": 1, "bcd": 2, "fista": 3}


def oracle_module(a):
    import oracle
    oracle.build()
    if len(a) == 4:                    # 8-connected 2D grid
        from oracle import conn8
        return conn8
    return oracle


def exact_min_cut(w, a):
    """The oracle's exact min-cut value E* (push-relabel max-flow) and its time."""
    orc = oracle_module(a)
    t0 = time.perf_counter()
    e_star = orc.maxflow(w, a, 1)[1]
    return e_star, time.perf_counter() - t0


def cpu_leg(name, w, a, kstar, budget_s=12.0, algo="aar", t_mf=0.0):
    """The oracle (FP64, the same algorithm, its taut-string prox with OpenMP
    over chains) on the host cores.  With k* known it runs exactly k*
    iterations from the cold start, keeping the primal at k*/2 and k* for the
    FP32-vs-FP64 comparison, and is timed over them; otherwise whole-grid
    iterations until the time budget is spent."""
    orc = oracle_module(a)
    cores = os.cpu_count() or 1
    n = int(np.prod(w.shape))
    code = ALGOS[algo]
    s = orc.cold_state(code, w)
    xs = {}
    t_it, iters = 0.0, 0
    if kstar:
        marks = sorted(set([max(1, kstar // 2), kstar]))
        if algo == "fista":            # the oracle's FISTA momentum restarts per call: one call per mark
            for k in marks:
                t0 = time.perf_counter()
                _, xs[k] = orc.iterate(code, w, a, orc.cold_state(code, w), k, nthreads=cores)
                dt = time.perf_counter() - t0
                if k == kstar:
                    t_it, iters = dt, k
        else:
            done = 0
            for k in marks:
                t0 = time.perf_counter()
                s, xs[k] = orc.iterate(code, w, a, s, k - done, nthreads=cores)
                t_it += time.perf_counter() - t0
                done = k
            iters = kstar
        sample = f"{iters} FP64 {algo.upper()} iterations (k*) over the full {name} grid ({t_it:.1f} s)"
    else:
        while t_it < budget_s and iters < 200:
            t0 = time.perf_counter()
            s, _ = orc.iterate(code, w, a, s, 1, nthreads=cores)
            t_it += time.perf_counter() - t0
            iters += 1
        sample = f"{iters} FP64 {algo.upper()} iterations over the full {name} grid ({t_it:.1f} s)"
    value = n * iters / t_it / 1e6
    return xs, {"value": value, "unit": "Mvertex-iter/s", "cores": cores, "kind": "oracle",
                "sample": sample + f", OpenMP over chains; max-flow E* took {t_mf:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "unet2048":
        return run_reference_unet(args)
    import oracle
    oracle.build()
    w, a = make_problem(args.workload)
    n = int(np.prod(w.shape))
    cores = os.cpu_count() or 1
    code = ALGOS[args.algo]
    orc = oracle
    if len(a) == 4:                    # 8-connected 2D grid
        from oracle import conn8 as orc
    s = orc.cold_state(code, w)
    for _ in range(args.warmup):
        s, _ = orc.iterate(code, w, a, s, 1, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, _ = orc.iterate(code, w, a, s, 1, nthreads=cores)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e6
    out = {"impl": "reference", "metric": "Mvertex-iter/s", "value": value, "unit": "Mvertex-iter/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "dims": list(WORKLOADS[args.workload].get("dims", ())),
                      "algo": args.algo.upper(),
                      "step": f"one whole-grid {args.algo.upper()} iteration of the CPU oracle"},
           "cpu_baseline": {"value": value, "unit": "Mvertex-iter/s", "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} whole-grid FP64 {args.algo.upper()} iterations"},
           "e2e": {"value": value, "unit": "Mvertex-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_reference_unet(args):
    """The oracle's U-Net forward (PyTorch CPU FP32) on 512x512 crops of the
    2048^2 input, reported in TFLOP/s."""
    import torch
    import oracle.unet_ref as unet_ref
    wl = WORKLOADS["unet2048"]
    H, W = wl["dims"]
    hs = 512
    flops = sum(2.0 * (hs >> l) * (hs >> l) * 9 * ci * co for l, ci, co in UNET_CONVS)
    g = np.random.default_rng(wl["seed"])
    x = torch.from_numpy(g.normal(size=(1, hs, hs, 3)).astype(np.float32))
    theta = torch.from_numpy(g.normal(size=unet_ref.num_params(wl["base"])).astype(np.float32) * 0.05)
    with torch.no_grad():
        for _ in range(args.warmup):
            unet_ref.forward(theta, x, wl["base"])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            unet_ref.forward(theta, x, wl["base"])
        dt = (time.perf_counter() - t0) / args.steps
    value = flops / dt / 1e12
    out = {"impl": "reference", "metric": "TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "unet2048", "dims": [H, W], "step": f"oracle forward on a {hs}x{hs} crop"},
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": torch.get_num_threads(), "kind": "oracle",
                            "sample": f"{args.steps} oracle forwards on {hs}x{hs} crops"},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def batch_problems(G, seed):
    dims = inputs.batch_dims(G, seed)
    return dims, [inputs.uniform_grid(d, 1000 * seed + g) for g, d in enumerate(dims)]


def batch_measure(dims, probs, algo, steps, warmup, stream, e_star, sample, cap, local, dist=None):
    """The batched solve of `probs` (one handle, graph-replayed iterations):
    autotune, k* = the first multiple of 10 iterations at which every sampled
    grid's cut equals its E* (when e_star is given), `steps` timed solves with
    the L2 flushed before each, then the same grids solved one after another
    with one handle each."""
    import torch
    from paper_1503_01563_gb300 import tvcut
    dev = torch.device("cuda", torch.cuda.current_device())
    dev_probs = [(torch.from_numpy(w).to(dev), [torch.from_numpy(x).to(dev) for x in a]) for w, a in probs]
    b = tvcut.Batch(dims, algo=algo, dtype=tvcut.F32, stream=stream.cuda_stream)
    for g, (w, a) in enumerate(dev_probs):
        b.set_problem(g, w, a)
    b.reset()
    b.iterate(2)
    chosen = b.autotune()
    kstar = None
    if e_star is not None:
        b.reset()
        k = 0
        while k < cap:
            _, st = b.iterate(10)
            k += 10
            if all(st[g].energy_i64 == e_star[g] for g in sample):
                kstar = k
                break
    iters = kstar if kstar else cap
    if dist is not None:
        t = torch.tensor([iters], device=dev)
        dist.broadcast(t, 0)
        iters = int(t.item())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        b.reset()
        b.iterate(iters)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, ok = 0.0, True
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        b.reset()
        _, st = b.iterate(iters)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        if e_star is not None:
            ok = ok and all(st[g].energy_i64 == e_star[g] for g in sample)
    clk = clocks.stop()
    singles = []
    for g, (w, a) in enumerate(dev_probs):
        sv = tvcut.Solver(dims[g], algo=algo, dtype=tvcut.F32, check_every=iters, stream=stream.cuda_stream)
        sv.set_problem(w, a)
        singles.append(sv)
    for sv in singles[:8]:
        sv.reset()
        sv.iterate(iters)
    torch.cuda.synchronize()
    ev0.record(stream)
    for sv in singles:
        sv.reset()
        sv.iterate(iters)
    ev1.record(stream)
    ev1.synchronize()
    sep_ms = ev0.elapsed_time(ev1)
    for sv in singles:
        sv.close()
    b.close()
    return {"kstar": kstar, "iters": iters, "total_ms": total_ms, "ok": ok, "clocks": clk, "chosen": chosen,
            "sep_ms": sep_ms}


def run_batch(args):
    """512 uneven 2D grids: one batched solve (graph-replayed iterations) vs
    the same grids solved one after another with one handle each.  --algo:
    AAR (default), AP or FISTA (the batched solver has no BCD)."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    wl = WORKLOADS["batch512"]
    if args.algo == "bcd":
        raise SystemExit("batch512: the batched solver runs AAR, AP or FISTA")
    algo = ALGOS[args.algo]
    dims, probs = batch_problems(wl["grids"], wl["seed"])
    n_all = int(sum(h * w for h, w in dims))
    if world > 1:                      # grids share nothing: each rank solves its own shard
        from paper_1503_01563_gb300 import shard
        mine = shard.shard(dims, rank, world)
        dims = [dims[g] for g in mine]
        probs = [probs[g] for g in mine]
    G = len(dims)
    n_total = int(sum(h * w for h, w in dims))
    sample = list(range(0, G, max(1, G // 16)))
    e_star, cpu_base = {}, None
    if rank == 0:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        for g in sample:
            e_star[g] = oracle.maxflow(probs[g][0], probs[g][1], 1)[1]
        t_mf = time.perf_counter() - t0
        nv, t_it = 0, 0.0
        for g in sample:
            w, a = probs[g]
            st = oracle.cold_state(algo, w)
            t0 = time.perf_counter()
            oracle.iterate(algo, w, a, st, 5, nthreads=cores)
            t_it += time.perf_counter() - t0
            nv += 5 * w.size
            if t_it > args.cpu_budget:
                break
        cpu_base = {"value": nv / t_it / 1e6, "unit": "Mvertex-iter/s", "cores": cores, "kind": "oracle",
                    "sample": f"5 FP64 {args.algo.upper()} iterations on each of up to {len(sample)} of the 512 grids "
                              f"({t_it:.1f} s); max-flow E* of {len(sample)} sampled grids took {t_mf:.1f} s"}
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1503_01563_gb300 import tvcut
    stream = torch.cuda.current_stream(dev)
    m = batch_measure(dims, probs, algo, args.steps, args.warmup, stream, e_star if rank == 0 else None, sample,
                      wl["cap"], local, dist if world > 1 else None)
    kstar, iters, total_ms, ok, clk, chosen, sep_ms = (m["kstar"], m["iters"], m["total_ms"], m["ok"], m["clocks"],
                                                       m["chosen"], m["sep_ms"])
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n_all * iters * args.steps / (total_ms / 1e3) / 1e6     # all ranks' grids / slowest rank
    # end to end with host buffers: upload every grid, solve, read every labelling
    e2e_b = tvcut.Batch(dims, algo=algo, dtype=tvcut.F32, stream=stream.cuda_stream)
    pinned = [(torch.from_numpy(w).pin_memory(), [torch.from_numpy(x).pin_memory() for x in a]) for w, a in probs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, (w, a) in enumerate(pinned):
        e2e_b.set_problem(g, w, a)
    e2e_b.reset()
    e2e_b.iterate(iters)
    for g in range(G):
        e2e_b.cut(g)
    e2e_s = time.perf_counter() - t0
    e2e_b.close()
    h2d = int(sum(w.nbytes + sum(x.nbytes for x in a) for w, a in probs))
    iter_bytes = (24 + 28) * n_total      # scan 24 B + update (FISTA: step) 28 B per vertex
    peak, peak_kind = peaks()
    achieved = iter_bytes * iters / (ms_per_step / 1e3) / 1e9
    if rank == 0:
        out = {"metric": "Mvertex-iter/s", "value": value, "unit": "Mvertex-iter/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": "batch512", "grids": 512, "vertices": n_all, "algo": args.algo.upper(),
                          "parallelism": f"grids sharded over {world} GPU(s), no collective" if world > 1 else "single",
                          "iterate": "f32", "iters_per_step": iters,
                          "step": "cold start + iterations to the oracle-equal cut of the sampled grids + check",
                          "autotuned_scan": {"threads": chosen[0], "ctas_per_sm": chosen[1],
                                             "step": ["branchy", "predicated", "padded"][chosen[2]]},
                          "l2": "256 MB buffer written between steps; working set 3 GB > L2"},
               "time_to_oracle_equal_cut_ms": {"cold": ms_per_step if kstar else None, "warm": None},
               "iters_to_oracle_equal_cut": kstar, "sampled_grids_match": ok,
               "separate_solves": {"ms": sep_ms, "value": n_total * iters / (sep_ms / 1e3) / 1e6,
                                   "speedup_of_batch": sep_ms / ms_per_step, "grids": G},
               "roofline": {"bound": "hbm", "kernel": "iteration (scan + update graph)", "achieved": achieved,
                            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                            "traffic": None, "alg_bytes_per_iteration": iter_bytes},
               "cpu_baseline": cpu_base,
               "e2e": {"value": n_total * iters / e2e_s / 1e6, "unit": "Mvertex-iter/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": n_total},
               "clocks": clk, "gpu_launches": (3 * iters + 4) if args.algo == "fista" else (2 * iters + 3)}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def warm_vs_cold(args, algos, local=0, cpu_leg=True):
    """Cold-started iteration vs the same iteration started from the U-Net's
    predicted block duals (AAR/AP state z = y_hat, BCD/FISTA state y = y_hat),
    both to the oracle-equal cut, on the 2048^2 warm-start problem, for each
    of `algos`.  The network is trained first (untimed); each timed warm step
    includes the prediction (device features, forward pass, rescaling into
    the state: tvcut_unet_predict_state).  Clocks are sampled over the timed
    region."""
    import torch
    from paper_1503_01563_gb300 import learn, tvcut
    wl = WORKLOADS["warm2048"]
    dims = wl["dims"]
    w, a = inputs.uniform_grid(dims, wl["seed"])
    n = int(np.prod(dims))
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    e_star = oracle.maxflow(w, a, 1)[1]
    t_mf = time.perf_counter() - t0
    cpu_base = None
    if cpu_leg:
        cores = os.cpu_count() or 1
        code0 = ALGOS[algos[0]]
        st0 = oracle.cold_state(code0, w)
        t0 = time.perf_counter()
        oracle.iterate(code0, w, a, st0, 2, nthreads=cores)
        t_it = time.perf_counter() - t0
        cpu_base = {"value": 2 * n / t_it / 1e6, "unit": "Mvertex-iter/s", "cores": cores, "kind": "oracle",
                    "sample": f"2 FP64 {algos[0].upper()} iterations over the 2048^2 grid ({t_it:.1f} s); "
                              f"max-flow E* {t_mf:.1f} s"}
    stream = torch.cuda.current_stream()
    # training (untimed): solver-generated targets, GPU forward/backward/Adam
    t0 = time.perf_counter()
    X, Y = learn.make_training_set(wl["train_n"], wl["train_hw"], wl["train_hw"], seed=1)
    t_data = time.perf_counter() - t0
    net = tvcut.UNet(base=32, batch=16, H=wl["train_hw"], W=wl["train_hw"], seed=3, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    hist = learn.train(net, X, Y, steps=wl["train_steps"], batch=16)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    wd = torch.from_numpy(w).cuda()
    ad = [torch.from_numpy(x).cuda() for x in a]
    res = {"workload": "warm2048", "dims": list(dims), "oracle_min_cut": e_star, "iterate": "f32",
           "network": "U-Net 4 levels, 32 channels, BF16 weights/activations, FP32 accumulation",
           "training": f"{wl['train_n']} solver-generated {wl['train_hw']}^2 problems, {wl['train_steps']} Adam "
                       f"steps of 16 (data {t_data:.1f} s, training {t_train:.1f} s, loss {hist[0]:.4f} -> "
                       f"{float(np.mean(hist[-20:])):.4f})",
           "step": "cold: cold start + k_cold iterations; warm: tvcut_unet_predict_state + k_warm iterations; "
                   "both end at the oracle-equal cut",
           "l2": "256 MB buffer written before each timed solve"}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name in algos:
        algo = ALGOS[name]
        s = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=1, stream=stream.cuda_stream)
        s.set_problem(wd, ad)

        def probe(warm):
            if warm:
                net.predict_state(s)
            else:
                s.reset()
            for k in range(1, wl["cap"] + 1):
                _, st = s.iterate(1)
                if st.energy_i64 == e_star:
                    return k
            return None
        k_cold = probe(False)
        k_warm = probe(True)
        s.close()
        timed = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=10 ** 6, stream=stream.cuda_stream)
        timed.set_problem(wd, ad)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        cold_ms, warm_ms, inf_ms, ok = [], [], [], True
        clocks = ClockSampler(local)
        for rep in range(args.warmup + args.steps):
            if rep == args.warmup:
                torch.cuda.synchronize()
                clocks.start()
            flush.zero_()
            ev[0].record(stream)
            timed.reset()
            _, st = timed.iterate(k_cold or wl["cap"])
            ev[1].record(stream)
            ok = ok and st.energy_i64 == e_star
            flush.zero_()
            ev[2].record(stream)
            net.predict_state(timed)
            ev[3].record(stream)
            _, st = timed.iterate(k_warm or wl["cap"])
            ev[4].record(stream)
            ev[4].synchronize()
            ok = ok and st.energy_i64 == e_star
            if rep >= args.warmup:
                cold_ms.append(ev[0].elapsed_time(ev[1]))
                inf_ms.append(ev[2].elapsed_time(ev[3]))
                warm_ms.append(ev[2].elapsed_time(ev[4]))
        clk = clocks.stop()
        timed.close()
        cold, warm = float(np.median(cold_ms)), float(np.median(warm_ms))
        res[name] = {"iters": {"cold": k_cold, "warm": k_warm},
                     "ms": {"cold": cold if k_cold else None, "warm": warm if k_warm else None,
                            "warm_prediction": float(np.median(inf_ms))},
                     "warm_faster": bool(k_cold and k_warm and warm < cold),
                     "cold_Mvertex_iter_s": n * (k_cold or wl["cap"]) / (cold / 1e3) / 1e6,
                     "energies_match": ok, "clocks": clk}
    net.close()
    return res, cpu_base


def run_warm(args):
    """The warm2048 workload on its own line (--algo picks the iteration)."""
    import torch

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank != 0:
        return 0                                   # single-GPU workload: extra ranks idle
    torch.cuda.set_device(local)
    res, cpu_base = warm_vs_cold(args, [args.algo], local)
    r = res[args.algo]
    n = int(np.prod(res["dims"]))
    cold = r["ms"]["cold"]
    out = {"metric": "Mvertex-iter/s", "value": r["cold_Mvertex_iter_s"], "unit": "Mvertex-iter/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": cold, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "warm2048", "dims": res["dims"], "algo": args.algo.upper(), "iterate": "f32",
                      "network": res["network"], "training": res["training"], "step": res["step"],
                      "l2": res["l2"]},
           "time_to_oracle_equal_cut_ms": {"cold": cold, "warm": r["ms"]["warm"],
                                           "warm_prediction": r["ms"]["warm_prediction"]},
           "iters_to_oracle_equal_cut": r["iters"], "oracle_min_cut": res["oracle_min_cut"],
           "step_energies_match": r["energies_match"], "cpu_baseline": cpu_base,
           "roofline": None, "e2e": None, "clocks": r["clocks"], "gpu_launches": None,
           "vertices": n}
    print(json.dumps(out), flush=True)
    return 0


def unet_layer_times(H, W, steps, warmup, only=None):
    """Each of the U-Net's 18 convolutions alone at its shape in the forward
    pass (batch 1, random BF16 input and weights, ReLU and bias, the default
    engine), L2 flushed before each launch, CUDA events; with its floor: the
    tensor peak for its flops or HBM for its BF16 input read once and output
    written once, whichever is slower."""
    import torch
    from paper_1503_01563_gb300 import tvcut
    lib = tvcut.lib()
    hbm, _ = peaks()
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    tc = float(json.load(open(p))["bf16_tflops"]) if os.path.exists(p) else 1900.0
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    rows = []
    for li, (lvl, ci, co) in enumerate(UNET_CONVS):
        if only is not None and li != only:
            continue
        h, w = H >> lvl, W >> lvl
        x = torch.randn((1, h, w, ci), device="cuda", generator=g).to(torch.bfloat16)
        wt = (torch.randn((9, co, ci), device="cuda", generator=g) * 0.05).to(torch.bfloat16)
        b = torch.randn((co,), device="cuda", generator=g)
        y = torch.empty((1, h, w, co), device="cuda", dtype=torch.bfloat16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for rep in range(warmup + steps):
            flush.zero_()
            e0.record()
            code = lib.tvcut_conv3x3_bf16_ex(x.data_ptr(), wt.data_ptr(), b.data_ptr(), y.data_ptr(), 1, h, w, ci, co,
                                             1, 0, None)
            e1.record()
            e1.synchronize()
            if code != 0:
                raise RuntimeError(f"tvcut_conv3x3_bf16_ex failed with status {code}")
            if rep >= warmup:
                ts.append(e0.elapsed_time(e1) * 1e3)
        t_us = float(np.median(ts))
        flops = 2.0 * h * w * 9 * ci * co
        byts = h * w * (ci + co) * 2.0
        floor_us = max(flops / (tc * 1e12), byts / (hbm * 1e9)) * 1e6
        rows.append({"layer": li, "hw": h, "cin": ci, "cout": co, "us": t_us, "floor_us": floor_us,
                     "bound": "hbm" if byts / (hbm * 1e9) > flops / (tc * 1e12) else "tensor",
                     "frac_of_floor": floor_us / t_us})
    return rows


def run_unet(args):
    """U-Net inference at 2048^2: TFLOP/s of the forward pass (its 18 3x3
    convolutions as implicit GEMMs; pooling, upsampling and concatenation
    counted as zero flops) with the tcgen05 convolutions, beside the same
    network on the mma.sync kernels; end to end with a host input and output."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank != 0:
        return 0                                   # single-GPU workload: extra ranks idle
    torch.cuda.set_device(local)
    from paper_1503_01563_gb300 import tvcut
    wl = WORKLOADS["unet2048"]
    H = W = args.unet_hw
    if args.unet_layer >= 0:                       # one convolution alone (for profiling)
        rows = unet_layer_times(H, W, args.steps, args.warmup, only=args.unet_layer)
        print(json.dumps({"workload": f"unet{H} layer {args.unet_layer}", "per_layer": rows}), flush=True)
        return 0
    flops = sum(2.0 * (H >> l) * (W >> l) * 9 * ci * co for l, ci, co in UNET_CONVS)
    g = np.random.default_rng(wl["seed"])
    x = g.normal(size=(1, H, W, 3)).astype(np.float32)
    stream = torch.cuda.current_stream()
    net = tvcut.UNet(base=wl["base"], batch=1, H=H, W=W, seed=wl["seed"], stream=stream.cuda_stream)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty((1, H, W, 2), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    clk = None
    for engine in (1, 3, 0):                       # the timed line is engine 0 (persistent tcgen05)
        net.set_engine(engine)
        for _ in range(args.warmup):
            net.forward(xd, out)
        torch.cuda.synchronize()
        if engine == 0:
            clocks = ClockSampler(local)
            clocks.start()
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            net.forward(xd, out)
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
        if engine == 0:
            clk = clocks.stop()
        res[engine] = tot / args.steps
    err = tvcut.lib().tvcut_conv_tc_error()
    per_layer = unet_layer_times(H, W, max(3, args.steps), args.warmup)
    # end to end: pinned host input -> forward -> host output
    xp = torch.from_numpy(x).pin_memory()
    op = torch.empty((1, H, W, 2), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd.copy_(xp, non_blocking=True)
        net.forward(xd, out)
        op.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    # CPU oracle (PyTorch CPU FP32 forward) on a 256^2 crop, scaled by flops
    import oracle.unet_ref as unet_ref
    theta = torch.from_numpy(net.params())
    hs = 256
    t0 = time.perf_counter()
    with torch.no_grad():
        unet_ref.forward(theta, torch.from_numpy(x[:, :hs, :hs].copy()), wl["base"])
    t_cpu = time.perf_counter() - t0
    cpu_flops = flops * (hs * hs) / (H * W)
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peak, peak_kind = float(json.load(open(p))["bf16_tflops"]), "measured (burst)"
    else:
        peak, peak_kind = 1900.0, "fallback"
    tf = flops / (res[0] / 1e3) / 1e12
    # per-layer floor: each convolution bound by the tensor peak or by HBM
    # (BF16 input read once and output written once), whichever is slower
    hbm, _ = peaks()
    floor_s = sum(max(2.0 * (H >> l) * (W >> l) * 9 * ci * co / (peak * 1e12),
                      (H >> l) * (W >> l) * (ci + co) * 2 / (hbm * 1e9)) for l, ci, co in UNET_CONVS)
    out_json = {"metric": "TFLOP/s", "value": tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res[0], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": "unet2048" if H == 2048 else f"unet{H}", "dims": [H, W],
                           "network": "U-Net 4 levels, 32 channels",
                           "weights": "random init", "gflop_per_forward": flops / 1e9,
                           "step": "one forward pass (all 29 launches)",
                           "l2": "256 MB buffer written between steps; activations > L2"},
                "mma_sync_engine": {"ms": res[1], "TFLOP/s": flops / (res[1] / 1e3) / 1e12},
                "tcgen05_one_tile_per_cta_engine": {"ms": res[3], "TFLOP/s": flops / (res[3] / 1e3) / 1e12},
                "tcgen05_wait_gave_up": bool(err),
                "roofline": {"bound": "tensor", "kernel": "forward pass (18 tcgen05 convolutions + elementwise)",
                             "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                             "peak_source": peak_kind, "traffic": None,
                             "layer_floor_ms": floor_s * 1e3, "frac_of_layer_floor": floor_s * 1e3 / res[0]},
                "per_layer": {"layers": per_layer, "sum_us": sum(r["us"] for r in per_layer),
                              "floor_sum_us": sum(r["floor_us"] for r in per_layer)},
                "cpu_baseline": {"value": cpu_flops / t_cpu / 1e12, "unit": "TFLOP/s",
                                 "cores": torch.get_num_threads(), "kind": "oracle",
                                 "sample": f"oracle forward (PyTorch CPU FP32) on a {hs}x{hs} crop ({t_cpu:.2f} s)"},
                "e2e": {"value": flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(x.nbytes),
                        "d2h_bytes_per_step": int(H * W * 2 * 4)},
                "clocks": clk, "gpu_launches": 29 * args.steps}
    print(json.dumps(out_json), flush=True)
    net.close()
    return 0


def time_to_cut(name, algo_name, steps, warmup, stream, flush, mapping=-1):
    """Cold start to the oracle-equal cut on another workload (the same rules
    as the main line: k* found untimed, L2 flushed before each timed solve,
    CUDA events on the library's stream)."""
    import torch
    from paper_1503_01563_gb300 import tvcut
    w, a = make_problem(name)
    dims = tuple(w.shape)
    n = int(np.prod(dims))
    e_star, _ = exact_min_cut(w, a)
    wd = torch.from_numpy(w).cuda()
    ad = [torch.from_numpy(x).cuda() for x in a]
    code = ALGOS[algo_name]
    cap = WORKLOADS[name]["cap"]
    pr = tvcut.Solver(dims, algo=code, dtype=tvcut.F32, check_every=1, stream=stream.cuda_stream, mapping=mapping)
    pr.set_problem(wd, ad)
    km = None
    for k in range(1, cap + 1):
        _, st = pr.iterate(1)
        if st.energy_i64 == e_star:
            km = k
            break
    pr.close()
    if km is None:
        return {"iters": None}
    sv = tvcut.Solver(dims, algo=code, dtype=tvcut.F32, check_every=km, stream=stream.cuda_stream, mapping=mapping)
    sv.set_problem(wd, ad)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, ok = [], True
    for rep in range(warmup + steps):
        flush.zero_()
        e0.record(stream)
        tvcut.tvcut_reset(sv.h)
        _, st = sv.iterate(km)
        e1.record(stream)
        e1.synchronize()
        ok = ok and st.energy_i64 == e_star
        if rep >= warmup:
            times.append(e0.elapsed_time(e1))
    sv.close()
    ms = float(np.median(times))
    return {"dims": list(dims), "iters": km, "ms": ms, "Mvertex_iter_s": n * km / (ms / 1e3) / 1e6,
            "energies_match": ok, "oracle_min_cut": e_star, "mapping": mapping}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1503_01563_gb300 import tvcut

    w, a = make_problem(args.workload)
    dims = tuple(w.shape)
    n = int(np.prod(dims))
    conn = WORKLOADS[args.workload].get("conn", 0)
    ndim = 4 if conn == 8 else len(dims)          # blocks per iteration
    algo = ALGOS[args.algo]

    # the oracle's exact min-cut value E* (rank 0)
    e_star, t_mf = (None, 0.0)
    if rank == 0:
        e_star, t_mf = exact_min_cut(w, a)

    stream = torch.cuda.current_stream(dev)
    wd = torch.from_numpy(w).to(dev)
    ad = [torch.from_numpy(x).to(dev) for x in a]

    # find k*: first iteration whose cut energy equals E* (untimed, checks every iteration)
    kstar = None
    cap = WORKLOADS[args.workload]["cap"]
    if rank == 0:
        probe = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=1, stream=stream.cuda_stream,
                             mapping=args.mapping, connectivity=conn)
        probe.set_problem(wd, ad)
        for k in range(1, cap + 1):
            _, st = probe.iterate(1)
            if st.energy_i64 == e_star:
                kstar = k
                break
        probe.close()
    iters = kstar if kstar else cap

    # CPU leg (rank 0): the oracle to k*, timed, and the FP32 primal against its FP64 one at k*/2 and k*
    cpu_base, drift = None, None
    if rank == 0:
        xs, cpu_base = cpu_leg(args.workload, w, a, kstar, budget_s=args.cpu_budget, algo=args.algo, t_mf=t_mf)
        if xs:
            chk = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=10 ** 6, stream=stream.cuda_stream,
                               mapping=args.mapping, connectivity=conn)
            chk.set_problem(wd, ad)
            drift, done = {}, 0
            for k in sorted(xs):
                chk.iterate(k - done)
                done = k
                ref = xs[k]
                got = chk.primal()
                drift[str(k)] = float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30))
            chk.close()
            drift = {"max_abs_rel_primal": drift, "reference": "FP64 oracle, same iterations from the cold start",
                     "tolerance": 1e-4}
    if world > 1:
        t = torch.tensor([iters], device=dev)
        dist.broadcast(t, 0)
        iters = int(t.item())

    solver = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=iters, stream=stream.cuda_stream,
                          mapping=args.mapping, connectivity=conn)
    solver.set_problem(wd, ad)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        tvcut.tvcut_reset(solver.h)
        _, st = solver.iterate(iters)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    tvcut.tvcut_profile(solver.h, True)
    clocks = ClockSampler(local)
    clocks.start()
    total_ms = 0.0
    energies = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        st = step()
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        energies.append(st.energy_i64)
    torch.cuda.synchronize()
    clk = clocks.stop()
    kms, klaunch = tvcut.tvcut_profile_read(solver.h)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = world * n * iters * args.steps / (total_ms / 1e3) / 1e6

    # roofline of the dominant kernel (largest device-time share)
    kinds = ["prox", "update", "check", "other"]
    bpv = kernel_bytes_per_vertex(ndim, args.algo)
    evals = args.steps if bpv["eval"] is not None else 0       # one checked iteration per step
    kind_bytes = [bpv["prox"] * klaunch[0] * n,
                  (bpv["update"] * (klaunch[1] - evals) + (bpv["eval"] or 0) * evals
                   + bpv["check_extra"] * args.steps) * n]
    dom = max(range(2), key=lambda k: kms[k])
    dom_name = kinds[dom]
    launches = int(klaunch[dom])
    alg_bytes = kind_bytes[dom] / max(launches, 1)
    avg_s = kms[dom] / 1e3 / max(launches, 1)
    achieved = alg_bytes / avg_s / 1e9
    peak, peak_kind = peaks()
    traffic = None if args.mapping != -1 else kernel_traffic(
        dom_name, args.workload if args.algo == "aar" else f"{args.workload}:{args.algo}")
    moved = kind_bytes[0] + kind_bytes[1]
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3,
                "share_of_step": float(kms[dom] / max(kms.sum(), 1e-9)),
                "iteration_GBps": float(moved / max((kms[0] + kms[1]) / 1e3, 1e-12) / 1e9)}
    # the whole step against HBM at the two per-vertex byte counts of the
    # method: the direction-wise sweep schedule (2D 44 B, 3D 72 B: one read of
    # each block's state and weights per sweep plus the intermediates the
    # sweeps hand on) and the lower bound (every state array read and written
    # once, w and the weights read once: 2D 28 B, 3D 40 B)
    if args.algo == "aar" and not conn:
        vps = value / world * 1e6                  # this GPU's vertex-iterations per second
        sched_b, lb_b = (72, 40) if ndim == 3 else (44, 28)
        roofline["step_frac_at_schedule_bytes"] = {"bytes_per_vertex_iter": sched_b,
                                                   "frac": vps * sched_b / (peak * 1e9)}
        roofline["step_frac_at_lower_bound_bytes"] = {"bytes_per_vertex_iter": lb_b,
                                                      "frac": vps * lb_b / (peak * 1e9)}

    # end to end through the C-ABI with host buffers: H2D inputs, solve, D2H labels
    e2e_solver = tvcut.Solver(dims, algo=algo, dtype=tvcut.F32, check_every=iters, stream=stream.cuda_stream,
                              mapping=args.mapping, connectivity=conn)
    labels = torch.empty(dims, dtype=torch.uint8).pin_memory()
    w_pin = torch.from_numpy(w).pin_memory()
    a_pin = [torch.from_numpy(x).pin_memory() for x in a]
    h2d = int(w.nbytes + sum(x.nbytes for x in a))
    d2h = int(labels.numel())
    e2e_steps = max(1, args.steps // 2)
    e2e_s = 0.0
    for i in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_solver.set_problem(w_pin, a_pin)
        e2e_solver.iterate(iters)
        st2 = tvcut.tvcut_cut(e2e_solver.h, labels)          # labels into pinned host memory
        if i > 0:                       # first call warms the path
            e2e_s += time.perf_counter() - t0
    e2e_value = world * n * iters * e2e_steps / e2e_s / 1e6

    # the library's own stop rules (no oracle k*): `certified` (energy - the rigorous bound < 1: a proof)
    # and, for FP32 iterates, stop_on_approx (energy - the iterate's own bound < 1: not a proof); FP64
    # iterates beside them for the rigorous rule
    own = None
    if rank == 0:
        own = {"rules": {"certified": "energy - certified_lb < 1 (Sec. 2.2 bound from exactly feasible FP64 block "
                                      "duals; FP32 iterates: duals recomputed in FP64 from the FP32 state when the "
                                      "approximate gap is small, params.certify = 2): a proof of optimality",
                         "approx": "stop_on_approx: energy - discrete_lb < 1 with the iterate's own dual: not a "
                                   "proof"}, "cap": cap}
        for tag, dtype, approx_rule, everies in (("f32_approx", tvcut.F32, 1, (5, 10)),
                                                 ("f32_certified", tvcut.F32, 0, (5, 10)),
                                                 ("f64_certified", tvcut.F64, 0, (5, 10))):
            for every in everies:
                sv = tvcut.Solver(dims, algo=algo, dtype=dtype, check_every=every, stream=stream.cuda_stream,
                                  connectivity=conn, stop_on_approx=approx_rule,
                                  certify=2 if tag == "f32_certified" else 0)
                sv.set_problem(wd, ad)
                times, res = [], None
                for rep in range(3):
                    flush.zero_()
                    ev0.record(stream)
                    tvcut.tvcut_reset(sv.h)
                    code, st = sv.iterate(cap)
                    ev1.record(stream)
                    ev1.synchronize()
                    times.append(ev0.elapsed_time(ev1))
                    res = (code, st)
                code, st = res
                own[f"{tag}_check_every_{every}"] = {
                    "ms": float(np.median(times)), "iters": int(st.iters), "stopped": bool(code == tvcut.OK),
                    "certified": bool(st.certified), "energy_equals_oracle": bool(st.energy_i64 == e_star),
                    "energy_minus_certified_lb": (float(st.energy_i64 - st.certified_lb)
                                                  if np.isfinite(st.certified_lb) else None)}
                sv.close()
    # the other methods on the same workload: cold start to the oracle-equal cut, same timing rules
    methods = None
    if rank == 0 and args.workload == "volume256" and args.algo == "aar":
        methods = {}
        for mname in ("bcd", "fista", "ap"):
            mcode = ALGOS[mname]
            pr = tvcut.Solver(dims, algo=mcode, dtype=tvcut.F32, check_every=1, stream=stream.cuda_stream)
            pr.set_problem(wd, ad)
            km = None
            for k in range(1, cap + 1):
                _, st = pr.iterate(1)
                if st.energy_i64 == e_star:
                    km = k
                    break
            pr.close()
            if km is None:
                methods[mname] = {"iters": None, "ms": None}
                continue
            sv = tvcut.Solver(dims, algo=mcode, dtype=tvcut.F32, check_every=km, stream=stream.cuda_stream)
            sv.set_problem(wd, ad)
            times, ok = [], True
            for rep in range(args.warmup + max(3, args.steps // 2)):
                flush.zero_()
                ev0.record(stream)
                tvcut.tvcut_reset(sv.h)
                _, st = sv.iterate(km)
                ev1.record(stream)
                ev1.synchronize()
                ok = ok and st.energy_i64 == e_star
                if rep >= args.warmup:
                    times.append(ev0.elapsed_time(ev1))
            sv.close()
            methods[mname] = {"iters": km, "ms": float(np.median(times)), "energies_match": ok,
                              "Mvertex_iter_s": n * km / (float(np.median(times)) / 1e3) / 1e6}
            if mname == "bcd":          # the same solve stopped by the library's certificate (FP64 duals)
                sv = tvcut.Solver(dims, algo=mcode, dtype=tvcut.F32, check_every=2, certify=2,
                                  stream=stream.cuda_stream)
                sv.set_problem(wd, ad)
                times, res = [], None
                for rep in range(3):
                    flush.zero_()
                    ev0.record(stream)
                    tvcut.tvcut_reset(sv.h)
                    code, st = sv.iterate(cap)
                    ev1.record(stream)
                    ev1.synchronize()
                    times.append(ev0.elapsed_time(ev1))
                    res = st
                sv.close()
                methods[mname]["certified"] = {
                    "ms": float(np.median(times)), "iters": int(res.iters), "certified": bool(res.certified),
                    "energy_equals_oracle": bool(res.energy_i64 == e_star), "check_every": 2}
    # the 2D segmentation (1024^2 blobs) on the same GPU, recorded beside the main line
    seg = None
    if rank == 0 and args.workload == "volume256" and args.algo == "aar":
        seg = {"workload": "seg1024",
               "aar": time_to_cut("seg1024", "aar", max(3, args.steps // 2), args.warmup, stream, flush),
               "bcd": time_to_cut("seg1024", "bcd", max(3, args.steps // 2), args.warmup, stream, flush),
               "bcd_message_passing": time_to_cut("seg1024", "bcd", max(3, args.steps // 2), args.warmup, stream,
                                                  flush, mapping=10),
               "fista": time_to_cut("seg1024", "fista", max(3, args.steps // 2), args.warmup, stream, flush),
               "fista_funnel": time_to_cut("seg1024", "fista", max(3, args.steps // 2), args.warmup, stream,
                                           flush, mapping=11)}
    # the batch of 512 uneven grids (AAR), recorded beside the main line
    batch = None
    if rank == 0 and args.workload == "volume256" and args.algo == "aar":
        import oracle
        oracle.build()
        bwl = WORKLOADS["batch512"]
        bdims, bprobs = batch_problems(bwl["grids"], bwl["seed"])
        bsample = list(range(0, len(bdims), max(1, len(bdims) // 16)))
        be = {g: oracle.maxflow(bprobs[g][0], bprobs[g][1], 1)[1] for g in bsample}
        bn = int(sum(h * w for h, w in bdims))
        bsteps = max(3, args.steps // 4)
        m = batch_measure(bdims, bprobs, ALGOS["aar"], bsteps, 2, stream, be, bsample, bwl["cap"], local)
        bms = m["total_ms"] / bsteps
        batch = {"workload": "batch512", "grids": len(bdims), "vertices": bn, "iters": m["kstar"],
                 "ms": bms if m["kstar"] else None, "Mvertex_iter_s": bn * m["iters"] / (bms / 1e3) / 1e6,
                 "sampled_grids_match": m["ok"], "separate_solves_ms": m["sep_ms"],
                 "speedup_of_batch": m["sep_ms"] / bms, "clocks": m["clocks"]}
    warm = None
    if rank == 0 and args.workload == "volume256" and args.algo == "aar" and not args.no_warm:
        warm, _ = warm_vs_cold(args, ["aar", "bcd", "fista"], local, cpu_leg=False)

    out = None
    if rank == 0:
        out = {
            "metric": "Mvertex-iter/s", "value": value, "unit": "Mvertex-iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(dims), "algo": args.algo.upper(), "iterate": "f32",
                       "connectivity": conn if conn else 2 * len(dims), "blocks": ndim, "mapping": args.mapping,
                       "iters_per_step": iters, "step": "cold start + iterations to the oracle-equal cut + cut",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MB buffer written between steps"},
            "time_to_oracle_equal_cut_ms": {
                "cold": ms_per_step if kstar else None, "warm": None,
                "warm2048": None if warm is None else {
                    k: warm[k]["ms"] for k in ("aar", "bcd", "fista")}},
            "iters_to_oracle_equal_cut": kstar, "oracle_min_cut": e_star,
            "time_to_cut_own_stop_ms": own,
            "time_to_oracle_equal_cut_other_methods": methods,
            "seg1024_time_to_oracle_equal_cut": seg,
            "batch512_time_to_oracle_equal_cut": batch,
            "fp32_vs_fp64": drift,
            "warm_start_2048": warm,
            "step_energies_match": all(e == e_star for e in energies),
            "roofline": roofline, "cpu_baseline": cpu_base,
            "e2e": {"value": e2e_value, "unit": "Mvertex-iter/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk, "gpu_launches": int(klaunch.sum()),
            "kernel_ms": dict(zip(kinds, [float(x) for x in kms])),
            "kernel_launches": dict(zip(kinds, [int(x) for x in klaunch])),
        }
        print(json.dumps(out), flush=True)
    solver.close()
    e2e_solver.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="volume256")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-warm", action="store_true",
                    help="skip the 2048^2 warm-vs-cold pair that the default volume256 line carries")
    ap.add_argument("--unet-layer", type=int, default=-1,
                    help="unet2048 workload: time one convolution of the network alone (0..17) and nothing else")
    ap.add_argument("--unet-hw", type=int, default=2048,
                    help="image size of the unet2048 workload (a multiple of 128; smaller for profiling)")
    ap.add_argument("--mapping", type=int, default=-1,
                    help="scan mapping of the timed solve (tvcut_params.mapping; -1 automatic, 10 message "
                         "passing, 11 funnel taut string)")
    ap.add_argument("--algo", choices=sorted(ALGOS), default="aar",
                    help="iteration of the volume256/seg1024 workloads: AAR (Eq. 3), AP (Sec. 4.2), BCD or FISTA (Sec. 4.1)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "warm2048":
        return run_warm(args)
    if args.workload == "unet2048":
        return run_unet(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
