"""Benchmark: tabu moves/s of the MPMA hot path on GB300.

Workload (one "step" = one generation of Alg. 2 on each instance):
  five synthetic n = 70 PLSE instances with fill ratio r in {0.3, 0.4, 0.5, 0.6,
  0.7} (random insertion for 0.3/0.5/0.7, permuted cyclic square for 0.4/0.6;
  seeds 3000+k), population p = 16384, phase-1 tabu iterations 10|V|, phase 2
  2|V| iterations, Philox seed 1 (+ rank).  The populations stay resident on the
  GPU between steps; the optimality stop is off so every step is a full
  generation.  Warm-up generations run first, so the timed generations are
  steady-state ones (walks start from AUX offspring, as in the paper's runs).

Default: python bench.py  (N=1, 5 timed steps, 3 warm-up steps)
Multi-GPU: torchrun ... bench.py --gpus N  (independent replicas, one per rank)
Reference arm: python bench.py --impl reference  (the CPU oracle on a bounded
sample of the same workload, on the host cores)
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RATIOS = (0.3, 0.4, 0.5, 0.6, 0.7)
POP = 16384
METRIC = "tabu moves/s (16k pop, n=70)"
UNIT = "moves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pop", type=int, default=POP)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serial", action="store_true",
                    help="run the five instances' generations one after another on one stream "
                         "instead of on five streams at once")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ls-case", type=float, default=None, metavar="R",
                    help="small profiling case instead of the benchmark: steady-state phase-1 local "
                         "search on the n=70 instance with fill ratio R (population --pop, "
                         "--ls-iters iterations per launch, --steps launches)")
    ap.add_argument("--ls-iters", type=int, default=3000)
    ap.add_argument("--launch", default=None, metavar="LANES,WALKS,PLACE",
                    help="local-search launch knobs for every instance (plse_set_launch): threads "
                         "per walk, walks per block, colouring placement; results do not change")
    ap.add_argument("--batch", action="store_true",
                    help="batching case instead of the benchmark: 64 uneven instances solved one "
                         "by one with plse_solve, then together with plse_solve_batch")
    ap.add_argument("--batch-set", default="both", choices=["mix", "multistart", "both"])
    ap.add_argument("--batch-pop", type=int, default=0,
                    help="with --batch: one population for every job (default: by the size rule)")
    ap.add_argument("--generations", type=int, default=10,
                    help="generations per job of --batch and --serve")
    ap.add_argument("--inflight", type=int, default=None,
                    help="concurrent runs of --batch (default 16) and --serve (default 64)")
    ap.add_argument("--serve", action="store_true",
                    help="serving case instead of the benchmark: Poisson arrivals into the "
                         "library's request server, latency percentiles")
    ap.add_argument("--pop-sweep", action="store_true",
                    help="population-size sweep on a synthetic (60, 0.7) instance: throughput "
                         "and best score per population size")
    ap.add_argument("--lsc", action="store_true",
                    help="Latin square completion case: time to a complete square on "
                         "cyclic-delete instances, n in {50, 60, 70}, r in {0.3..0.8}")
    ap.add_argument("--dist-case", action="store_true",
                    help="distance kernel case: plse_distances on --pop x --pop colourings of the "
                         "n=70, r=0.3 instance, ALU roofline")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--serve-walks", type=int, default=4,
                    help="with --serve: cap on local-search walks per block (0 = automatic); a "
                         "low cap leaves each SM room for other requests' short kernels")
    ap.add_argument("--serve-mem", type=float, default=1.0,
                    help="with --serve: device-memory budget of the server in GB")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--serve-seq-sample", type=int, default=0, metavar="K",
                    help="serve: run the sequential leg on K evenly spaced requests only "
                         "(0 = all); served results are checked against those")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(pop, iters_note="10|V|"):
    return {"workload": "n70_r0.3-0.7_p%d" % pop, "n": 70, "fill_ratios": list(RATIOS),
            "instances": len(RATIOS), "population": pop, "phase1_iters": iters_note,
            "phase2_iters": "2|V|", "generations_per_step": 1, "seed": 1,
            "l2": "inputs larger than L2: five resident populations (colourings, bit planes, "
                  "scores) of about 0.5 GB in total are touched every step",
            "optimal_stop": False}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(ms, moves, device):
    """Replicas: the job's time is the slowest rank's timed region, its work the
    sum of every rank's moves (a no-op for one process)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    mv = torch.tensor([float(moves)], dtype=torch.float64, device=device)
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tdist.all_reduce(mv, op=tdist.ReduceOp.SUM)
    return float(t.item()), float(mv.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# DRAM bytes per tabu move of local_search_kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a launch with walks as long
# as the benchmark's (bench.py --ls-case 0.3 --pop 3040 --ls-iters 34300
# --steps 1: 193.8 MB + 365.0 MB for 3.7253e7 moves); scaled to a benchmark
# launch by its moves.  None whenever the kernel has changed since the capture.
LS_DRAM_BYTES_PER_MOVE = (193757184 + 365008384) / 37.2530e6   # 15.00 B per move


def union_ms(intervals):
    """Length of the union of [start, end] intervals (ms): the time during which
    at least one of them was running."""
    total, cur_s, cur_e = 0.0, None, None
    for a, b in sorted((float(a), float(b)) for a, b in intervals):
        if b <= a:
            continue
        if cur_e is None or a > cur_e:
            if cur_e is not None:
                total += cur_e - cur_s
            cur_s, cur_e = a, b
        else:
            cur_e = max(cur_e, b)
    if cur_e is not None:
        total += cur_e - cur_s
    return total


def drive_runs(insts, streams, generations):
    """Issues `generations` more generations of every run, each on its own
    stream, refilling whichever run has room (two generations in flight per
    run), and returns once all are enqueued."""
    left = [generations] * len(insts)
    while any(left):
        progressed = False
        for k, (G, st) in enumerate(zip(insts, streams)):
            if left[k] == 0:
                continue
            G.run_query()
            if G.run_issue(stream=st):
                left[k] -= 1
                progressed = True
        if not progressed:
            time.sleep(0.0002)


def walk_bytes(w):
    """Algorithmic bytes of tabu moves (explicit-gamma accounting): per scanned
    candidate 1 B colour, per scanned (v, j) pair 1 B gamma + 2 B tabu expiry,
    per applied move 5 B per neighbour of v* (colour read + two gamma updates)
    plus a 1 B colour write and a 2 B expiry write."""
    return w["cand"] + 3 * w["pairs"] + 5 * w["deg"] + 3 * w["moves"]


def run_gpu(args):
    import torch
    import torch.distributed as tdist
    from paper_2103_10453_gb300 import inputs, plse

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    seed = 1 + rank

    grids = [inputs.n70(r) for r in RATIOS]
    ref_ev = torch.cuda.Event(enable_timing=True)       # time origin of the local-search timeline
    ref_ev.record(stream)
    torch.cuda.synchronize()
    insts, streams = [], []
    for g in grids:
        G = plse.Instance(g)
        prm = plse.default_params(stop_at_bound=0)
        G.set_params(prm)
        if args.launch:
            G.set_launch(*[int(x) for x in args.launch.split(",")])
        st = None if args.serial else torch.cuda.Stream(device=dev)
        G.run_begin(args.pop, args.warmup + args.steps + 1, 10 * G.nv, seed, stream=st)
        insts.append(G)
        streams.append(st)

    def steps(k):
        # one step = one generation of each of the five runs
        if args.serial:
            for _ in range(k):
                for G in insts:
                    G.run_step(1)
        else:
            drive_runs(insts, streams, k)

    steps(args.warmup)
    before = [G.run_result(stream=st) for G, st in zip(insts, streams)]

    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in streams:
        if st is not None:
            st.wait_stream(stream)
    steps(args.steps)
    for st in streams:
        if st is not None:
            stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if world > 1:
        tdist.barrier()
    after = [G.run_result(stream=st) for G, st in zip(insts, streams)]
    # when the local-search launches of the timed generations ran (ms after ref_ev)
    timeline = [G.run_timeline(ref_ev, args.warmup, args.steps) for G in insts]
    ls_busy_ms = union_ms([tuple(iv) for tl in timeline for iv in tl])

    moves = sum(a["walks"]["moves"] - b["walks"]["moves"] for a, b in zip(after, before))
    wdelta = {k: sum(a["walks"][k] - b["walks"][k] for a, b in zip(after, before))
              for k in ("iterations", "moves", "cand", "pairs", "deg")}
    ls_ms = sum(a["ms_local_search"] - b["ms_local_search"] for a, b in zip(after, before))
    launches = sum(a["launches"] - b["launches"] for a, b in zip(after, before))
    per_inst = []
    for r, a, b in zip(RATIOS, after, before):
        mv = a["walks"]["moves"] - b["walks"]["moves"]
        it = a["walks"]["iterations"] - b["walks"]["iterations"]
        nvr = insts[RATIOS.index(r)].nv
        budget = args.steps * args.pop * 12 * nvr        # phase 1 10|V| + phase 2 2|V| per walk
        per_inst.append({"r": r, "nv": nvr, "moves": mv,
                         "ls_ms": round(a["ms_local_search"] - b["ms_local_search"], 2),
                         "cand_per_iter": round((a["walks"]["cand"] - b["walks"]["cand"]) / max(it, 1), 2),
                         "iters_budget_use": round(it / budget, 4),
                         "best_score": a["score"]})

    ms_max, total_moves = reduce_over_ranks(ms, moves, "cuda")
    value = total_moves / (ms_max / 1e3)

    # roofline of the dominant kernel (the local search), live from this run:
    # the shared-memory peak is measured here by the library's own probe
    # (conflict-free 16-byte loads on every SM), with the SM clock sampled
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    probe_clk = ClockSampler(dev)
    probe_clk.start()
    smem_bw = max(plse.smem_bandwidth(1 << 17)[0] for _ in range(3))
    probe_clocks = probe_clk.stop()
    smem_peak = smem_bw / 1e9                                  # GB/s
    smem_derived = sm_count * 128 * sm_max * 1e6 / 1e9
    bytes_alg = walk_bytes(wdelta)
    launches_ls = len(insts) * args.steps
    # the local-search launches of different runs overlap on five streams: the
    # kernel's time is the union of their intervals (equal to the sum of their
    # durations when they run one after another)
    achieved = bytes_alg / (ls_busy_ms / 1e3) / 1e9 if ls_busy_ms > 0 else None
    roofline = {"bound": "smem", "achieved": round(achieved, 1) if achieved else None,
                "peak": round(smem_peak, 1), "unit": "GB/s",
                "frac": round(achieved / smem_peak, 4) if achieved else None,
                "traffic": (round(LS_DRAM_BYTES_PER_MOVE * wdelta["moves"] / launches_ls)
                            if LS_DRAM_BYTES_PER_MOVE else None),
                "traffic_note": ("DRAM bytes per launch, scaled by moves from one ncu capture of a "
                                 "launch with benchmark-length walks (%.1f B per move)" % LS_DRAM_BYTES_PER_MOVE
                                 if LS_DRAM_BYTES_PER_MOVE else "no capture of the current kernel"),
                "kernel": "local_search_kernel",
                "peak_source": ("measured: shared-memory load probe (plse_smem_bandwidth, 16-byte loads, 2 "
                                "blocks of 1024 threads per SM), best of 3, SM clock %s MHz during the probe; "
                                "derived bound %d SMs x 128 B/clk x %.0f MHz = %.1f GB/s"
                                % (probe_clocks.get("sm_mhz"), sm_count, sm_max, smem_derived)),
                "bytes_per_launch": round(bytes_alg / launches_ls),
                "ms_per_launch": round(ls_busy_ms / launches_ls, 3),
                "ms_busy": round(ls_busy_ms, 2),
                "busy_share_of_step": round(ls_busy_ms / ms, 4) if ms > 0 else None,
                "ms_launch_durations_sum": round(ls_ms, 2),
                "time_note": ("ms_per_launch = the time during which any local-search launch of the "
                              "timed steps ran (union of their CUDA-event intervals on their own "
                              "streams) / launches; achieved = algorithmic bytes / that time"),
                "moves_per_launch": round(wdelta["moves"] / launches_ls)}

    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic (seeded instances of the paper's benchmark shapes; random initial colourings)",
           "config": dict(workload_config(args.pop), parallelism="replicas" if world > 1 else "single"),
           "schedule": ("the five runs one after another on one stream" if args.serial
                        else "the five runs on five CUDA streams at once (plse_run_issue)"),
           "roofline": roofline, "clocks": clk, "gpu_launches": launches,
           "per_instance": per_inst}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = run_e2e(args, plse, inputs, seed)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(sample_seconds=10.0)
    for G in insts:
        G.close()
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_e2e(args, plse, inputs, seed):
    """Same metric through the public C ABI with host buffers: plse_create of
    each instance (host grid -> device), one plse_solve_batch call solving the
    five one-generation jobs at once (concurrent runs), best grids back to the
    host; wall clock around all of it.  With --serial: one plse_solve_ex per
    instance, one after another."""
    import numpy as np
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    moves, h2d, d2h = 0, 0, 0
    insts = []
    for r in RATIOS:
        g = np.ascontiguousarray(inputs.n70(r), dtype=np.int8)
        G = plse.Instance(g)
        G.set_params(plse.default_params(stop_at_bound=0))
        insts.append(G)
        h2d += g.nbytes + G.nv * 24 + 2 * 70 * 20          # grid + uploaded instance image
    if args.serial:
        res = [G.solve(args.pop, 1, 10 * G.nv, seed, with_stats=True) for G in insts]
    else:
        res, rc = plse.solve_batch(insts, [(args.pop, 1, 10 * G.nv, seed) for G in insts],
                                   max_inflight=len(insts))
        if rc != plse.PLSE_OK:
            raise plse.PlseError(rc, "plse_solve_batch")
    for r in res:
        moves += r["walks"]["moves"]
        d2h += r["best_grid"].nbytes + 8 * r["generations"] + 64
    for G in insts:
        G.close()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return {"value": round(moves / secs, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "note": ("one generation (from random colourings) of each of the five instances through "
                     "%s, host grid in, host best grid out, wall clock"
                     % ("plse_solve_ex one by one" if args.serial else "one plse_solve_batch call"))}


# ---------------------------------------------------------------------------
def oracle_sample(budget_s=15.0, chain=0):
    """The CPU oracle as it stands on a bounded sample of the workload, in the
    GA's steady state.  For each of the five instances two individuals A, B are
    brought to a steady state by an untimed generation of local search from
    random colourings.  Then, until that instance's share of the budget is
    spent: the AUX offspring of A with partner B (untimed, cheap) gets one timed
    generation of local search (phase 1 with 10|V| iterations, phase 2 with
    2|V|, repair), and the pair becomes (B, result).  Single-threaded; `chain`
    offsets the individual indices (and so the trajectories) of independent
    samples run side by side.  Returns (moves, seconds, generations)."""
    import numpy as np
    import oracle
    from paper_2103_10453_gb300 import inputs
    oracle.build()
    moves, secs, gens = 0, 0.0, 0
    share = budget_s / len(RATIOS)
    base = 2 * chain

    def generation(I, S, ind, gen):
        S1, _, st1 = I.tabu_walk(S, ind, gen, 1, 10 * I.nv, 1)
        S2, _, st2 = I.tabu_walk(S1, ind, gen, 2, 2 * I.nv, 1)
        S3, _ = I.repair(S2)
        return S3, st1["moves"] + st2["moves"]

    for r in RATIOS:
        I = oracle.Instance(inputs.n70(r))
        P0 = I.init_population(base + 2, 1)
        A, _ = generation(I, P0[base], base, 0)
        B, _ = generation(I, P0[base + 1], base + 1, 0)
        t_inst, gen = 0.0, 1
        while t_inst < share:
            d = int(I.distances(A, B)[0, 0])
            if d == 0:                      # identical parents: restart B from random
                B, _ = generation(I, I.init_population(1, 100 + gen)[0], base + 1, gen)
                gen += 1
                continue
            pair = np.stack([A, B])
            O = I.crossover(pair, [1, 0], [[0, d], [d, 0]], gen, 1)[0]
            t0 = time.perf_counter()
            S, m = generation(I, O, base, gen)
            t_inst += time.perf_counter() - t0
            moves += m
            A, B = B, S
            gen += 1
            gens += 1
        secs += t_inst
    return moves, secs, gens


def _oracle_chain(args):
    budget_s, chain = args
    t0 = time.perf_counter()
    moves, secs, gens = oracle_sample(budget_s, chain)
    return moves, secs, gens, time.perf_counter() - t0


def cpu_baseline(sample_seconds=15.0, cores=None):
    """The oracle on the host: one single-threaded sample, then one independent
    sample per core at once (walks are independent, so the all-core rate is the
    sum of the chains' moves over the wall time of the slowest).  The pool uses
    'spawn' so that no child inherits a CUDA context."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    m1, s1, g1 = oracle_sample(sample_seconds)
    single = m1 / s1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_chain, [(sample_seconds, k + 1) for k in range(cores)])
    wall = time.perf_counter() - t0
    moves = sum(r[0] for r in res)
    busy = max(r[3] for r in res)
    value = moves / busy
    desc = ("steady-state generations of local search (phase 1 10|V| + phase 2 2|V| + repair) of one "
            "AUX offspring each, spread over the five n=70 instances; the C oracle single-threaded "
            "(%d generations, %.1f s timed: %.4g moves/s), then %d independent chains at once on %d "
            "host cores (%d generations, %.1f s wall)" % (g1, s1, single, cores, cores,
                                                        sum(r[2] for r in res), busy))
    return {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": desc, "seconds": round(wall, 2), "single_core_value": round(single, 1),
            "host_cores": os.cpu_count()}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    vals, total_m, total_s, gens = [], 0, 0.0, 0
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup + args.steps):
            budget = 2.0 if k < args.warmup else 10.0
            res = pool.map(_oracle_chain, [(budget, c + 1) for c in range(cores)])
            if k < args.warmup:
                continue
            m = sum(r[0] for r in res)
            s = max(r[3] for r in res)
            vals.append(m / s)
            total_m += m
            total_s += s
            gens += sum(r[2] for r in res)
    value = total_m / total_s
    desc = ("%d steady-state generations of local search (phase 1 10|V| + phase 2 2|V| + repair) of one "
            "AUX offspring each over the five n=70 instances, as %d independent single-threaded "
            "chains of the C oracle at once on %d host cores, %d steps of 10 s" % (gens, cores, cores, args.steps))
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * total_s / args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic (seeded instances of the paper's benchmark shapes)",
           "config": dict(workload_config(args.pop), parallelism="single"), "impl": "reference",
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ls_case(args):
    """One instance, one population brought to a steady state by an untimed
    two-phase walk from random colourings, then --steps phase-1 launches of
    --ls-iters iterations, each timed with CUDA events on the launching stream.
    Prints one JSON line; meant as the small case for kernel profiles."""
    import torch
    from paper_2103_10453_gb300 import inputs, plse
    G = plse.Instance(inputs.n70(args.ls_case))
    if args.launch:
        G.set_launch(*[int(x) for x in args.launch.split(",")])
    pop = args.pop
    P = torch.empty((pop, G.nv), dtype=torch.uint8, device="cuda")
    Q = torch.empty_like(P)
    st = torch.zeros((pop, 7), dtype=torch.int64, device="cuda")
    G.init_population(pop, 1, P)
    G.local_search(P, Q, pop, 0, 0, 10 * G.nv, 1, plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR,
                   stats=st)
    G.sync()
    runs = []
    for k in range(args.steps):
        src, dst = (Q, P) if k % 2 == 0 else (P, Q)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.local_search(src, dst, pop, 0, 1 + k, args.ls_iters, 1, plse.LS_PHASE1, stats=st)
        e1.record()
        G.sync()
        s = st.sum(0).tolist()
        ms = e0.elapsed_time(e1)
        runs.append({"ms": round(ms, 3), "moves_per_s": round(s[1] / ms * 1e3, 1),
                     "cand_per_iter": round(s[2] / max(s[0], 1), 2),
                     "pairs_per_iter": round(s[3] / max(s[0], 1), 2),
                     "bytes_alg": walk_bytes(dict(zip(["iterations", "moves", "cand", "pairs", "deg"], s)))})
    print(json.dumps({"case": "ls_steady", "n": 70, "r": args.ls_case, "nv": G.nv, "population": pop,
                      "iters": args.ls_iters, "launch": args.launch, "runs": runs}), flush=True)
    G.close()


def batch_pop(nv, cells=1 << 22):
    """Population of a batched job, fixed by its size (never by load): the
    largest power of two p with p*|V| <= 4M colour cells (about 4 MB per copy
    of the population), within [1024, 16384]."""
    p = 1024
    while p * 2 <= 16384 and p * 2 * nv <= cells:
        p *= 2
    return p


def run_batch_case(args):
    """Batching.  Two job sets:
      mix        -- 64 uneven instances (n in {20..70}, r ~ U[0.3, 0.8],
                    cyclic-delete or random insertion by a coin, seeds 4000+k),
                    population by the size rule of batch_pop (--batch-pop
                    overrides it);
      multistart -- 16 runs of the n = 70, r = 0.5 instance with seeds 1..16,
                    population 1024;
    --generations generations, phase-1 iterations 10|V|, optimality stop on.
    Each set runs as sequential plse_solve calls, as one plse_solve_batch call
    with 16 concurrent runs (each run on its own stream), and as one
    plse_solve_batch call in lockstep mode (every generation's local searches
    in one persistent multi-instance launch per colour-word class); every job's
    score, grid and walk counters must be identical across the three."""
    import numpy as np
    import torch
    from paper_2103_10453_gb300 import inputs, plse

    def run_set(name, grids, jobs):
        warm = plse.Instance(grids[0])
        warm.solve(*jobs[0])
        warm.close()
        torch.cuda.synchronize()
        out = {"jobs": len(jobs), "generations": args.generations, "phase1_iters": "10|V|"}
        pops = [j[0] for j in jobs]
        out["population"] = {"min": min(pops), "max": max(pops), "sum": sum(pops)}
        insts = [plse.Instance(g) for g in grids]
        t0 = time.perf_counter()
        seq = [G.solve(*j, with_stats=True) for G, j in zip(insts, jobs)]
        t_seq = time.perf_counter() - t0
        for G in insts:
            G.close()
        moves = sum(r["walks"]["moves"] for r in seq)
        out["sequential"] = {"s": round(t_seq, 3), "solves_per_s": round(len(jobs) / t_seq, 3),
                             "moves_per_s": round(moves / t_seq, 1)}
        for mode, inflight in (("concurrent", 16), ("lockstep", 0)):
            binsts = [plse.Instance(g) for g in grids]
            t0 = time.perf_counter()
            bat, rc = plse.solve_batch(binsts, jobs, max_inflight=inflight, lockstep=(mode == "lockstep"))
            t_b = time.perf_counter() - t0
            same = rc == 0 and all(a["score"] == b["score"] and np.array_equal(a["best_grid"], b["best_grid"])
                                   and a["walks"] == b["walks"] for a, b in zip(seq, bat))
            out[mode] = {"s": round(t_b, 3), "solves_per_s": round(len(jobs) / t_b, 3),
                         "moves_per_s": round(moves / t_b, 1), "speedup": round(t_seq / t_b, 3),
                         "identical": bool(same)}
            for G in binsts:
                G.close()
        out["solved_to_bound"] = sum(1 for g, r in zip(grids, seq) if r["score"] == plse.Instance(g).ub)
        return out

    res = {"case": "batch"}
    if args.batch_set in ("mix", "both"):
        grids = inputs.batch_mix(64)
        nvs = [plse.Instance(g).nv for g in grids]
        jobs = [(args.batch_pop or batch_pop(nv), args.generations, 10 * nv, 1) for nv in nvs]
        res["mix"] = run_set("mix", grids, jobs)
        res["mix"]["population_rule"] = ("largest power of two with p*|V| <= 2^22, in [1024, 16384]"
                                         if not args.batch_pop else "fixed")
    if args.batch_set in ("multistart", "both"):
        g = inputs.n70(0.5)
        nv = plse.Instance(g).nv
        grids = [g] * 16
        jobs = [(1024, args.generations, 10 * nv, 1 + k) for k in range(16)]
        res["multistart"] = run_set("multistart", grids, jobs)
    print(json.dumps(res), flush=True)


def run_serve_case(args):
    """Serving: --requests requests of the serving mix (a quarter LSC-style
    cyclic-delete requests with n in [60, 100], the rest random insertion with n
    uniform over {10..100}, r ~ U[0.3, 0.8], seeds 5000+k), --generations
    generations each with the optimality stop, phase-1 iterations 10 x empty
    cells, population by size (never by load).  Three measurements:
      sequential  -- the same requests through plse_solve one after another
                     (--serve-seq-sample K: K evenly spaced ones, the rate taken
                     from them);
      capacity    -- all requests submitted at once to one plse_server (closed
                     loop): the sustainable solves/s;
      open loop   -- Poisson arrivals at min(--rate, 0.8 x capacity) into a fresh
                     server: time to result (arrival to completion) p50/p90/p99.
    The servers admit by device memory (--serve-mem GB) and by --inflight run
    slots; every served result must equal plse_solve of the same request."""
    import numpy as np
    from paper_2103_10453_gb300 import inputs, plse
    grids = inputs.serve_mix(args.requests)
    jobs = [(inputs.serve_pop(g), args.generations, 10 * int((g == 0).sum()), 1) for g in grids]
    inflight = args.inflight or 64
    budget = int(args.serve_mem * (1 << 30))

    def same(a, b):
        return a["score"] == b["score"] and np.array_equal(a["best_grid"], b["best_grid"]) and \
            a["walks"] == b["walks"]

    def new_server():
        srv = plse.Server(max_inflight=inflight, max_queue=args.requests + 8, mem_budget=budget)
        srv.set_launch(0, args.serve_walks)
        w = srv.submit(inputs.tiny_n10(), 32, 2, 100, 1)       # warm-up, not counted
        srv.poll(w, wait_ms=-1)
        return srv

    # sequential plse_solve (all requests, or an evenly spaced sample of them)
    G = plse.Instance(inputs.tiny_n10())
    G.solve(32, 2, 100, 1)
    G.close()
    k = args.serve_seq_sample
    sample = list(range(len(grids))) if k <= 0 or k >= len(grids) else \
        sorted({(q * len(grids)) // k for q in range(k)})
    t0 = time.perf_counter()
    seq = {}
    for q in sample:
        H = plse.Instance(grids[q])
        seq[q] = H.solve(*jobs[q], with_stats=True)
        H.close()
    t_seq = time.perf_counter() - t0
    seq_rate = len(sample) / t_seq

    def identical(results):
        return all(same(results[q], seq[q]) for q in sample)

    # capacity: closed loop
    srv = new_server()
    t0 = time.perf_counter()
    tickets = [srv.submit(g, *j) for g, j in zip(grids, jobs)]
    cap_res = [srv.poll(t, wait_ms=-1) for t in tickets]
    t_cap = time.perf_counter() - t0
    cap_mem = srv.memory()
    srv.close()
    capacity = len(grids) / t_cap

    # open loop at a sustainable rate
    rate = min(args.rate, 0.8 * capacity)
    arrivals = inputs.poisson_arrivals(args.requests, rate)
    srv = new_server()
    tickets = []
    t0 = time.perf_counter()
    for (g, j), ta in zip(zip(grids, jobs), arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(srv.submit(g, *j))
    res = [srv.poll(t, wait_ms=-1) for t in tickets]
    t_all = time.perf_counter() - t0
    mem = srv.memory()
    srv.close()
    lat = np.array([r["ms_wall"] for r in res])
    qms = np.array([r["ms_queue"] for r in res])
    ok = sum(1 for r in res if r["status"] == 0)
    errors = {}
    for g, r in zip(grids, res):
        if r["status"] != 0:
            key = "%d: %s" % (r["status"], r["detail"][:80])
            errors.setdefault(key, []).append(int(g.shape[0]))
    print(json.dumps({
        "case": "serve", "requests": args.requests, "generations": args.generations,
        "phase1_iters": "10 x empty cells", "population": "2^16 / empty cells, power of two in [32, 512]",
        "max_inflight": inflight, "mem_budget_bytes": budget,
        "sequential": {"requests": len(sample), "wall_s": round(t_seq, 3), "solves_per_s": round(seq_rate, 3)},
        "capacity": {"wall_s": round(t_cap, 3), "solves_per_s": round(capacity, 3),
                     "vs_sequential": round(capacity / seq_rate, 3),
                     "identical_to_sequential": identical(cap_res),
                     "memory": cap_mem},
        "open_loop": {"rate_per_s": round(rate, 3), "requested_rate_per_s": args.rate, "ok": ok,
                      "wall_s": round(t_all, 3), "solves_per_s": round(ok / t_all, 3),
                      "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 1),
                                     "p90": round(float(np.percentile(lat, 90)), 1),
                                     "p99": round(float(np.percentile(lat, 99)), 1),
                                     "max": round(float(lat.max()), 1)},
                      "queue_ms": {"p50": round(float(np.percentile(qms, 50)), 1),
                                   "p99": round(float(np.percentile(qms, 99)), 1)},
                      "identical_to_sequential": identical(res),
                      "memory": mem},
        "generations_mean": round(float(np.mean([r["generations"] for r in res])), 2),
        "moves": sum(r["walks"]["moves"] for r in res),
        "errors": {k: {"count": len(v), "n": sorted(set(v))[:10]} for k, v in errors.items()}}),
        flush=True)


def run_pop_sweep(args):
    """Population sizes 16 .. 16384 on one synthetic (n, r) = (60, 0.7) instance
    (random insertion, seed 6000), --generations generations (default 10 here:
    pass it), phase-1 iterations 10|V|, optimality stop off: tabu moves per
    device second and the best score after the run, per population size."""
    from paper_2103_10453_gb300 import inputs, plse
    G = plse.Instance(inputs.random_insertion(60, 0.7, 6000))
    G.set_params(plse.default_params(stop_at_bound=0))
    rows = []
    for pop in (16, 64, 256, 1024, 4096, 16384):
        res = G.solve(pop, args.generations, 10 * G.nv, 1, with_stats=True)
        rows.append({"pop": pop, "best_score": res["score"], "ms_total": round(res["ms_total"], 2),
                     "ms_per_generation": round(res["ms_total"] / max(res["generations"], 1), 2),
                     "moves_per_s": round(res["walks"]["moves"] / (res["ms_local_search"] / 1e3), 1)})
    print(json.dumps({"case": "pop_sweep", "n": 60, "r": 0.7, "nv": G.nv, "ub": G.ub,
                      "generations": args.generations, "rows": rows}), flush=True)
    G.close()


def run_lsc_case(args):
    """Latin square completion (App. B): cyclic-delete instances, which have a
    complete square as witness, two per (n, r) with n in {50, 60, 70} and
    r in {0.3, ..., 0.8} (seeds 7000 + k); population --batch-pop (default
    1024), at most --generations generations, phase-1 iterations 10|V|,
    optimality stop on.  Solved fraction, generations and device time to the
    complete square."""
    import numpy as np
    from paper_2103_10453_gb300 import inputs, plse
    pop = args.batch_pop or 1024
    rows, k = [], 0
    for n in (50, 60, 70):
        for r in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8):
            for rep in range(2):
                grid = inputs.cyclic_delete(n, r, 7000 + k)[0]
                k += 1
                G = plse.Instance(grid)
                res = G.solve(pop, args.generations, 10 * G.nv, 1, with_stats=True)
                rows.append({"n": n, "r": r, "solved": res["score"] == n * n,
                             "generations": res["generations"], "ms": round(res["ms_total"], 1)})
                G.close()
    solved = [x for x in rows if x["solved"]]
    ms = np.array([x["ms"] for x in solved]) if solved else np.zeros(1)
    print(json.dumps({"case": "lsc", "instances": len(rows), "solved": len(solved),
                      "population": pop, "max_generations": args.generations,
                      "ms_to_solve": {"p50": round(float(np.percentile(ms, 50)), 1),
                                      "p90": round(float(np.percentile(ms, 90)), 1),
                                      "max": round(float(ms.max()), 1)},
                      "generations_to_solve_max": max((x["generations"] for x in solved), default=0),
                      "rows": rows}), flush=True)


def run_dist_case(args):
    """Hamming distances (Sec. 3.4) between two sets of --pop random colourings
    of the n=70, r=0.3 instance through plse_distances (bit planes, then the 64 x
    64 tile kernel); --steps timed launches after a warm-up one, CUDA events on
    the launching stream.  ALU roofline: per (pair, 32-vertex word) the kernel
    does nb XORs, nb - 1 ORs, one popcount and one add (2 nb + 1 integer
    operations), against SMs x 128 lanes x the maximum SM clock."""
    import torch
    from paper_2103_10453_gb300 import inputs, plse
    G = plse.Instance(inputs.n70(0.3))
    p = args.pop
    A = torch.empty((p, G.nv), dtype=torch.uint8, device="cuda")
    B = torch.empty_like(A)
    G.init_population(p, 1, A)
    G.init_population(p, 2, B)
    D = torch.empty((p, p), dtype=torch.int32, device="cuda")
    G.distances(A, p, B, p, D)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.distances(A, p, B, p, D)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    nw, nb = (G.nv + 31) // 32, 7
    t = statistics.median(ms) / 1e3
    ops = float(p) * p * nw * (2 * nb + 1)
    peaks = measured_peaks()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sm * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    print(json.dumps({"case": "distances", "n": 70, "r": 0.3, "nv": G.nv, "pairs": p * p,
                      "ms": round(statistics.median(ms), 3),
                      "pair_words_per_s": round(p * p * nw / t, 1),
                      "roofline": {"bound": "alu", "achieved": round(ops / t / 1e12, 3),
                                   "peak": round(peak / 1e12, 3), "unit": "Tops/s",
                                   "frac": round(ops / t / peak, 4),
                                   "peak_source": "derived: %d SMs x 128 lanes x max SM clock" % sm,
                                   "note": "includes the bit-plane pass over both sets"}}), flush=True)
    G.close()


def main():
    args = parse()
    if args.ls_case is not None:
        run_ls_case(args)
    elif args.batch:
        run_batch_case(args)
    elif args.serve:
        run_serve_case(args)
    elif args.pop_sweep:
        run_pop_sweep(args)
    elif args.lsc:
        run_lsc_case(args)
    elif args.dist_case:
        run_dist_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
