#!/usr/bin/env python3
"""Benchmark of the pilot-assignment hot path on one GB300 per rank.

Workload (one "step"): a whole solve of one synthetic 19-cell instance --
L = 19 hexagonal cells (2 rings, R = 500 m), K = 10 users per cell,
tau_p = 10, M = 256 antennas, beta = d^-3.8 * 10^(N(0, 8 dB)/10) stored as
FP32, finite-M uplink SINR, population N = 256, G = 200 generations, K-means
k = 10 seeding -- i.e. K-means, 201 population evaluations, 200 GA
generations and the best-member selection, all through the C ABI.

Printed (rank 0, one JSON line): chromosome fitness evaluations per second
over the whole job (value), GA generations per second, per-solve latency
percentiles, an end-to-end figure through host buffers, the roofline of the
step's dominant kernel (the fused solve) and of the population-wide
evaluation kernel on 2^20 chromosomes, the 512-instance batched solve, the
61-cell streamed evaluation and solve, the serving comparison (Poisson
arrivals, continuous batching vs one plain solve at a time, plus an
overload point), the PK-means island solve (Alg. 2) beside the plain solve,
the max-min objective's evaluation throughput, and the CPU oracle as a
reported baseline (one core for whole solves, every core for the
evaluation).  `--only eval | solve | stream | batch | islands` runs one part
untimed, for profilers.

Under torchrun each rank solves its own instance (seed = rank): the units
are independent, so there is no data-path collective ("weak" scaling).

`--impl reference` times the FP64 CPU oracle on the same workload (rank 0
only; other ranks exit without work).
"""
import argparse
import csv
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L, K, TAU_P, M_ANT, N_POP, G_GEN, KMEANS_K = 19, 10, 10, 256.0, 256, 200, 10
BATCH_LOG2 = 20
# DRAM bytes (read + write) per launch of the two roofline kernels, from one
# ncu capture of each; None while a kernel has changed since its capture
TRAFFIC_K_SOLVE = 146_688
TRAFFIC_EVAL = 205_056_000
METRIC = ("chromosome fitness evals/sec and GA gens/sec (L=19,K=10); "
          "p50/p99 solve latency served vs plain")
WORKLOAD = ("single instance at paper-like scale: L=19 hex cells (2 rings), K=10 users/cell, "
            "tau_p=10, M=256, FP32 beta (d^-3.8 x 8 dB log-normal), finite-M uplink SINR, "
            "population 256, 200 generations, K-means k=10 seeding; one step = one whole solve")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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
        with open(self.path) as f:
            for row in csv.reader(f):
                if len(row) < 9:
                    continue
                try:
                    sm.append(float(row[1]))
                    smax.append(float(row[2]))
                except ValueError:
                    continue
                for n, v in zip(names, row[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest x over all ranks (x itself with one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, units_per_step, seconds):
    """Whole-job throughput: every rank processes its own units (its own
    instance: weak scaling, no data-path collective) and the job takes the
    slowest rank's time."""
    return world * steps * units_per_step / seconds


def make_instance(seed):
    import numpy as np

    from paper_2511_20511_gb300 import inputs

    return inputs.instance(L, K, seed=seed, dtype=np.float32)


def oracle_solve_step(inst, seed):
    import oracle

    sp = oracle.sinr_params(oracle.FINITE_M, TAU_P, M_ANT, inst["rho"], 1.0)
    gp = oracle.ga_params(N_POP, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.05), seed)
    return oracle.solve(inst["beta"], sp, gp, G_GEN, inst["user_xy_mm"], inst["bs_xy_mm"],
                        kmeans_k=KMEANS_K)


def host_cpu():
    """Host core count and CPU model (lscpu), for the CPU baseline record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_eval_all_cores(inst, seconds=6.0):
    """The oracle's fitness evaluation (FP64, unchanged arithmetic) over
    chromosomes split across every host core: one thread per core, each
    calling the C oracle on its own chunk (ctypes releases the GIL during the
    call).  Returns (evals/s, threads, chromosomes evaluated, seconds)."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    from paper_2511_20511_gb300 import inputs

    threads = os.cpu_count() or 1
    sp = oracle.sinr_params(oracle.FINITE_M, TAU_P, M_ANT, inst["rho"], 1.0)
    chunk = 2048
    pops = [inputs.random_population(chunk, L, K, seed=50 + t) for t in range(threads)]
    oracle.fitness_batch(inst["beta"], pops[0][:8], sp)  # build + warm

    def work(t):
        n = 0
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            oracle.fitness_batch(inst["beta"], pops[t], sp)
            n += chunk
        return n

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        total = sum(ex.map(work, range(threads)))
    dt = time.perf_counter() - t0
    return total / dt, threads, total, dt


def cpu_baseline(target_s=12.0):
    """The oracle as it stands on a bounded sample: whole solves of the
    benchmark instance on one core for about target_s seconds (the solve is
    one dependent chain), and the population evaluation alone on every host
    core (chromosomes are independent) for about half that."""
    inst = make_instance(0)
    oracle_solve_step(inst, 0)  # build + warm
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle_solve_step(inst, reps)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    evals = reps * N_POP * (G_GEN + 1)
    ev_rate, threads, n_ev, ev_s = oracle_eval_all_cores(inst, seconds=target_s / 2)
    return {"value": evals / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} whole solves of the benchmark instance (N=256, G=200), "
                      f"{dt:.1f} s, FP64 plain C, single thread",
            "gens_per_s": reps * G_GEN / dt,
            "host": host_cpu(),
            "eval_all_cores": {"value": ev_rate, "unit": "evals/s", "cores": threads,
                               "kind": "oracle",
                               "sample": f"{n_ev} random chromosomes of the benchmark instance "
                                         f"evaluated in {ev_s:.1f} s, FP64 plain C, one "
                                         f"thread per host core"}}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    inst = make_instance(0)
    oracle_solve_step(inst, 0)
    for w in range(args.warmup):
        oracle_solve_step(inst, w)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve_step(inst, s)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * N_POP * (G_GEN + 1) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "K": K, "N": N_POP, "G": G_GEN},
        "gens_per_s": args.steps * G_GEN / total,
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} whole solves (N=256, G=200), FP64 plain C, "
                                   "single thread"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()


    from paper_2511_20511_gb300 import binding as B
    from paper_2511_20511_gb300 import build as pa_build
    from paper_2511_20511_gb300 import inputs

    pa_build.build()
    stream = torch.cuda.Stream(device=dev)
    inst = make_instance(rank)
    cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=M_ANT, tau_p=TAU_P, N=N_POP,
                              rho=inst["rho"], kmeans_k=KMEANS_K, seed=rank)
    ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"], stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    best = np.zeros((L, K), dtype=np.uint8)

    def timed(fn, steps, flush_between=True):
        """Per-step CUDA-event durations on the context stream (ms); the L2
        flush between steps stays outside the events."""
        ms = []
        for _ in range(steps):
            if flush_between:
                with torch.cuda.stream(stream):
                    flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    def solve_step():
        ctx.solve(G_GEN)

    if args.only == "eval":
        return run_eval_only(args, B, inputs, ctx, stream, dev, rank)
    if args.only == "stream":
        return run_stream_only(args, B, inputs, dev)
    if args.only == "batch":
        insts = c3_instances(B, inputs, 512)
        batch = B.Batch(insts)
        batch.tune(100)  # the shapes the benchmark's batched section uses
        for _ in range(args.warmup + args.steps):
            torch.cuda.nvtx.range_push("batch_solve")  # profilers can select the tuned solves
            batch.solve(100)
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"only": "batch", "solves": args.warmup + args.steps}))
        batch.close()
        ctx.close()
        return 0
    if args.only == "islands":
        icfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=M_ANT, tau_p=TAU_P, N=N_POP,
                                   rho=inst["rho"], kmeans_k=KMEANS_K, islands=5)
        ictx = B.Context(icfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
        for _ in range(args.warmup + args.steps):
            ictx.solve(G_GEN)
        print(json.dumps({"only": "islands", "solves": args.warmup + args.steps}))
        ictx.close()
        ctx.close()
        return 0
    if args.only == "solve":
        for _ in range(args.warmup + args.steps):
            ctx.solve(G_GEN)
        print(json.dumps({"only": "solve", "solves": args.warmup + args.steps}))
        ctx.close()
        return 0

    # ---- device-resident solves (value)
    for _ in range(args.warmup):
        solve_step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = B.pa_kernel_launches()
    step_ms = timed(solve_step, args.steps)
    launches = B.pa_kernel_launches() - l0
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    value = job_value(world, args.steps, N_POP * (G_GEN + 1), total_s)
    gens = job_value(world, args.steps, G_GEN, total_s)

    # ---- end to end through host buffers (pinned): fresh instance upload +
    #      solve + best member back to the host, every step
    pin_beta = torch.from_numpy(inst["beta"]).pin_memory()
    pin_xy = torch.from_numpy(inst["user_xy_mm"]).pin_memory()
    pin_bs = torch.from_numpy(inst["bs_xy_mm"]).pin_memory()
    keep = (pin_beta.numpy(), pin_xy.numpy(), pin_bs.numpy())

    def e2e_step():
        B.pa_load_instance(ctx.handle, *keep)
        B.pa_solve(ctx.handle, G_GEN, best)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    e2e_ms = timed(e2e_step, args.steps, flush_between=False)
    wall_e2e = time.perf_counter() - t0
    e2e_total = max_over_ranks(max(sum(e2e_ms) / 1e3, wall_e2e), world, dev)
    h2d = keep[0].nbytes + keep[1].nbytes + keep[2].nbytes
    d2h = best.nbytes + 8

    # ---- the step's dominant kernel: the fused solve k_solve (all G
    #      generations and the final evaluation in one cluster launch), timed
    #      alone through pa_step on the context stream
    ctas = B.pa_solve_cluster_ctas(ctx.handle)
    ctx.kmeans_seed()

    def generations_step():
        B.pa_step(ctx.handle, G_GEN)

    generations_step()
    ks_ms = timed(generations_step, max(3, min(args.steps, 10)))
    ks_avg = statistics.mean(ks_ms) / 1e3

    # ---- population-wide evaluation kernel on 2^20 chromosomes (> L2)
    nb = 1 << BATCH_LOG2
    pop = inputs.random_population_torch(nb, L, K, seed=1000 + rank, device=dev)
    fit = torch.empty(nb, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        torch.cuda.current_stream().wait_stream(torch.cuda.default_stream(dev))

    def eval_step():
        B.pa_eval_population(ctx.handle, pop, fit)

    for _ in range(max(3, args.warmup)):
        eval_step()
    stream.synchronize()
    ev_ms = timed(eval_step, max(args.steps, 10), flush_between=False)
    ev_avg = statistics.mean(ev_ms) / 1e3
    evals_batch = nb / ev_avg
    words = L * L * K  # algorithmic shared-memory words per chromosome (Eq. 5 gathers)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    peak_gword = n_sms * 32 * sm_max * 1e6 / 1e9
    achieved_gword = nb * words / ev_avg / 1e9
    path = (f"shared-memory gather data path: 32 x 4-byte words/clk/SM x {n_sms} SMs x "
            f"{sm_max:.0f} MHz")
    # the step's dominant kernel: (G+1) evaluations of N members per launch
    ks_units = N_POP * (G_GEN + 1)
    ks_gword = ks_units * words / ks_avg / 1e9
    roofline = {"bound": "alu", "kernel": "k_solve (fused GA run: G generations + final "
                                          "evaluation, one cluster)",
                "achieved": ks_gword, "peak": peak_gword, "unit": "Gword/s",
                "frac": ks_gword / peak_gword, "traffic": TRAFFIC_K_SOLVE, "path": path,
                "units_per_launch": ks_units, "words_per_unit": words,
                "avg_launch_ms": ks_avg * 1e3, "cluster_ctas": ctas,
                "frac_of_cluster_sms": ks_gword / (peak_gword * ctas / n_sms) if ctas > 0
                else None,
                "note": "one instance: 201 dependent generations on one cluster, latency-bound"}
    roofline_eval = {"bound": "alu", "kernel": "k_eval_f32_pilot (population fitness, FP32)",
                     "achieved": achieved_gword, "peak": peak_gword, "unit": "Gword/s",
                     "frac": achieved_gword / peak_gword, "traffic": TRAFFIC_EVAL, "path": path,
                     "units_per_launch": nb, "words_per_unit": words,
                     "avg_launch_ms": ev_avg * 1e3}

    lat = sorted(step_ms)

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "K": K, "tau_p": TAU_P, "M": M_ANT,
                   "N": N_POP, "G": G_GEN, "kmeans_k": KMEANS_K, "sinr": "finite_m",
                   "l2": "L2 flushed (256 MB write) between timed steps; the 2^20-chromosome "
                         "evaluation input (199 MB) is larger than L2"},
        "gens_per_s": gens,
        "solve_latency_ms": {"p50": pct(50), "p99": pct(99), "mean": statistics.mean(lat)},
        "eval_batch": {"chromosomes": nb, "evals_per_s": evals_batch * world,
                       "avg_launch_ms": ev_avg * 1e3},
        "roofline": roofline,
        "roofline_eval_batch": roofline_eval,
        "e2e": {"value": job_value(world, args.steps, N_POP * (G_GEN + 1), e2e_total),
                "unit": "evals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "pa_load_instance (pinned host beta + positions) + pa_solve (best row "
                        "and fitness back to host) per step"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_batched:
        line["batched_c3"] = run_batched(B, inputs)
        line["streamed_c5"] = run_streamed(B, inputs, dev)
        line["serving_c4"] = run_serving(B, inputs, seconds=args.serve_seconds,
                                         tick=args.serve_tick)
        # twice the rate: beyond what one solve at a time can sustain
        line["serving_c4"]["overload_4000_per_s"] = run_serving(
            B, inputs, rate=4000.0, seconds=max(0.5, args.serve_seconds / 2), tick=args.serve_tick)
    line["islands_pkmeans"] = run_islands(B, inputs, dev)
    line["objective_min_sinr"] = run_min_sinr(B, inputs, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def c3_instances(B, inputs, n=512, seed0=0):
    """Batched uneven instances: L from {7, 19, 37}, K uniform in [4, 16],
    tau_p = K, M = 256 (finite-M SINR), N = 128, FP32 beta, seeds 0..n-1."""
    import numpy as np

    rng = np.random.default_rng(seed0)
    out = []
    for i in range(n):
        L = int(rng.choice([7, 19, 37]))
        K = int(rng.integers(4, 17))
        inst = inputs.instance(L, K, seed=seed0 + i, dtype=np.float32)
        cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=256.0, tau_p=K, N=128,
                                  rho=inst["rho"], seed=seed0 + i)
        out.append(dict(cfg=cfg, beta=inst["beta"], user_xy_mm=inst["user_xy_mm"],
                        bs_xy_mm=inst["bs_xy_mm"]))
    return out


def run_batched(B, inputs, G=100, n=512, reps=3, tune_generations=None):
    """512 uneven instances: one batched solve (persistent cluster launches
    per kernel variant, CUDA graph, shapes tuned on the batch itself with
    the solve's generation count) against the same instances solved one
    launch sequence per instance."""
    import numpy as np
    import torch

    insts = c3_instances(B, inputs, n)
    batch = B.Batch(insts)
    chosen = batch.tune(G if tune_generations is None else tune_generations)
    batch.solve(G)  # capture + warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        batch.solve(G)
    t_batch = (time.perf_counter() - t0) / reps
    rows, fits = batch.solve(G)
    done_ms = np.sort(batch.completion_times_ms())  # per instance, since the batch started
    _, cta_threads, lat_split, resident, _ = batch.group_tiling()
    batch.close()
    ctxs = [B.Context(d["cfg"], d["beta"], d["user_xy_mm"], d["bs_xy_mm"]) for d in insts]
    ctxs[0].solve(G)
    lat = []
    done_seq = []  # completion of each instance since all were submitted at t0
    t0 = time.perf_counter()
    same = True
    for i, c in enumerate(ctxs):
        t1 = time.perf_counter()
        best, bf = c.solve(G)
        t2 = time.perf_counter()
        lat.append(t2 - t1)
        done_seq.append(t2 - t0)
        same = same and bool((best == rows[i]).all()) and bool(bf == fits[i])
    t_seq = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    lat.sort()
    evals = sum(d["cfg"].N for d in insts) * (G + 1)
    # gather words of all evaluations (L^2 K per chromosome), against the
    # shared-memory data path of the whole GPU
    words = sum(d["cfg"].N * d["cfg"].L * d["cfg"].L * d["cfg"].K for d in insts) * (G + 1)
    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = n_sms * 32 * peaks().get("sm_max_mhz", 2070.0) * 1e6 / 1e9
    ach = words / t_batch / 1e9
    q = lambda v, p: float(v[min(len(v) - 1, int(round(p / 100.0 * (len(v) - 1))))])  # noqa: E731
    done_seq = np.sort(np.array(done_seq)) * 1e3
    return {"instances": n, "generations": G, "population": 128,
            "batched": {"seconds_per_batch": t_batch, "solves_per_s": n / t_batch,
                        "evals_per_s": evals / t_batch, "cluster_sizes": [int(x) for x in chosen],
                        "cta_threads": [int(x) for x in cta_threads],
                        "latency_split": [int(x) for x in lat_split],
                        "resident_clusters": [int(x) for x in resident],
                        "completion_ms": {"p50": q(done_ms, 50), "p99": q(done_ms, 99),
                                          "max": float(done_ms[-1]),
                                          "what": "each instance's completion since the batch "
                                                  "started (device clock)"},
                        "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                                     "unit": "Gword/s", "frac": ach / peak,
                                     "what": "all gathers of the batch / batch wall time"}},
            "one_launch_sequence_per_instance": {
                "seconds": t_seq, "solves_per_s": n / t_seq, "evals_per_s": evals / t_seq,
                "completion_ms": {"p50": q(done_seq, 50), "p99": q(done_seq, 99),
                                  "max": float(done_seq[-1]),
                                  "what": "each instance's completion since all were submitted"},
                "per_solve_p50_ms": 1e3 * lat[len(lat) // 2],
                "per_solve_p99_ms": 1e3 * lat[int(0.99 * (len(lat) - 1))]},
            "speedup": t_seq / t_batch, "identical_results": same,
            "timing": "host wall clock around synchronous calls (batched: graph replay)"}


def run_streamed(B, inputs, dev, n=1 << 17, reps=5):
    """61 cells x 32 users (1952 users), tau_p = 32, M = 512: the gain table
    (476 KB) exceeds shared memory and is streamed in BS-column tiles.
    Throughput of the population evaluation on 2^17 random chromosomes
    (256 MB > L2), with 64 sampled outputs checked against the oracle."""
    import numpy as np
    import torch

    import oracle

    L5, K5 = 61, 32
    inst = inputs.instance(L5, K5, seed=0, dtype=np.float32)
    cfg = B.pa_config_default(L5, K5, mode=B.PA_SINR_FINITE_M, M=512.0, tau_p=K5, N=2048,
                              rho=inst["rho"], kmeans_k=K5)
    ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    pop = inputs.random_population_torch(n, L5, K5, seed=7, device=dev)
    fit = torch.empty(n, dtype=torch.float32, device=dev)
    for _ in range(2):
        ctx.eval_population(pop, fit)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.eval_population(pop, fit)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    idx = np.sort(np.random.default_rng(1).choice(n, 64, replace=False))
    sub = pop[torch.from_numpy(idx).to(dev)].cpu().numpy()
    sp = oracle.sinr_params(oracle.FINITE_M, K5, 512.0, inst["rho"], 1.0)
    ref = oracle.fitness_batch(inst["beta"], sub, sp)
    got = fit.cpu().numpy()[idx].astype(np.float64)
    # the whole configured solve: N = 2048, 500 generations (per-generation
    # evaluation and GA launches; the table does not fit the fused kernel)
    G5 = 500
    ctx.solve(5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.solve(G5)
    t_solve = time.perf_counter() - t0
    ctx.close()
    words = L5 * L5 * K5
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sms * 32 * peaks().get("sm_max_mhz", 2070.0) * 1e6 / 1e9
    ach = n * words / (ms / 1e3) / 1e9
    return {"workload": "61 hex cells x 32 users, tau_p=32, M=512, finite-M SINR, FP32 beta "
                        "streamed in BS-column tiles (TMA bulk copies)",
            "chromosomes": n, "avg_launch_ms": ms, "evals_per_s": n / (ms / 1e3),
            "input_GBps": n * L5 * K5 / (ms / 1e3) / 1e9,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gword/s",
                         "frac": ach / peak, "words_per_unit": words},
            "sampled_max_rel_err_vs_oracle": float(np.max(np.abs(got - ref) / ref)),
            "solve": {"population": 2048, "generations": G5, "seconds": t_solve,
                      "evals_per_s": 2048 * (G5 + 1) / t_solve,
                      "gens_per_s": G5 / t_solve}}


def run_serving(B, inputs, rate=2000.0, seconds=10.0, G=40, N=64, tick=40, budget=40 << 30):
    """Poisson arrivals (rate per second for `seconds`), each request a solve
    of a fresh seeded instance with L in {7, 19}, K in {8, 16} (tau_p = K,
    M = 256, finite-M SINR, N = 64, G = 40, FP32 beta).  Served: the
    continuous-batching server (slots admitted under a device-memory budget,
    populations resident, `tick` generations per scheduling round).  Plain:
    one resident context per (L, K), requests solved one at a time in arrival
    order (load instance + pa_solve).  Latency = completion - arrival."""
    import numpy as np

    rng = np.random.default_rng(0)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.5)))
    arr = arr[arr < seconds]
    n = len(arr)
    shapes = [(int(rng.choice([7, 19])), int(rng.choice([8, 16]))) for _ in range(n)]
    insts = make_serving_instances(shapes)
    base = B.pa_config_default(7, 8, mode=B.PA_SINR_FINITE_M, M=256.0, N=N,
                               rho=insts[0]["rho"])

    def pct(v, p):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(p / 100.0 * (len(v) - 1))))]

    # ---- served
    srv = B.Server(base, G, tick, budget)
    for i in range(min(8, n)):  # warm the slot pool and kernels
        srv.submit(-1 - i, shapes[i][0], shapes[i][1], 1, insts[i]["beta"],
                   insts[i]["user_xy_mm"], insts[i]["bs_xy_mm"])
    srv.run_until_idle()
    # no cyclic-GC pauses inside the timed replays (the instances are tens of
    # thousands of objects); the same for the plain replay below
    gc.collect()
    gc.freeze()
    gc.disable()
    done_at = {}
    results = {}
    t0 = time.perf_counter()
    nxt = 0
    polls = 0
    while len(done_at) < n:
        now = time.perf_counter() - t0
        while nxt < n and arr[nxt] <= now:
            L, K = shapes[nxt]
            srv.submit(nxt, L, K, 10_000 + nxt, insts[nxt]["beta"], insts[nxt]["user_xy_mm"],
                       insts[nxt]["bs_xy_mm"])
            nxt += 1
        done, active, pending = srv.poll()
        polls += 1
        tnow = time.perf_counter() - t0
        for rid, best, fit in done:
            if rid >= 0:
                done_at[rid] = tnow
                results[rid] = fit
        if not done:
            # nothing finished: wait for a tick in flight, at most until the
            # next arrival is due; with nothing in flight, sleep until then
            until = (arr[nxt] - tnow) if nxt < n else 0.002
            if active > 0:
                srv.wait(int(max(0.0, min(until, 0.002)) * 1e6))
            elif pending == 0 and nxt < n:
                time.sleep(max(0.0, until))
    gc.enable()
    served_lat = [done_at[i] - arr[i] for i in range(n)]
    served_span = max(done_at.values()) - arr[0]
    stats = srv.stats()
    srv.close()

    # ---- plain: one solve at a time in arrival order
    ctxs = {}
    for (L, K) in set(shapes):
        i = shapes.index((L, K))
        cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=256.0, tau_p=K, N=N,
                                  rho=insts[i]["rho"], kmeans_k=K)
        ctxs[(L, K)] = B.Context(cfg, insts[i]["beta"], insts[i]["user_xy_mm"],
                                 insts[i]["bs_xy_mm"])
        ctxs[(L, K)].solve(G)
    plain_lat = []
    same = True
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    for i in range(n):
        now = time.perf_counter() - t0
        if now < arr[i]:
            time.sleep(arr[i] - now)
        c = ctxs[shapes[i]]
        B.pa_load_instance(c.handle, insts[i]["beta"], insts[i]["user_xy_mm"],
                           insts[i]["bs_xy_mm"])
        B.pa_set_seed(c.handle, 10_000 + i)
        _, bf = c.solve(G)
        plain_lat.append(time.perf_counter() - t0 - arr[i])
        same = same and bool(bf == results[i])
    plain_span = time.perf_counter() - t0 - arr[0]
    gc.enable()
    gc.unfreeze()
    for c in ctxs.values():
        c.close()
    ms = lambda x: 1e3 * x  # noqa: E731
    return {"requests": n, "rate_per_s": rate, "seconds": seconds, "generations": G,
            "population": N, "tick_generations": tick, "budget_bytes": budget,
            "served": {"p50_ms": ms(pct(served_lat, 50)), "p99_ms": ms(pct(served_lat, 99)),
                       "p999_ms": ms(pct(served_lat, 99.9)), "solves_per_s": n / served_span,
                       "polls": polls, "slots": stats["slots"],
                       "slot_bytes": stats["used_bytes"]},
            "plain_sequential": {"p50_ms": ms(pct(plain_lat, 50)),
                                 "p99_ms": ms(pct(plain_lat, 99)),
                                 "p999_ms": ms(pct(plain_lat, 99.9)),
                                 "solves_per_s": n / plain_span},
            "identical_results": same,
            "timing": "host wall clock; arrivals replayed in real time"}


def _serving_instance(job):
    """One serving request's instance (runs in a worker process)."""
    import numpy as np

    from paper_2511_20511_gb300 import inputs

    i, L, K = job
    return inputs.instance(L, K, seed=10_000 + i, dtype=np.float32)


def make_serving_instances(shapes):
    """The fresh instance of every request (seed 10000 + request id), built on
    all host cores by spawned worker processes before the replay starts."""
    import concurrent.futures as cf
    import multiprocessing as mp

    jobs = [(i, L, K) for i, (L, K) in enumerate(shapes)]
    workers = max(1, min(os.cpu_count() or 1, 32))
    if len(jobs) < 256 or workers == 1:
        return [_serving_instance(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=workers,
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_serving_instance, jobs, chunksize=128))


def run_islands(B, inputs, dev, steps=10):
    """The PK-means GA (Alg. 2) on the benchmark instance: C = 5 islands
    found by K-means over the population every 3 generations (Sec. 6.1),
    N = 256, G = 200, finite-M SINR, FP32 -- one cluster launch of the fused
    solve in island mode with the K-means of the population inside -- beside
    the plain one-population solve of the same instance; plus the island
    K-means alone (one re-clustering of 256 chromosomes)."""
    import numpy as np
    import torch

    inst = make_instance(0)
    out = {}
    for C in (0, 5):
        cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=M_ANT, tau_p=TAU_P, N=N_POP,
                                  rho=inst["rho"], kmeans_k=KMEANS_K, islands=C)
        ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
        ctx.solve(G_GEN)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            t0 = time.perf_counter()
            _, bf = ctx.solve(G_GEN)
            ms.append(1e3 * (time.perf_counter() - t0))
        key = "plain" if C == 0 else f"islands_{C}"
        out[key] = {"ms_per_solve": statistics.median(ms), "best_fitness": bf,
                    "evals_per_s": N_POP * (G_GEN + 1) / (statistics.median(ms) / 1e3),
                    "gens_per_s": G_GEN / (statistics.median(ms) / 1e3)}
        if C:
            pop, _, _ = ctx.get_population(with_fitness=False)
            dpop = torch.from_numpy(pop).to(dev)
            lab = torch.empty(N_POP, dtype=torch.int32, device=dev)
            B.pa_island_cluster(ctx.handle, dpop, 0, lab)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(20):
                B.lib().pa_island_cluster(ctx.handle, B._dev_ptr(dpop), 0, B._dev_ptr(lab), None)
            e1.record()
            e1.synchronize()
            out[key]["kmeans_ms"] = e0.elapsed_time(e1) / 20
            out[key]["labels_per_island"] = np.bincount(lab.cpu().numpy(), minlength=C).tolist()
        ctx.close()
    out["what"] = ("host wall clock per whole solve (K-means seeding + 200 generations + final "
                   "evaluation); islands: one cluster launch of the fused solve in island mode, "
                   "the population K-means every third generation inside it")
    return out


def run_min_sinr(B, inputs, dev):
    """The max-min objective (Sec. 2): population evaluation of the 2^20
    chromosomes of the evaluation roofline, on the same instance and
    kernels, smallest SINR instead of the sum SE."""
    import torch

    inst = make_instance(0)
    nb = 1 << BATCH_LOG2
    pop = inputs.random_population_torch(nb, L, K, seed=1000, device=dev)
    res = {}
    for obj in (0, 1):
        cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=M_ANT, tau_p=TAU_P, N=N_POP,
                                  rho=inst["rho"], objective=obj)
        ctx = B.Context(cfg, inst["beta"])
        fit = torch.empty(nb, dtype=torch.float32, device=dev)
        for _ in range(3):
            B.pa_eval_population(ctx.handle, pop, fit)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            B.pa_eval_population(ctx.handle, pop, fit)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 10
        res["min_sinr" if obj else "sum_se"] = {"avg_launch_ms": ms, "evals_per_s": nb / (ms / 1e3)}
        ctx.close()
    return res


def run_stream_only(args, B, inputs, dev):
    """Only the 61-cell, 32-user streamed evaluation of 2^17 chromosomes (for
    profilers)."""
    import numpy as np
    import torch

    inst = inputs.instance(61, 32, seed=0, dtype=np.float32)
    cfg = B.pa_config_default(61, 32, mode=B.PA_SINR_FINITE_M, M=512.0, tau_p=32, N=2048,
                              rho=inst["rho"], kmeans_k=32)
    ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    n = 1 << 17
    pop = inputs.random_population_torch(n, 61, 32, seed=7, device=dev)
    fit = torch.empty(n, dtype=torch.float32, device=dev)
    for _ in range(args.warmup + args.steps):
        ctx.eval_population(pop, fit)
    torch.cuda.synchronize()
    print(json.dumps({"only": "stream", "launches": args.warmup + args.steps,
                      "checksum": float(fit.double().sum().item())}))
    ctx.close()
    return 0


def run_eval_only(args, B, inputs, ctx, stream, dev, rank):
    """Only the population evaluation of 2^20 chromosomes (for profilers)."""
    import torch

    nb = 1 << BATCH_LOG2
    pop = inputs.random_population_torch(nb, L, K, seed=1000 + rank, device=dev)
    fit = torch.empty(nb, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    for _ in range(args.warmup + args.steps):
        B.pa_eval_population(ctx.handle, pop, fit)
    stream.synchronize()
    print(json.dumps({"only": "eval", "launches": args.warmup + args.steps,
                      "checksum": float(fit.double().sum().item())}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-tick", type=int, default=40,
                    help="generations per scheduling tick of the serving comparison (the "
                         "default, G = 40, finishes a request in the tick that admits it)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson arrival window of the serving comparison "
                         "(the configured workload: 10 s at 2000 requests/s)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-instance batched-solve comparison")
    ap.add_argument("--only", choices=["all", "eval", "solve", "stream", "batch", "islands"],
                    default="all",
                    help="eval / solve / stream / batch / islands: run only the 2^20-chromosome "
                         "evaluation, the solves, the 61x32 streamed evaluation, the "
                         "512-instance batched solve (tuned shapes) or the island solves, "
                         "untimed (for profilers)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
