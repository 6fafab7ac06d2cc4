#!/usr/bin/env python3
"""Throughput of full population-annealing runs on one GB300 (or N, one
independent run per GPU).

Metric: spin-flip attempts per ns, L^2 theta sum_{i>=1} R_i / t_run (the
inverse of the paper's time per spin flip, Sec. 5 Eq. spinflip). One bench
step is one complete run of the paper's default workload: L = 64,
R = 20000, theta = 100, beta 0 -> 1 in steps of 0.005 (200 steps),
bit-packed spins, a new seed every step (seed = 2 + step). Inputs are
synthetic (random initial spins generated on the device).

  value   device time (CUDA events on the run's stream) of pa_reset +
          pa_launch, i.e. init, 200 temperature steps as one CUDA graph;
  e2e     wall clock of the public API a user calls: pa_create (allocation,
          host tables uploaded), pa_run, pa_observables (rows read back),
          pa_destroy;
  roofline  the sweep kernel's average launch time from CUDA events captured
          in the same graph, against the integer-pipe peak of the device;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload on
          all host cores (independent processes).

--impl reference times that oracle alone on the same metric and workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/ns (batched vs single-run, bit-exact); p50/p99 run latency"
UNIT = "flips/ns"
WL = dict(L=64, R=20000, theta=100, beta_f=1.0, dbeta=0.005, dim=2, potts_q=0)
DEFAULT_WL = dict(WL)


def workload_label():
    lattice = (f"2D Ising L={WL['L']} periodic" if WL["dim"] == 2 else
               f"3D Ising (simple cubic) L={WL['L']}^3 periodic")
    if WL["potts_q"]:
        lattice = f"2D {WL['potts_q']}-state Potts L={WL['L']} periodic"
    if WL["dbeta"] > 0:
        n = int(round(WL["beta_f"] / WL["dbeta"]))
        steps = f"dbeta={WL['dbeta']:g} ({n} steps)"
    else:
        steps = "adaptive dbeta (histogram overlap 0.85, one host decision per step)"
    return f"plain PA, {lattice}, R={WL['R']}, theta={WL['theta']}, beta 0->1 {steps}, bit-packed spins"


def sites():
    return WL["L"] ** WL["dim"]


WORKLOAD = workload_label()
# paper, program summary: 17 s on a Tesla K80 for this workload with multi-spin
# coding (151 s single-spin); attempts = 4096 * 100 * sum R_i ~ 1.64e12
PAPER_K80_MSC_FLIPS_PER_NS = 4096 * 100 * 200 * 20000 / 17.0 / 1e9

# Integer work of one attempt (one site update) of the sweep kernel:
#  - a quarter of a Philox4x32-10 block: 20 wide 32x32->64 multiplies and 20
#    three-input XORs per block; with the counter layout of the sweep the two
#    first-round products are the same for all lanes of a warp, leaving 16
#    lane-varying multiplies and 18 XORs, i.e. 4 and 4.5 per attempt;
#  - one threshold comparison and ~0.5 logic ops (15 LOP3 per 32-site word).
#    (The kernel compares each word with both thresholds and lets the
#    neighbour count pick, two compares per site: cheaper than selecting the
#    threshold; the count here is the algorithmic one.)
# A wide multiply occupies the FMA-heavy pipe for 4 cycles per warp (32 lanes
# per SM per clock, measured: the Philox-only kernel reaches 84% of it); LOP3
# and compares go to the ALU pipe (64 lanes per SM per clock).
MUL_OPS_PER_ATTEMPT = 4.0
ALU_OPS_PER_ATTEMPT = 4.5 + 1.0 + 0.5
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_sweep_bits_L64_R20000_theta100.md")


def kernel_source_hash() -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_1703_03676_gb300", "csrc", "pa_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def clocks_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def clocks_sampler_stop(h, path, gpu_index):
    p, f = h
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def _oracle_sample(args):
    """One worker: the oracle on R_s replicas of the workload `wl` for n_steps
    temperature steps; returns (attempts, seconds). (Workers are spawned, so
    the workload comes in the arguments, not from this module's globals.)"""
    R_s, n_steps, seed, wl = args
    sys.path.insert(0, ROOT)
    from oracle.pa_oracle import PopulationAnnealing
    t0 = time.perf_counter()
    pa = PopulationAnnealing(wl["L"], R_s, wl["theta"], beta_f=wl["beta_f"], dbeta=wl["dbeta"], seed=seed,
                             dim=wl["dim"], potts_q=wl["potts_q"])
    att = 0
    for _ in range(n_steps):
        rec = pa.step()
        att += wl["L"] ** wl["dim"] * wl["theta"] * rec.R
    return att, time.perf_counter() - t0


def cpu_oracle(workers: int, R_s: int, n_steps: int, seed0: int):
    ctx = mp.get_context("spawn")
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_sample, [(R_s, n_steps, seed0 + w, dict(WL)) for w in range(workers)])
    wall = time.perf_counter() - t0
    att = sum(a for a, _ in res)
    return att / wall / 1e9, att, wall


def cpu_baseline_obj(workers, R_s, n_steps):
    v, att, wall = cpu_oracle(workers, R_s, n_steps, 9000)
    return {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} independent oracle processes, each the first {n_steps} temperature step(s) of the "
                      f"workload with R={R_s} (not R={WL['R']}): {att:.3e} attempts in {wall:.1f} s wall"}


# ------------------------------------------------------------------ helpers
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, dist


def max_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, ws, dist = dist_setup()
    if rank != 0:
        return 0
    workers = os.cpu_count() or 1
    R_s = args.ref_replicas
    for _ in range(args.warmup):
        cpu_oracle(workers, max(8, R_s // 4), 1, 500)
    tot_att, tot_wall = 0, 0.0
    for k in range(args.steps):
        _, att, wall = cpu_oracle(workers, R_s, 1, 1000 + 100 * k)
        tot_att += att
        tot_wall += wall
    v = tot_att / tot_wall / 1e9
    sample = (f"each step: {workers} independent oracle processes, each the first temperature step of the workload "
              f"with R={R_s} (not R={WL['R']})")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": {"workload": workload_label(), "sample_replicas": R_s},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ engine arm
def run_engine(args):
    import torch

    import paper_1703_03676_gb300 as eng
    rank, ws, dist = dist_setup()
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)  # the engine's stream; the timing events are recorded on it
    torch.cuda.set_stream(stream)
    L, theta = WL["L"], WL["theta"]
    seed_of = lambda k: 2 + k + 100000 * rank  # noqa: E731
    fmt = {"bits": eng.SPIN_BITS32, "msc": eng.SPIN_MSC32, "int8": eng.SPIN_INT8,
           "replica": eng.SPIN_REPLICA8}[args.format]
    cfg = eng.PAConfig(L=L, R=WL["R"], theta=theta, beta_f=WL["beta_f"], dbeta=WL["dbeta"], seed=seed_of(0),
                       spin_format=fmt, use_graph=True, profile=args.profile, dim=WL["dim"], potts_q=WL["potts_q"],
                       group_threads=args.group_threads or 0)
    run = eng.PARun(cfg, stream=stream)
    adaptive = not (WL["dbeta"] > 0)  # steps chosen by histogram overlap, one host decision per step
    n_steps = None if adaptive else int(round(WL["beta_f"] / WL["dbeta"]))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (126 MB)

    def one(seed):
        run.reset(seed)
        run.launch()

    for w in range(args.warmup):
        one(seed_of(10_000 + w))
        run.sync()
    if args.profile:
        run.phase_times()  # drop warm-up
        base = run.phase_times()
    torch.cuda.synchronize(dev)
    barrier(dist)
    clk_path = os.path.join(tempfile.gettempdir(), f"pa_clocks_{os.getpid()}.csv")
    clk = clocks_sampler_start(clk_path)
    time.sleep(0.3)
    dev_ms = 0.0
    attempts = 0
    launches = 0
    per_step_ms = []
    for k in range(args.steps):
        flush.fill_(k)  # evict L2 between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one(seed_of(k))
        e1.record(stream)
        run.sync()
        ms = e0.elapsed_time(e1)
        rows = run.rows()
        assert adaptive or len(rows) == n_steps + 1
        attempts += sites() * theta * int(rows["R"][1:].sum())
        launches += 2 + 6 * (len(rows) - 1)
        dev_ms += ms
        per_step_ms.append(ms)
    torch.cuda.synchronize(dev)
    barrier(dist)
    clocks = clocks_sampler_stop(clk, clk_path, local)
    t_max = max_over_ranks(dev_ms, dist)
    att_all = sum_over_ranks(attempts, dist)
    value = att_all / (t_max * 1e6)

    roofline = None
    if args.profile and args.format == "bits":
        pt = run.phase_times()
        sw_ms = pt["sweep"][0] - base["sweep"][0]
        sw_n = pt["sweep"][1] - base["sweep"][1]
        avg_ms = sw_ms / max(sw_n, 1)
        att_per_launch = attempts / max(sw_n, 1)
        sm = torch.cuda.get_device_properties(dev).multi_processor_count
        clk_max = clocks.get("sm_max_mhz") or 2070.0
        apn = att_per_launch / (avg_ms * 1e6)  # attempts per ns in the sweep kernel
        mul_peak = sm * 32 * clk_max * 1e6 / 1e9  # Gop/s, wide multiplies
        alu_peak = sm * 64 * clk_max * 1e6 / 1e9  # Gop/s, ALU pipe
        achieved = MUL_OPS_PER_ATTEMPT * apn
        default_wl = WL == DEFAULT_WL
        shape = run.launch_shape()
        gt = shape["group_threads"]
        roofline = {"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Gop/s",
                    "frac": achieved / mul_peak, "traffic": profiled_traffic() if default_wl else None,
                    "kernel": f"k_sweep_bits<{L},{gt}" + (",3>" if WL["dim"] == 3 else ">"), "launch": shape,
                    "ops": "lane-varying 32x32->64 multiplies of Philox4x32-10, 4 per attempt",
                    "peak_note": "FMA-heavy pipe: SMs x 32 wide multiplies/clk x max SM clock (derived)",
                    "alu_pipe": {"achieved": ALU_OPS_PER_ATTEMPT * apn, "peak": alu_peak,
                                 "frac": ALU_OPS_PER_ATTEMPT * apn / alu_peak,
                                 "ops": "4.5 Philox XOR + 1 compare + 0.5 logic per attempt"},
                    "attempts_per_ns": apn, "launch_ms": avg_ms, "launches": sw_n,
                    "share_of_step": sw_ms / dev_ms if dev_ms else None,
                    "algorithmic_bytes_per_launch": 2 * att_per_launch / (sites() * theta) * (sites() / 8)}
        try:
            roofline["rng_ceiling_words_per_ns"] = eng.measure_rng_peak(2048, stream)
        except Exception as e:  # measurement only
            roofline["rng_ceiling_words_per_ns"] = f"unavailable: {e}"
        try:
            # measured issue rates of the instruction classes behind the derived peaks
            mp = {"wide_mul": eng.measure_pipe_peak(eng.PIPE_WIDE_MUL, 16384, stream),
                  "lop3": eng.measure_pipe_peak(eng.PIPE_LOP3, 16384, stream),
                  "imad": eng.measure_pipe_peak(eng.PIPE_IMAD, 16384, stream)}
            roofline["measured_pipe_peaks_gops"] = mp
            roofline["frac_of_measured_wide_mul"] = achieved / mp["wide_mul"]
            roofline["alu_pipe"]["frac_of_measured_lop3"] = ALU_OPS_PER_ATTEMPT * apn / mp["lop3"]
        except Exception as e:  # measurement only
            roofline["measured_pipe_peaks_gops"] = f"unavailable: {e}"

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e and not adaptive:
        wall = 0.0
        att_e2e = 0
        h2d = d2h = 0
        for k in range(max(1, args.e2e_steps)):
            t0 = time.perf_counter()
            r2 = eng.PARun(eng.PAConfig(L=L, R=WL["R"], theta=theta, beta_f=WL["beta_f"], dbeta=WL["dbeta"],
                                        seed=seed_of(50_000 + k), spin_format=fmt, dim=WL["dim"],
                                        potts_q=WL["potts_q"]), stream=stream)
            r2.run()
            rows = r2.rows()
            r2.close()
            wall += time.perf_counter() - t0
            att_e2e += sites() * theta * int(rows["R"][1:].sum())
            # host tables uploaded by pa_create (thresholds, level weights, key)
            # per step T4-1, T8-1 (and T12-1 in 3D, T1-1..T4-1 for Potts); level weights per level
            thr_words = 3 if WL["dim"] == 3 else (6 if WL["potts_q"] else 2)
            nlev = (2 * sites() if WL["potts_q"] else WL["dim"] * sites() // 2) + 1
            h2d = thr_words * (n_steps + 1) * 4 + nlev * 8 + 8
            d2h = (n_steps + 1) * 128 + 4 + rows.nbytes
        wmax = max_over_ranks(wall, dist)
        e2e = {"value": sum_over_ranks(att_e2e, dist) / (wmax * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "wall clock of pa_create + pa_run + pa_observables + pa_destroy per run"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_obj(os.cpu_count() or 1, args.cpu_replicas, 1)

    run.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak",
                "vs_baseline": value / PAPER_K80_MSC_FLIPS_PER_NS if WL == DEFAULT_WL else None,
                "dtype": "u32", "data": "synthetic",
                "config": {"workload": workload_label() if args.format == "bits" else workload_label().replace(
                               "bit-packed spins", f"{args.format} spins"),
                           "seeds": "2+step (+100000*rank)", "spin_format": args.format,
                           "group_threads": args.group_threads or "auto",
                           "l2": "flushed between timed steps (256 MB write)",
                           "baseline_ref": "paper K80 multi-spin-coded run, 17 s for this workload",
                           "parallelism": f"independent runs x{ws}"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "roofline": roofline, "cpu_baseline": cpu,
                "per_step_ms": per_step_ms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ other workloads
def run_batched(args):
    """Config 4: 64 runs (L, R, theta drawn from Philox tag 3, seed 99), fixed
    dbeta = 0.005 over beta 0->1, seeds 100..163; all runs in one batched
    graph launch vs the same runs one at a time (each a graph-captured run)."""
    import torch

    import paper_1703_03676_gb300 as eng
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.batch_set == "config1":
        # 64 small runs of the config-1 shape (L = 16, R = 1000, theta = 10, 100 steps), bit-packed:
        # each alone is latency-bound, so this is where batching pays
        n_steps, bf = 100, 1.0
        cfgs = [eng.PAConfig(L=16, R=1000, theta=10, beta_f=1.0, dbeta=0.01, seed=100 + i) for i in range(64)]
        desc = "64 runs of the config-1 shape (L=16, R=1000, theta=10, dbeta 0.01, 100 steps)"
    else:
        draw = eng.batch_config4_draw(64)
        n_steps = args.c4_steps
        bf = n_steps * 0.005
        cfgs = [eng.PAConfig(L=L, R=R, theta=th, beta_f=bf, dbeta=0.005, seed=100 + i)
                for i, (L, R, th) in enumerate(draw)]
        desc = f"64 runs, L/R/theta from Philox tag 3 seed 99, dbeta 0.005, {n_steps} steps (beta 0->{bf:g})"
    att_of = lambda rows, c: c.L * c.L * c.theta * int(rows["R"][1:].sum())  # noqa: E731
    b = eng.PABatch(cfgs, stream=stream)
    times = []
    att_b = 0
    for k in range(args.warmup + args.steps):
        b.reset([100 + i + 1000 * k for i in range(64)])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.launch()
        e1.record(stream)
        b.sync()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
            att_b += sum(att_of(r.rows(), c) for r, c in zip(b.runs, cfgs))
    v_batched = att_b / (sum(times) * 1e6)
    shapes = {c.L: b.shape(i)["group_threads"] for i, c in enumerate(cfgs)}
    b.close()
    runs = [eng.PARun(c, stream=stream) for c in cfgs]
    t_alone, att_a = 0.0, 0
    for k in range(max(1, args.warmup // 3) + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i, r in enumerate(runs):
            r.reset(100 + i + 1000 * k)
        e0.record(stream)
        for r in runs:
            r.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= max(1, args.warmup // 3):
            t_alone += e0.elapsed_time(e1)
            att_a += sum(att_of(r.rows(), c) for r, c in zip(runs, cfgs))
    for r in runs:
        r.close()
    v_alone = att_a / (t_alone * 1e6)
    line = {"metric": METRIC, "workload": "batched", "value": v_batched, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(times) / len(times),
            "higher_is_better": True, "single_run_value": v_alone, "batched_over_single": v_batched / v_alone,
            "config": {"workload": f"{desc}, seeds 100..163 (+1000 per bench step), bit-packed",
                       "attempts_per_step": att_b / len(times), "group_threads_by_L": shapes},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    """Config 5, scaled: the first n requests of the served trace (Poisson
    arrivals at 20/s, L in {32..512}, seeds 1000+q, all drawn from Philox tag
    4 seed 999), theta = 50, adaptive steps with overlap 0.85, with R divided
    by r_div and beta_f lowered to beta_f_serve. Continuous batching
    (max_active, HBM budget) vs one run at a time; p50/p99 latency."""
    import torch

    import paper_1703_03676_gb300 as eng
    torch.cuda.set_device(0)
    trace = eng.served_trace(args.serve_n)
    reqs = [(t, eng.PAConfig(L=L, R=max(100, R // args.serve_rdiv), theta=50, beta_f=args.serve_beta_f, dbeta=0.0,
                             overlap=0.85, seed=seed)) for (t, L, R, seed) in trace]
    free, total = torch.cuda.mem_get_info()
    budget = int(min(args.serve_budget_gb * 2 ** 30, 0.8 * free))
    out = {}
    for name, max_active in (("served", args.serve_active), ("one_at_a_time", 1)):
        t0 = time.perf_counter()
        res, _ = eng.serve(reqs, hbm_budget=budget, max_active=max_active)
        wall = time.perf_counter() - t0
        lat = sorted(r["finish_s"] - t for r, (t, _) in zip(res, reqs))
        att = sum(r["attempts"] for r in res)
        ok = all(r["status"] == 0 for r in res)
        out[name] = {"flips_per_ns": att / (wall * 1e9), "makespan_s": wall, "p50_latency_s": lat[len(lat) // 2],
                     "p99_latency_s": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                     "all_ok": ok, "attempts": att}
    line = {"metric": METRIC, "workload": "served", "value": out["served"]["flips_per_ns"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True,
            "p50_latency_s": out["served"]["p50_latency_s"], "p99_latency_s": out["served"]["p99_latency_s"],
            "one_at_a_time": out["one_at_a_time"],
            "served_over_one_at_a_time": out["served"]["flips_per_ns"] / out["one_at_a_time"]["flips_per_ns"],
            "served": out["served"],
            "config": {"workload": f"first {args.serve_n} requests of the 500-request trace (Poisson 20/s, L in "
                                   f"32..512, seeds 1000+q); deviation: R/{args.serve_rdiv}, beta_f "
                                   f"{args.serve_beta_f} instead of 1 (the full trace is ~1e17 attempts)",
                       "max_active": args.serve_active, "hbm_budget_bytes": budget, "theta": 50, "overlap": 0.85},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--workload", choices=["default", "batched", "served"], default="default")
    ap.add_argument("--format", choices=["bits", "msc", "int8", "replica"], default="bits",
                    help="spin format of the default workload: bits (Philox per attempt, the reference contract), "
                         "msc (the paper's multi-spin coding with a Philox-seeded LCG), int8")
    ap.add_argument("--L", type=int, default=None, help="override the default workload's lattice edge")
    ap.add_argument("--R", type=int, default=None, help="override the default workload's population")
    ap.add_argument("--theta", type=int, default=None, help="override the default workload's sweeps per step")
    ap.add_argument("--dbeta", type=float, default=None, help="override the default workload's step size")
    ap.add_argument("--dim", type=int, choices=[2, 3], default=None,
                    help="3: the simple cubic L x L x L lattice instead of the square one")
    ap.add_argument("--potts-q", type=int, default=None,
                    help="2..8: the q-state Potts model (byte states, --format int8)")
    ap.add_argument("--group-threads", type=int, default=None,
                    help="threads per replica of the bit-packed sweep (default: chosen by the engine)")
    ap.add_argument("--c4-steps", type=int, default=200)
    ap.add_argument("--batch-set", choices=["config4", "config1"], default="config4",
                    help="runs of --workload batched: the config-4 draw, or 64 runs of the config-1 shape")
    ap.add_argument("--serve-n", type=int, default=48)
    ap.add_argument("--serve-rdiv", type=int, default=50)
    ap.add_argument("--serve-beta-f", type=float, default=0.5)
    ap.add_argument("--serve-active", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=100.0)
    ap.add_argument("--no-profile", dest="profile", action="store_false")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-replicas", type=int, default=2000)
    ap.add_argument("--ref-replicas", type=int, default=400)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.potts_q and args.format != "int8":
        ap.error("--potts-q needs --format int8")
    for k in ("L", "R", "theta", "dbeta", "dim", "potts_q"):  # labelled variants of the default workload
        if getattr(args, k) is not None:
            WL[k] = getattr(args, k)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
