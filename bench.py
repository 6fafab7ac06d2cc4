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
          pa_launch, i.e. init, 200 temperature steps as one CUDA graph
          (no profiling events inside the graph);
  e2e     wall clock of the public API a user calls: pa_create (allocation,
          host tables uploaded), pa_run, pa_observables (rows read back),
          pa_destroy;
  roofline  the sweep kernel's average launch time from CUDA events captured
          in the graph of a separate profiled pass of the same workload,
          against the wide-multiply issue peak of the device;
  batched / served  the batched and served forms of the same engine on
          labelled prefixes of the batched and served workloads, each beside
          the same runs one at a time (single GPU only);
  cpu_baseline  the CPU oracle on a bounded sample of the same workload (whole
          anneals of a few replicas) on all host cores (independent
          processes).

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
    return (f"plain PA, {lattice}, R={WL['R']}, theta={WL['theta']}, beta 0->{WL['beta_f']:g} {steps}, "
            f"bit-packed spins")


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
MUL_OPS_PER_ATTEMPT = 4.0       # issued by the kernel (lane-varying products)
MUL_OPS_ALGORITHMIC = 5.0       # a quarter of Philox4x32-10's 20 wide products
ALU_OPS_PER_ATTEMPT = 4.5 + 1.0 + 0.5
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_sweep_bits_L64_R20000_theta100.md")
GATHER_SUMMARY = os.path.join(ROOT, "profiles", "k_gather_L128_R50000.md")


def kernel_source_hash() -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_1703_03676_gb300", "csrc", "pa_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(summary=PROFILE_SUMMARY):
    """DRAM bytes per launch from a committed ncu summary (the sweep's by
    default), if it was taken on the current kernel source (else None)."""
    try:
        text = open(summary).read()
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
    """One worker: the oracle on R_s replicas of the workload `wl`, for
    n_steps temperature steps (None: the whole anneal to beta_f); returns
    (attempts, seconds, restarts). A population this small can die out (all
    copy numbers 0 when R_{i-1} > R); the sample then starts a new anneal
    from beta0 with the next seed, counting the steps already done, until
    n_steps steps (or one whole anneal) are complete; `restarts` counts
    these. (Workers are spawned, so the workload comes in the arguments, not
    from this module's globals.)"""
    R_s, n_steps, seed, wl = args
    sys.path.insert(0, ROOT)
    from oracle.pa_oracle import OracleError, PopulationAnnealing
    t0 = time.perf_counter()
    att = 0
    k = 0
    restarts = 0
    while True:
        pa = PopulationAnnealing(wl["L"], R_s, wl["theta"], beta_f=wl["beta_f"], dbeta=wl["dbeta"],
                                 seed=seed + 1000003 * restarts, dim=wl["dim"], potts_q=wl["potts_q"])
        try:
            while not pa.done and (n_steps is None or k < n_steps):
                rec = pa.step()
                att += wl["L"] ** wl["dim"] * wl["theta"] * rec.R
                k += 1
        except OracleError as e:
            if e.kind != "extinct" or restarts >= 100:
                raise
            restarts += 1
            continue
        return att, time.perf_counter() - t0, restarts


def cpu_oracle(workers: int, R_s: int, n_steps, seed0: int):
    ctx = mp.get_context("spawn")
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_sample, [(R_s, n_steps, seed0 + w, dict(WL)) for w in range(workers)])
    wall = time.perf_counter() - t0
    att = sum(r[0] for r in res)
    restarts = sum(r[2] for r in res)
    return att / wall / 1e9, att, wall, restarts


def restart_note(restarts: int) -> str:
    return (f"; {restarts} population(s) died out and restarted from beta0 with the next seed, their steps "
            f"counted" if restarts else "")


def anneal_label():
    return "the whole anneal (every temperature step to beta_f)" if WL["dbeta"] > 0 else \
        "the whole adaptive anneal to beta_f"


def cpu_baseline_obj(workers, R_s):
    v, att, wall, restarts = cpu_oracle(workers, R_s, None, 9000)
    return {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} independent oracle processes, each {anneal_label()} of the workload with "
                      f"R={R_s} (not R={WL['R']}): {att:.3e} attempts in {wall:.1f} s wall"
                      f"{restart_note(restarts)}"}


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
        cpu_oracle(workers, 1, 10, 500)  # untimed: spawn, build and page in
    tot_att, tot_wall, tot_restarts = 0, 0.0, 0
    for k in range(args.steps):
        _, att, wall, restarts = cpu_oracle(workers, R_s, None, 1000 + 100 * k)
        tot_att += att
        tot_wall += wall
        tot_restarts += restarts
    v = tot_att / tot_wall / 1e9
    sample = (f"each step: {workers} independent oracle processes, each {anneal_label()} of the workload "
              f"with R={R_s} (not R={WL['R']}){restart_note(tot_restarts)}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": {"workload": workload_label(), "sample_replicas": R_s},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ engine arm
def sweep_roofline(eng, cfg, stream, dev, runs, clocks, seed0):
    """The sweep kernel against its binding pipe, from a separate profiled
    pass (runs complete runs with CUDA events around every launch, recorded
    on the engine's stream inside the graph)."""
    import dataclasses

    import torch
    pcfg = dataclasses.replace(cfg, profile=True)
    run = eng.PARun(pcfg, stream=stream)
    run.reset(seed0)
    run.launch()
    run.sync()
    base = run.phase_times()
    attempts, dev_ms = 0, 0.0
    for k in range(runs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.reset(seed0 + 1 + k)
        run.launch()
        e1.record(stream)
        run.sync()
        dev_ms += e0.elapsed_time(e1)
        attempts += sites() * WL["theta"] * int(run.rows()["R"][1:].sum())
    pt = run.phase_times()
    shape = run.launch_shape()
    run.close()
    sw_ms = pt["sweep"][0] - base["sweep"][0]
    sw_n = pt["sweep"][1] - base["sweep"][1]
    avg_ms = sw_ms / max(sw_n, 1)
    att_per_launch = attempts / max(sw_n, 1)
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_max = clocks.get("sm_max_mhz") or 2070.0
    apn = att_per_launch / (avg_ms * 1e6)  # attempts per ns in the sweep kernel
    mul_peak = sm * 32 * clk_max * 1e6 / 1e9  # Gop/s, wide multiplies (FMA-heavy pipe)
    alu_peak = sm * 64 * clk_max * 1e6 / 1e9  # Gop/s, ALU pipe
    achieved = MUL_OPS_ALGORITHMIC * apn
    gt = shape["group_threads"]
    roof = {"bound": "fma_heavy", "achieved": achieved, "peak": mul_peak, "unit": "Gop/s",
            "frac": achieved / mul_peak,
            "traffic": profiled_traffic() if WL == DEFAULT_WL else None,
            "kernel": f"k_sweep_bits<{WL['L']},{gt}" + (",3>" if WL["dim"] == 3 else ">"), "launch": shape,
            "ops": "wide 32x32->64 multiplies of Philox4x32-10, 5 per attempt (a quarter of a block's 20)",
            "peak_note": "FMA-heavy (integer wide-multiply) pipe: SMs x 32 lanes/clk x max SM clock (derived, "
                         "of measured max clock)",
            "issued": {"ops_per_attempt": MUL_OPS_PER_ATTEMPT, "achieved": MUL_OPS_PER_ATTEMPT * apn,
                       "frac": MUL_OPS_PER_ATTEMPT * apn / mul_peak,
                       "note": "the kernel issues 4 lane-varying products per attempt: the two first-round "
                               "products are warp-uniform under its counter layout"},
            "alu_pipe": {"achieved": ALU_OPS_PER_ATTEMPT * apn, "peak": alu_peak,
                         "frac": ALU_OPS_PER_ATTEMPT * apn / alu_peak,
                         "ops": "4.5 Philox XOR + 1 compare + 0.5 logic per attempt"},
            "attempts_per_ns": apn, "launch_ms": avg_ms, "launches": sw_n,
            "share_of_step": sw_ms / dev_ms if dev_ms else None,
            "timing": f"separate profiled pass: {runs} complete runs, CUDA events around every launch",
            "algorithmic_bytes_per_launch": 2 * att_per_launch / (sites() * WL["theta"]) * (sites() / 8)}
    try:
        roof["rng_ceiling_words_per_ns"] = eng.measure_rng_peak(2048, stream)
    except Exception as e:  # measurement only
        roof["rng_ceiling_words_per_ns"] = f"unavailable: {e}"
    try:
        # measured issue rates of the instruction classes behind the derived peaks
        mp_ = {"wide_mul": eng.measure_pipe_peak(eng.PIPE_WIDE_MUL, 16384, stream),
               "lop3": eng.measure_pipe_peak(eng.PIPE_LOP3, 16384, stream),
               "imad": eng.measure_pipe_peak(eng.PIPE_IMAD, 16384, stream)}
        roof["measured_pipe_peaks_gops"] = mp_
        roof["frac_of_measured_wide_mul"] = achieved / mp_["wide_mul"]
        roof["alu_pipe"]["frac_of_measured_lop3"] = ALU_OPS_PER_ATTEMPT * apn / mp_["lop3"]
    except Exception as e:  # measurement only
        roof["measured_pipe_peaks_gops"] = f"unavailable: {e}"
    return roof


def measured_peaks():
    """(HBM GB/s, label) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def gather_roofline(eng, stream, reps=20, warm=3):
    """The resampling copy alone (pa_gather) on the sizes of the adaptive
    L = 128, R = 50000 workload, where the two populations (2 x 102 MB)
    exceed L2: algorithmic bytes = read + write of every new replica
    (2 x R_i x L^2/8) + its parent index (4 B), over the kernel's device
    time, against the measured HBM copy bandwidth."""
    import numpy as np
    import torch
    L, R = 128, 50000
    words = L * L // 32
    rng = np.random.default_rng(12345)
    r = rng.choice(4, size=R, p=[0.3, 0.45, 0.2, 0.05])  # copy numbers of a resampling step, mean 1
    parent = torch.from_numpy(np.repeat(np.arange(R), r).astype(np.int32)).cuda()
    n_new = parent.numel()
    src = torch.randint(-2 ** 31, 2 ** 31 - 1, (R * words,), dtype=torch.int32, device="cuda")
    dst = torch.empty(n_new * words, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    ts = []
    for k in range(warm + reps):
        flush.fill_(k)
        torch.cuda.synchronize()
        _, ms = eng.gather(src, parent, words, dst=dst, stream=stream)
        if k >= warm:
            ts.append(ms)
    ms = sorted(ts)[len(ts) // 2]
    byts = 2.0 * n_new * words * 4 + 4.0 * n_new
    peak, lab = measured_peaks()
    gbs = byts / (ms * 1e6)
    return {"bound": "hbm", "kernel": "k_gather<32> (pa_gather)", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "peak_note": lab + " (MEASURED_PEAKS.json hbm_gbs)" if lab == "of measured"
            else lab, "algorithmic_bytes_per_launch": byts, "launch_ms": ms, "reps": reps,
            "traffic": profiled_traffic(GATHER_SUMMARY),
            "workload": f"resampling copy of L={L} bit-packed replicas ({words * 4} B each), R_(i-1)={R}, "
                        f"R_i={n_new}, sorted parents with copy numbers 0..3; L2 flushed before each launch"}


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
                       spin_format=fmt, use_graph=True, profile=False, dim=WL["dim"], potts_q=WL["potts_q"],
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
        n0 = run.kernel_launches()
        e0.record(stream)
        one(seed_of(k))
        e1.record(stream)
        run.sync()
        ms = e0.elapsed_time(e1)
        rows = run.rows()
        assert adaptive or len(rows) == n_steps + 1
        attempts += sites() * theta * int(rows["R"][1:].sum())
        launches += run.kernel_launches() - n0
        dev_ms += ms
        per_step_ms.append(ms)
    torch.cuda.synchronize(dev)
    barrier(dist)
    clocks = clocks_sampler_stop(clk, clk_path, local)
    t_max = max_over_ranks(dev_ms, dist)
    att_all = sum_over_ranks(attempts, dist)
    value = att_all / (t_max * 1e6)

    roofline = None
    gather = None
    if args.profile and args.format == "bits":
        roofline = sweep_roofline(eng, cfg, stream, dev, args.prof_runs, clocks, seed_of(20_000))
        if WL == DEFAULT_WL and ws == 1:
            gather = gather_roofline(eng, stream)

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
    run.close()
    del flush

    batched = served = None
    if ws == 1 and not args.no_extras and WL == DEFAULT_WL and args.format == "bits":
        clk2 = clocks_sampler_start(clk_path)
        batched = {"config4_prefix": measure_batched(eng, stream, "config4", args.extras_c4_steps, 2, 1),
                   "config1_set": measure_batched(eng, stream, "config1", 100, 5, 3)}
        served = measure_served(eng, args.extras_serve_n, args.extras_serve_rdiv, args.extras_serve_beta_f,
                                args.serve_active, args.serve_budget_gb)
        c2 = clocks_sampler_stop(clk2, clk_path, local)
        batched["clocks"] = c2
        served["clocks"] = c2

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_obj(os.cpu_count() or 1, args.cpu_replicas)

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
                "roofline": roofline, "gather": gather, "batched": batched, "served": served, "cpu_baseline": cpu,
                "per_step_ms": per_step_ms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ batched and served forms
def batch_configs(eng, which: str, n_steps: int):
    """(configs, label) of a batched workload: the config-4 draw (64 runs;
    L, R, theta from Philox tag 3 seed 99; dbeta 0.005) over its first
    n_steps steps, or 64 runs of the config-1 shape."""
    if which == "config1":
        cfgs = [eng.PAConfig(L=16, R=1000, theta=10, beta_f=1.0, dbeta=0.01, seed=100 + i) for i in range(64)]
        return cfgs, "64 runs of the config-1 shape (L=16, R=1000, theta=10, dbeta 0.01, 100 steps), bit-packed"
    draw = eng.batch_config4_draw(64)
    bf = n_steps * 0.005
    cfgs = [eng.PAConfig(L=L, R=R, theta=th, beta_f=bf, dbeta=0.005, seed=100 + i)
            for i, (L, R, th) in enumerate(draw)]
    label = (f"64 runs, L/R/theta from Philox tag 3 seed 99, dbeta 0.005, bit-packed; "
             + ("all 200 steps" if n_steps == 200 else
                f"deviation: the first {n_steps} of 200 steps (beta 0->{bf:g})"))
    return cfgs, label


def measure_batched(eng, stream, which: str, n_steps: int, reps: int, warm: int):
    """All runs in one batched graph launch vs the same runs one at a time
    (each its own graph-captured run, launched back to back), device time
    with CUDA events on the shared stream."""
    import torch
    cfgs, label = batch_configs(eng, which, n_steps)
    att_of = lambda rows, c: c.L * c.L * c.theta * int(rows["R"][1:].sum())  # noqa: E731
    b = eng.PABatch(cfgs, stream=stream)
    times, att_b = [], 0
    for k in range(warm + reps):
        b.reset([100 + i + 1000 * k for i in range(len(cfgs))])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.launch()
        e1.record(stream)
        b.sync()
        if k >= warm:
            times.append(e0.elapsed_time(e1))
            att_b += sum(att_of(r.rows(), c) for r, c in zip(b.runs, cfgs))
    v_batched = att_b / (sum(times) * 1e6)
    shapes = {c.L: b.shape(i)["group_threads"] for i, c in enumerate(cfgs)}
    b.close()
    runs = [eng.PARun(c, stream=stream) for c in cfgs]
    t_alone, att_a = 0.0, 0
    for k in range(warm + reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i, r in enumerate(runs):
            r.reset(100 + i + 1000 * k)
        e0.record(stream)
        for r in runs:
            r.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= warm:
            t_alone += e0.elapsed_time(e1)
            att_a += sum(att_of(r.rows(), c) for r, c in zip(runs, cfgs))
    for r in runs:
        r.close()
    v_alone = att_a / (t_alone * 1e6)
    return {"value": v_batched, "unit": UNIT, "single_run_value": v_alone,
            "batched_over_single": v_batched / v_alone, "ms_per_batch": sum(times) / len(times),
            "reps": reps, "warmup": warm, "workload": f"{label}; seeds 100..163 (+1000 per repetition)",
            "attempts_per_batch": att_b / len(times), "group_threads_by_L": shapes}


def measure_served(eng, n: int, rdiv: int, beta_f: float, active: int, budget_gb: float):
    """Continuous batching (pa_serve, up to `active` resident runs within an
    HBM budget) vs the same requests one at a time, on the first n requests
    of the served trace with R divided by rdiv and beta_f lowered."""
    import torch
    trace = eng.served_trace(n)
    reqs = [(t, eng.PAConfig(L=L, R=max(100, R // rdiv), theta=50, beta_f=beta_f, dbeta=0.0,
                             overlap=0.85, seed=seed)) for (t, L, R, seed) in trace]
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(budget_gb * 2 ** 30, 0.8 * free))
    out = {}
    for name, max_active in (("served", active), ("one_at_a_time", 1)):
        t0 = time.perf_counter()
        res, _ = eng.serve(reqs, hbm_budget=budget, max_active=max_active)
        wall = time.perf_counter() - t0
        lat = sorted(r["finish_s"] - t for r, (t, _) in zip(res, reqs))
        att = sum(r["attempts"] for r in res)
        out[name] = {"flips_per_ns": att / (wall * 1e9), "makespan_s": wall, "p50_latency_s": lat[len(lat) // 2],
                     "p99_latency_s": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                     "all_ok": all(r["status"] == 0 for r in res), "attempts": att}
    return {"value": out["served"]["flips_per_ns"], "unit": UNIT,
            "p50_latency_s": out["served"]["p50_latency_s"], "p99_latency_s": out["served"]["p99_latency_s"],
            "served_over_one_at_a_time": out["served"]["flips_per_ns"] / out["one_at_a_time"]["flips_per_ns"],
            "served": out["served"], "one_at_a_time": out["one_at_a_time"],
            "workload": f"deviation: the first {n} requests of the 500-request served trace (Poisson 20/s, L in "
                        f"32..512, theta 50, adaptive overlap 0.85, seeds 1000+q) with R/{rdiv} and beta_f "
                        f"{beta_f:g} instead of 1 (the full trace is ~1e17 attempts)",
            "max_active": active, "hbm_budget_bytes": budget}


def run_gather(args):
    """The resampling copy alone (--workload gather, see gather_roofline)."""
    import torch

    import paper_1703_03676_gb300 as eng
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g = gather_roofline(eng, stream, reps=args.steps, warm=args.warmup)
    line = {"metric": "resampling copy bandwidth", "workload": "gather", "value": g["achieved"], "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["launch_ms"],
            "higher_is_better": True, "roofline": g, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """The batched workload alone (--workload batched): the config-4 draw or
    the 64 config-1-shaped runs."""
    import torch

    import paper_1703_03676_gb300 as eng
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_steps = 100 if args.batch_set == "config1" else args.c4_steps
    r = measure_batched(eng, stream, args.batch_set, n_steps, args.steps, args.warmup)
    line = {"metric": METRIC, "workload": "batched", "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True,
            "single_run_value": r["single_run_value"], "batched_over_single": r["batched_over_single"],
            "config": {"workload": r["workload"], "attempts_per_step": r["attempts_per_batch"],
                       "group_threads_by_L": r["group_threads_by_L"]},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    """The served workload alone (--workload served), scaled (see
    measure_served)."""
    import torch

    import paper_1703_03676_gb300 as eng
    torch.cuda.set_device(0)
    r = measure_served(eng, args.serve_n, args.serve_rdiv, args.serve_beta_f, args.serve_active,
                       args.serve_budget_gb)
    line = {"metric": METRIC, "workload": "served", "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"],
            "one_at_a_time": r["one_at_a_time"], "served_over_one_at_a_time": r["served_over_one_at_a_time"],
            "served": r["served"],
            "config": {"workload": r["workload"], "max_active": r["max_active"],
                       "hbm_budget_bytes": r["hbm_budget_bytes"], "theta": 50, "overlap": 0.85},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--workload", choices=["default", "batched", "served", "gather"], default="default")
    ap.add_argument("--format", choices=["bits", "msc", "int8", "replica"], default="bits",
                    help="spin format of the default workload: bits (Philox per attempt, the reference contract), "
                         "msc (the paper's multi-spin coding with a Philox-seeded LCG), int8")
    ap.add_argument("--L", type=int, default=None, help="override the default workload's lattice edge")
    ap.add_argument("--R", type=int, default=None, help="override the default workload's population")
    ap.add_argument("--theta", type=int, default=None, help="override the default workload's sweeps per step")
    ap.add_argument("--dbeta", type=float, default=None, help="override the default workload's step size")
    ap.add_argument("--beta-f", type=float, default=None,
                    help="override the default workload's final inverse temperature (a labelled prefix)")
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
    ap.add_argument("--no-profile", dest="profile", action="store_false",
                    help="skip the separate profiled pass behind the roofline")
    ap.add_argument("--prof-runs", type=int, default=2, help="complete runs of the profiled pass")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served sub-objects of the default line")
    ap.add_argument("--extras-c4-steps", type=int, default=20,
                    help="steps of the config-4 prefix in the default line's batched object")
    ap.add_argument("--extras-serve-n", type=int, default=16)
    ap.add_argument("--extras-serve-rdiv", type=int, default=100)
    ap.add_argument("--extras-serve-beta-f", type=float, default=0.3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-replicas", type=int, default=8,
                    help="replicas per process of the cpu_baseline sample (whole anneals)")
    ap.add_argument("--ref-replicas", type=int, default=4,
                    help="replicas per process of each --impl reference step (whole anneals)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.potts_q and args.format != "int8":
        ap.error("--potts-q needs --format int8")
    for k in ("L", "R", "theta", "dbeta", "beta_f", "dim", "potts_q"):  # labelled variants of the default workload
        if getattr(args, k) is not None:
            WL[k] = getattr(args, k)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "gather":
        return run_gather(args)
    return run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
