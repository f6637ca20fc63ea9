"""Throughput of the dynamic-chromatic MH sweep on one GB300.

One step = one sweep: the partition is shifted, every region of each colour
runs k MH steps, colours in order.  The default workload is the float32 sweep
at scale (4000 x 4000 km, 24 h, ~10^4 events, 1600 stations x 864000 samples,
40 x 40 regions of 100 km, k = 32).

Printed (one JSON line): MH proposals/s over the timed sweeps (value), sweeps/s,
an end-to-end figure through the C ABI with host buffers (model creation from
pinned host signals, the sweeps, and a read-back of the state after every
sweep), the roofline of the colour-phase kernel measured live with CUDA
events, and the oracle timed on the host cores.

--impl reference times the CPU oracle (the only other implementation) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import worldgen  # noqa: E402

K_PER_PHASE = 32
MAG_HALF_WIDTH = 0.3
SEED = 1000
CHAIN_SEED = 7


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = ["paper_1612_00595_gb300/csrc/cmh_phase32.cu", "paper_1612_00595_gb300/csrc/cmh_common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep32_scale_dram.json")


def _kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic():
    """DRAM bytes per launch of the colour-phase kernel from the committed ncu
    capture, or None when the kernel sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, "no ncu capture committed"
    if rec.get("kernel_sha256") != _kernel_digest():
        return None, "kernel changed since the ncu capture"
    return float(rec["dram_bytes_per_launch"]), rec.get("command", "")


FP32_ERROR_FILE = os.path.join(ROOT, "profiles", "fp32_error_scale_density.json")


def _fp32_error():
    """The float32 sweep's error against the float64 oracle, from the
    committed record of the parity test at the bench workload's density
    (>= 1e5 proposals), or None when the kernel changed since."""
    try:
        with open(FP32_ERROR_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return {"value": None, "reason": "no record committed"}
    if rec.get("kernel_sha256") != _kernel_digest():
        return {"value": None, "reason": "kernel changed since the record"}
    return rec


def n_proposals(st) -> int:
    """Every MH proposal a model made: birth, death, move, joint pair and
    arrival-time moves."""
    return int(sum(st["proposed"]) + st["pair"][0] + st["arrival"][0])


def n_evaluated(st) -> int:
    """The proposals that were priced: those not rejected outright (a
    candidate outside its region, the domain, [0, T) or m >= 2)."""
    return int(sum(st["evaluated"]) + st["pair"][1] + st["arrival"][1])


# algorithmic work per priced sample of the float32 variance pricing: the
# logarithm and the reciprocal of each sample's term on the special-function
# unit, and ~12 float32 FMA (24 flops) for the envelope, the change, the
# ratio, the series and the compensated sum
MUFU_PER_SAMPLE = 2.0
FLOPS_PER_SAMPLE = 24.0


def _workload(name: str, likelihood: str = "variance", p_pair: float = 0.0, sig_a: float = 0.0,
              p_arr: float = 0.0):
    if name == "scale":
        return worldgen.config_scale(seed=SEED, likelihood=likelihood, sig_a=sig_a), \
            "fp32 sweep at scale: 4000x4000 km, 24 h, ~1e4 events, 1600 stations x 864000 f32 samples, " \
            "40x40 regions, k=32" + ("" if likelihood == "variance" else ", additive-mean likelihood reading") + \
            (", joint pair moves p_pair=%g" % p_pair if p_pair else "") + (
                ", latent arrival times sig_a=%g s (offsets of the generated world), arrival-time moves "
                "p_arr=%g" % (sig_a, p_arr) if sig_a else "")
    if name == "replay":
        return worldgen.config_replay(seed=SEED, sig_a=sig_a), \
            "fp64 replay: 1000x1000 km, 1 h, ~500 events, 100 stations x 36000 f64 samples, 10x10 regions, " \
            "k=32" + (", joint pair moves p_pair=%g" % p_pair if p_pair else "") + (
                ", latent arrival times sig_a=%g s (offsets of the generated world), arrival-time moves "
                "p_arr=%g" % (sig_a, p_arr) if sig_a else "")
    raise SystemExit("unknown workload " + name)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int = 0):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_baseline(world, seconds_target: float = 15.0, p_pair: float = 0.0, sig_a: float = 0.0,
                  p_arr: float = 0.0, sig_da: float = 1.0):
    """The oracle's chromatic sampler on a 1000 x 1000 km corner of the world
    (same station density, event intensity and record length)."""
    import oracle
    oracle.build()
    sub_side = 1000.0
    sub = worldgen.subworld(world, 0.0, sub_side, 0.0, sub_side)
    frac = (sub_side / world.params.W) ** 2
    p = worldgen.ModelParams(**{**world.params.__dict__, "W": sub_side, "Lambda": world.params.Lambda * frac})
    sub.params = p
    threads = os.cpu_count() or 1
    o = oracle.World(sub, k_per_phase=K_PER_PHASE, seed=CHAIN_SEED, p_pair=p_pair, sig_a=sig_a, p_arr=p_arr,
                     sig_da=sig_da)
    ev = sub.events
    ids = None
    off = sub.offsets if sig_a else None
    t0 = time.perf_counter()
    props, sweeps = 0, 0
    while True:
        ev, ids, tr, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=sweeps, trace_cap=200000, threads=threads, off=off)
        off = o.last_offsets if sig_a else None
        props += len(tr)
        sweeps += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    # the serial sampler (Algorithm "Serial Metropolis Hastings") on one core,
    # same corner and start, for a third of the time (at most 5 s)
    o1 = oracle.World(sub, k_per_phase=K_PER_PHASE, seed=CHAIN_SEED, p_pair=p_pair, sig_a=sig_a, p_arr=p_arr,
                      sig_da=sig_da)
    ev1, ids1, off1 = sub.events, None, (sub.offsets if sig_a else None)
    t1 = time.perf_counter()
    steps1 = 0
    while True:
        ev1, ids1, _, _ = o1.run_serial(ev1, 1000, ids=ids1, step0=steps1, off=off1)
        off1 = o1.last_offsets if sig_a else None
        steps1 += 1000
        if time.perf_counter() - t1 > min(seconds_target / 3.0, 5.0):
            break
    dt1 = time.perf_counter() - t1
    return {"value": props / dt, "unit": "proposals/s", "cores": threads, "kind": "oracle",
            "sample": "%d sweeps of the oracle's chromatic sampler (OpenMP over same-colour regions) on a "
                      "1000x1000 km corner of the same world (100 stations x %d samples, ~%d events), "
                      "started from the ground truth" % (sweeps, world.params.n_samples, len(sub.events)),
            "sweeps": sweeps, "proposals": props, "seconds": dt,
            "serial": {"value": steps1 / dt1, "unit": "proposals/s", "cores": 1, "steps": steps1, "seconds": dt1,
                       "sample": "the oracle's serial sampler on the same corner and start, one core"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    world, desc = _workload(args.workload, args.likelihood, args.p_pair, args.sig_a, args.p_arr)
    base = _cpu_baseline(world, seconds_target=max(5.0, 3.0 * args.steps / 10.0), p_pair=args.p_pair,
                         sig_a=args.sig_a, p_arr=args.p_arr, sig_da=args.sig_da)
    line = {"impl": "reference", "metric": "MH proposals/sec and sweeps/sec on 1 GB300",
            "value": base["value"], "unit": "proposals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded worldgen)",
            "config": {"workload": desc + " [oracle on a 1000x1000 km corner]"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "proposals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def chain_seed(rank: int) -> int:
    """Seed of rank's chain: every rank runs an independent replica."""
    return CHAIN_SEED + 1000 * rank


def reduce_max_sum(x_max: float, x_sum: float, dist=None, device="cpu"):
    """(max over ranks of x_max, sum over ranks of x_sum): the job's time is
    its slowest rank's, its work the sum of the ranks' work."""
    import torch
    a = torch.tensor([float(x_max)], dtype=torch.float64, device=device)
    b = torch.tensor([float(x_sum)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(a, op=dist.ReduceOp.MAX)
        dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def run_ours(args):
    import torch

    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world_size > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1612_00595_gb300 as cm

    world, desc = _workload(args.workload, args.likelihood, args.p_pair, args.sig_a, args.p_arr)
    p = world.params
    f32 = world.signals.dtype == np.float32
    dtype = cm.F32 if f32 else cm.F64
    esz = 4 if f32 else 8
    # each rank runs an independent chain (weak scaling: fixed work per GPU)
    params = cm.make_params(p, k_per_phase=K_PER_PHASE, seed=chain_seed(rank), dtype=dtype, p_pair=args.p_pair,
                            sig_a=args.sig_a, p_arr=args.p_arr, sig_da=args.sig_da)
    stream = torch.cuda.Stream()
    sig_dev = torch.from_numpy(world.signals).to("cuda", non_blocking=False)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident throughput ----------------
    m = cm.create_model(world.events, world.stations, sig_dev, params, stream=stream)
    if args.sig_a:
        m.set_arrival_offsets(world.offsets)
    m.partition_and_color(p.L, shift_mode=1)
    m.run_sweeps(args.warmup)
    m.sync()
    _, _, _, st0 = m.read_state(cap=0)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        e0.record(stream)
        m.run_sweeps(args.steps)
        e1.record(stream)
        e1.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    _, _, _, st1 = m.read_state(cap=0)
    props = n_proposals(st1) - n_proposals(st0)
    evals = n_evaluated(st1) - n_evaluated(st0)
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    ms_max, total_props = reduce_max_sum(ms, props, dist, "cuda")
    _, total_evals = reduce_max_sum(ms, evals, dist, "cuda")
    value = total_props / (ms_max / 1e3)
    evaluated_per_s = total_evals / (ms_max / 1e3)
    sweeps_per_s = args.steps / (ms_max / 1e3)

    # ---------------- live kernel timing for the roofline ----------------
    m.set_timing(True)
    _, _, _, sa = m.read_state(cap=0)
    m.run_sweeps(args.steps)
    _, _, _, sb = m.read_state(cap=0)
    m.set_timing(False)
    n_launch = sb["phase_launches"] - sa["phase_launches"]
    phase_ms = sb["phase_ms"] - sa["phase_ms"]
    priced = sb["priced_samples"] - sa["priced_samples"]
    rewritten = sb["rewritten_samples"] - sa["rewritten_samples"]
    unique = sb["unique_samples"] - sa["unique_samples"]
    nl = max(n_launch, 1)
    per_launch_s = phase_ms / 1e3 / nl
    peaks, peak_kind = _peaks()
    if f32:
        # algorithmic HBM bytes of a launch: per region and colour phase, the
        # union of the windows its proposals priced at each station, read once
        # (s and V), plus the variance written back on accepted steps
        per_launch_bytes = (unique * 2 * esz + rewritten * esz) / nl
        bytes_rule = "unique window samples per region phase x 2 x 4 B (s, V) + re-synthesised samples x 4 B"
    else:
        # the float64 form does not count unique windows: every priced sample
        per_launch_bytes = (priced * 2 * esz + rewritten * esz) / nl
        bytes_rule = "priced samples x 2 x 8 B (s, V) + re-synthesised samples x 8 B"
    mufu_peak, fma_peak = cm.measure_alu_peaks(stream)
    t_hbm = per_launch_bytes / (peaks["hbm_gbs"] * 1e9)
    t_mufu = MUFU_PER_SAMPLE * priced / nl / mufu_peak
    t_fma = FLOPS_PER_SAMPLE * priced / nl / fma_peak
    terms = {"hbm": {"work_per_launch": per_launch_bytes, "unit": "B", "peak": peaks["hbm_gbs"] * 1e9,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind, "rule": bytes_rule,
                     "t_us": t_hbm * 1e6},
             "mufu": {"work_per_launch": MUFU_PER_SAMPLE * priced / nl, "unit": "ops", "peak": mufu_peak,
                      "peak_source": "cmh_measure_alu_peaks (ex2/lg2/rcp chains, measured in this run)",
                      "rule": "%g per priced sample" % MUFU_PER_SAMPLE, "t_us": t_mufu * 1e6},
             "fma": {"work_per_launch": FLOPS_PER_SAMPLE * priced / nl, "unit": "flop", "peak": fma_peak,
                     "peak_source": "cmh_measure_alu_peaks (FMA chains, measured in this run)",
                     "rule": "%g per priced sample" % FLOPS_PER_SAMPLE, "t_us": t_fma * 1e6}}
    bound = max(terms, key=lambda k: terms[k]["t_us"])
    if bound == "hbm":
        achieved, peak_v, unit = per_launch_bytes / per_launch_s / 1e9, peaks["hbm_gbs"], "GB/s"
    elif bound == "mufu":
        achieved, peak_v, unit = terms["mufu"]["work_per_launch"] / per_launch_s / 1e12, mufu_peak / 1e12, "Tops/s"
    else:
        achieved, peak_v, unit = terms["fma"]["work_per_launch"] / per_launch_s / 1e12, fma_peak / 1e12, "TFLOP/s"
    if not f32:
        traffic, traffic_src = None, "float64 path not captured"
    elif args.likelihood != "variance":
        traffic, traffic_src = None, "the ncu capture is of the variance reading"
    else:
        traffic, traffic_src = _traffic()
    roof = {"bound": "alu" if bound in ("mufu", "fma") else "hbm", "bound_term": bound, "achieved": achieved,
            "peak": peak_v, "unit": unit, "frac": achieved / peak_v if peak_v else 0.0,
            "traffic": traffic, "traffic_source": traffic_src,
            "kernel": "sweep32_kernel<false> (one launch per sweep: all colour phases)" if f32
                      else "phase_kernel (float64 replay, one launch per colour phase)",
            "avg_launch_us": per_launch_s * 1e6, "alg_bytes_per_launch": per_launch_bytes,
            "priced_samples_per_launch": priced / nl, "unique_samples_per_launch": unique / nl,
            "rewritten_samples_per_launch": rewritten / nl, "terms": terms,
            "roofline_us": max(t_hbm, t_mufu, t_fma) * 1e6, "peak_source": peak_kind}
    m.destroy()
    del sig_dev
    torch.cuda.empty_cache()

    # ---------------- end to end through the C ABI, host buffers ----------------
    pinned = torch.from_numpy(world.signals).pin_memory()
    host_sig = pinned.numpy()
    barrier()
    t0 = time.perf_counter()
    m2 = cm.create_model(world.events, world.stations, host_sig, params, stream=stream)
    if args.sig_a:
        m2.set_arrival_offsets(world.offsets)
    m2.partition_and_color(p.L, shift_mode=1)
    torch.cuda.synchronize()
    t_created = time.perf_counter()
    d2h = 0
    # every sweep's state is read: requested right after the sweep into one of
    # two pinned slots, fetched while the next sweep runs
    for i in range(args.steps):
        m2.run_sweeps(1)
        m2.read_state_async(i % 2)
        if i > 0:
            ev, ids, lp, st = m2.read_state_fetch((i - 1) % 2)
            d2h += ev.nbytes + ids.nbytes + 8
    ev, ids, lp, st = m2.read_state_fetch((args.steps - 1) % 2)
    d2h += ev.nbytes + ids.nbytes + 8
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    e2e_s = t_end - t0
    _, _, _, st2 = m2.read_state(cap=0)
    e2e_props = n_proposals(st2)
    m2.destroy()
    e2e_max, e2e_total = reduce_max_sum(e2e_s, e2e_props, dist, "cuda")
    e2e_value = e2e_total / e2e_max
    sweeps_max, _ = reduce_max_sum(t_end - t_created, 0, dist, "cuda")
    create_max, _ = reduce_max_sum(t_created - t0, 0, dist, "cuda")
    h2d_per_step = world.signals.nbytes / args.steps

    if rank == 0:
        cpu = _cpu_baseline(world, p_pair=args.p_pair, sig_a=args.sig_a, p_arr=args.p_arr,
                            sig_da=args.sig_da) if world_size == 1 else None
        line = {"metric": "MH proposals/sec and sweeps/sec on 1 GB300", "value": value, "unit": "proposals/s",
                "sweeps_per_s": sweeps_per_s, "evaluated_per_s": evaluated_per_s,
                "evaluated_note": "proposals priced (not rejected outright for leaving their region, the "
                                  "domain, [0, T) or m >= 2), same timed sweeps", "n_gpus": world_size, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if f32 else "f64",
                "data": "synthetic (seeded worldgen, the model's generative story)",
                "config": {"workload": desc, "l2": "inputs larger than L2 (signals + variance %.1f GB)" % (
                    2 * world.signals.nbytes / 1e9), "chain_start": "ground truth",
                           "parallelism": "independent chain per GPU" if world_size > 1 else "1 GPU"},
                "clocks": clocks.summary(), "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": "proposals/s", "h2d_bytes_per_step": h2d_per_step,
                        "d2h_bytes_per_step": d2h / args.steps,
                        "value_excluding_creation": e2e_total / sweeps_max,
                        "creation_s": create_max,
                        "note": "cmh_create_model from pinned host signals (copied once, amortised over the "
                                "steps) + per step cmh_run_sweeps(1) and the read of that sweep's state "
                                "(cmh_read_state_async into a pinned slot, fetched while the next sweep runs)"},
                "roofline": roof, "cpu_baseline": cpu,
                "fp32_error": _fp32_error() if f32 and args.likelihood == "variance" else None}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def instance_capacities(p, k: int = K_PER_PHASE):
    """Capacities of a batched instance from its density: events per region
    and arrivals per station, mean + 6 sd + slack."""
    per_region = p.Lambda * p.L * p.L / (p.W * p.W)
    per_station = p.Lambda * math.pi * p.R_max ** 2 / (p.W * p.W)
    ev_cap = int(min(512, max(128, per_region + 6 * math.sqrt(per_region) + k + 16)))
    frz_cap = int(max(64, per_station + 6 * math.sqrt(per_station) + 16))
    return ev_cap, frz_cap


def instance_cost(n_stations: int, p) -> float:
    """Estimated work of one sweep of a batched instance: its regions times k
    steps times the samples a step prices (the stations within R_max of an
    event, at the instance's station density, times the window length)."""
    n_cells = (int(p.W // p.L) + 2) ** 2
    st_near = n_stations * math.pi * p.R_max ** 2 / (p.W * p.W)
    return float(n_cells * K_PER_PHASE * (1.0 + st_near * p.n_w))


def shard_instances(costs, world_size: int, rank: int):
    """Rank `rank`'s share of the instances: largest estimated cost first, each
    to the rank with the least cost so far (the lowest rank on a tie).  Every
    rank computes the same split from the same costs, so the shares are
    disjoint, cover every instance and need no communication."""
    load = [0.0] * world_size
    mine = []
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def gather_summaries(summary, dist=None):
    """Every rank's summary dict, in rank order (one all-gather; the only
    collective of the batched workload, after the timed region)."""
    if dist is None:
        return [summary]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, summary)
    return out


def _batched_cpu_baseline(worlds, seconds_target: float = 15.0):
    """The oracle's chromatic sampler on the instances, one after another
    from the ground truth, each on all host cores, for about seconds_target."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    props, sweeps, used = 0, 0, 0
    t0 = time.perf_counter()
    for i, w in enumerate(worlds):
        o = oracle.World(w, k_per_phase=K_PER_PHASE, seed=CHAIN_SEED + i)
        ev, ids = w.events, None
        for s in range(3):
            ncx = int(w.params.W // w.params.L) + 2
            ev, ids, tr, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=s, trace_cap=ncx * ncx * K_PER_PHASE + 16,
                                             threads=threads)
            props += len(tr)
            sweeps += 1
        used += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": props / dt, "unit": "proposals/s", "cores": threads, "kind": "oracle",
            "sample": "3 sweeps of each of the first %d instances of this rank's share, from the ground truth, "
                      "the oracle's chromatic sampler (OpenMP over same-colour regions)" % used,
            "sweeps": sweeps, "proposals": props, "seconds": dt}


def run_batched(args):
    """256 independent instances of uneven size swept together: one
    persistent launch per sweep over every instance's regions.  With N ranks
    the instances are split by estimated cost (shard_instances) and each rank
    sweeps its share as one batch: no data-path collective."""
    import torch
    import paper_1612_00595_gb300 as cm
    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world_size > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sizes = worldgen.batched_instances(256, seed=2000)
    costs = [instance_cost(S, p) for S, p in sizes]
    share = shard_instances(costs, world_size, rank)
    worlds = worldgen.config_batched(256, seed=2000, indices=share)
    models, kept, skipped = [], [], []
    for i, w in zip(share, worlds):
        p = w.params
        ev_cap, frz_cap = instance_capacities(p)
        m = cm.create_model(w.events, w.stations, w.signals,
                            cm.make_params(p, k_per_phase=K_PER_PHASE, seed=CHAIN_SEED + i, dtype=cm.F32,
                                           ev_capacity=ev_cap, frozen_capacity=frz_cap))
        try:
            m.partition_and_color(p.L, shift_mode=1)
        except cm.ChromhError:   # a region's structures exceed shared memory
            skipped.append(i)
            m.destroy()
            continue
        models.append(m)
        kept.append(w)
    stream = torch.cuda.Stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    b = cm.create_batch(models, stream=stream)
    b.run_sweeps(args.warmup)
    b.sync()
    p0 = sum(n_proposals(m.read_state(cap=0)[3]) for m in models)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        e0.record(stream)
        b.run_sweeps(args.steps)
        e1.record(stream)
        e1.synchronize()
    barrier()
    b.sync()
    ms = e0.elapsed_time(e1)
    p1 = sum(n_proposals(m.read_state(cap=0)[3]) for m in models)
    groups = b.groups()
    b.destroy()
    ms_max, total_props = reduce_max_sum(ms, p1 - p0, dist, "cuda")

    # roofline of the batched sweep: a second batch of the same models with
    # the unique-window count on, timed with CUDA events around its sweeps
    # (the persistent batch kernel plus the short re-binning kernels)
    for m in models:
        m.set_timing(True)
    sa = [m.read_state(cap=0)[3] for m in models]
    b2 = cm.create_batch(models, stream=stream)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    b2.run_sweeps(args.steps)
    r1.record(stream)
    r1.synchronize()
    b2.sync()
    roof_ms = r0.elapsed_time(r1)
    sb = [m.read_state(cap=0)[3] for m in models]
    b2.destroy()
    for m in models:
        m.set_timing(False)
    unique = sum(y["unique_samples"] - x["unique_samples"] for x, y in zip(sa, sb))
    priced = sum(y["priced_samples"] - x["priced_samples"] for x, y in zip(sa, sb))
    rewritten = sum(y["rewritten_samples"] - x["rewritten_samples"] for x, y in zip(sa, sb))
    peaks, peak_kind = _peaks()
    per_sweep_s = roof_ms / 1e3 / args.steps
    per_sweep_bytes = (unique * 8 + rewritten * 4) / args.steps
    achieved = per_sweep_bytes / per_sweep_s / 1e9
    summary = {"rank": rank, "instances": len(kept), "skipped": skipped, "ms": ms, "proposals": p1 - p0,
               "groups": groups, "cells": sum((int(w.params.W // w.params.L) + 2) ** 2 for w in kept),
               "signal_bytes": int(sum(w.signals.nbytes for w in kept)), "cost": sum(costs[i] for i in share)}
    summaries = gather_summaries(summary, dist)
    if rank == 0:
        cpu = _batched_cpu_baseline(kept) if world_size == 1 else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "traffic_source": "no ncu capture of the batched workload",
                "kernel": "batched sweep (sweep32_batch persistent kernel + re-binning), rank 0, CUDA events "
                          "around its sweeps",
                "avg_sweep_us": per_sweep_s * 1e6, "alg_bytes_per_sweep": per_sweep_bytes,
                "rule": "unique window samples per region phase x 2 x 4 B (s, V) + re-synthesised samples x 4 B",
                "priced_samples_per_sweep": priced / args.steps, "peak_source": peak_kind}
        line = {"metric": "MH proposals/sec and sweeps/sec on 1 GB300 (batched instances)",
                "value": total_props / (ms_max / 1e3), "unit": "proposals/s",
                "sweeps_per_s": args.steps / (ms_max / 1e3), "n_gpus": world_size, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "strong" if world_size > 1 else "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded worldgen, the model's generative story)",
                "config": {"workload": "256 independent instances: stations logU[16,256], Lambda logU[10,500], side "
                                       "logU[200,2000] km, T logU[600,7200] s, f32, k=32; one sweep of every "
                                       "instance per step",
                           "parallelism": "instances split across %d GPUs by estimated cost, one batch per GPU, no "
                                          "collective in the timed region" % world_size if world_size > 1
                                          else "1 GPU",
                           "ranks": [{k: v for k, v in x.items() if k != "groups"} for x in summaries],
                           "groups (models, CTAs), rank 0": groups},
                "clocks": clocks.summary(), "gpu_launches": (4 + 2 * len(groups)) * args.steps,
                "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line))
    for m in models:
        m.destroy()
    if dist is not None:
        dist.destroy_process_group()


def run_learned(args):
    """Time to F1 >= 0.9 with the learned birth mixture against the plain
    sampler on the 1000 x 1000 km, 1 h, 100-station float32 world.

    The network is trained on 1M simulated windows (4000 steps of 256) and
    slid over the world's signals into a birth table (80 x 80 pixels, 10 s
    bins) with per-entry magnitude centres; table births draw the magnitude
    from a window around the centre (also reported: the same table with
    magnitudes from the prior).  Both samplers start from the empty
    hypothesis.  Chain GPU time is
    taken with CUDA events on the model's stream around each block of 5
    sweeps; the F1 evaluation on the host between blocks is excluded.
    Training and tabulation are timed separately, and the learned figure is
    also given with training amortised over 256 instances."""
    import torch
    import paper_1612_00595_gb300 as cm
    from paper_1612_00595_gb300 import metrics
    torch.cuda.set_device(0)
    w = worldgen.config_learned(seed=SEED)
    P = w.params
    seeds = [CHAIN_SEED + i for i in range(4)]
    every, max_sweeps, thr = 5, 600, 0.9

    def chain(tab, seed, centre=None):
        stream = torch.cuda.Stream()
        m = cm.create_model(None, w.stations, w.signals,
                            cm.make_params(P, k_per_phase=K_PER_PHASE, seed=seed, dtype=cm.F32), stream=stream)
        m.partition_and_color(P.L)
        if tab is not None:
            m.set_birth_table(tab, 0.5)
            if centre is not None:
                m.set_birth_magnitude(centre, MAG_HALF_WIDTH)
        m.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gpu_s, done, hit, curve = 0.0, 0, None, []
        while done < max_sweeps:
            e0.record(stream)
            m.run_sweeps(every)
            e1.record(stream)
            e1.synchronize()
            gpu_s += e0.elapsed_time(e1) / 1e3
            done += every
            sc = metrics.scores(w.events, m.read_state()[0], P.L, P.tau, w.stations, P.R_max)
            curve.append((done, gpu_s, sc["f1"], sc["recall"], sc["loc_err"]))
            if hit is None and sc["f1"] >= thr:
                hit = (done, gpu_s)
        m.destroy()
        return hit, curve

    def summary(runs):
        hits = [h for h, _ in runs]
        ok = [h for h in hits if h is not None]
        last = [c[-1] for _, c in runs]
        at5 = [c[0] for _, c in runs]
        return {"time_to_f1_s_median": float(np.median([h[1] for h in ok])) if len(ok) == len(hits) else None,
                "sweeps_to_f1": [h[0] if h else None for h in hits],
                "time_to_f1_s": [round(h[1], 4) if h else None for h in hits],
                "f1_after_5_sweeps": float(np.mean([a[2] for a in at5])),
                "recall_after_5_sweeps": float(np.mean([a[3] for a in at5])),
                "f1_after_%d_sweeps" % max_sweeps: float(np.mean([a[2] for a in last])),
                "loc_err_km_after_%d_sweeps" % max_sweeps: float(np.mean([a[4] for a in last])),
                "us_per_sweep": float(np.mean([a[1] / a[0] for a in last]) * 1e6)}

    plain = summary([chain(None, s) for s in seeds])
    net = cm.Net(max_batch=256, seed=CHAIN_SEED)
    geo = cm.create_model(None, w.stations, w.signals, cm.make_params(P, k_per_phase=K_PER_PHASE, dtype=cm.F32))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = net.train(geo, 4000, 256, 3e-4)
    train_s = time.perf_counter() - t0
    tiles, origins = cm.grid_tiles(10, 100.0)
    t0 = time.perf_counter()
    tab, centre = net.birth_table(geo, tiles, origins, 80, 80, 360, hop_s=12.8, magnitudes=True)
    table_s = time.perf_counter() - t0
    learned = summary([chain(tab, s, centre) for s in seeds])
    learned_prior_m = summary([chain(tab, s) for s in seeds])
    net.destroy()
    geo.destroy()
    lv = learned["time_to_f1_s_median"]
    line = {"metric": "time to F1 >= 0.9 (detectable zone), learned birth mixture vs plain", "value": lv,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f32 sweep, bf16 network",
            "data": "synthetic (seeded worldgen, the model's generative story)",
            "config": {"workload": "1000x1000 km, 1 h, Lambda 500, 100 jittered stations, f32 signals, 10x10 "
                                   "regions, k=32, empty start, %d chains per sampler, F1 every %d sweeps"
                                   % (len(seeds), every),
                       "network": "4 conv1d (64 ch, k5, s2) + 1024-512-4101 MLP, 1M simulated windows",
                       "table": "80x80 pixels x 360 bins, mix 0.5, magnitude windows of half-width %.2f "
                                "around the network's per-entry magnitude" % MAG_HALF_WIDTH},
            "plain": plain, "learned": learned, "learned_prior_magnitudes": learned_prior_m, "training_s": train_s, "training_loss": loss, "table_s": table_s,
            "learned_time_to_f1_s_with_training_amortised_over_256":
                None if lv is None else lv + (train_s + table_s) / 256.0,
            "vs_baseline": None}
    print(json.dumps(line))


def run_learned_posterior(args):
    """Long-run posterior summaries of the plain sampler and of the learned
    birth mixture on the 1000 x 1000 km, 1 h, 100-station float32 world: 4
    chains each from the empty set; summaries every 100 sweeps over sweeps
    2000-4000 (both) and 14000-16000 (plain).  Both chains target the same
    posterior; the plain chain's summaries judge the learned chain's."""
    import torch
    import paper_1612_00595_gb300 as cm
    from paper_1612_00595_gb300 import metrics
    torch.cuda.set_device(0)
    w = worldgen.config_learned(seed=SEED)
    P = w.params
    net = cm.Net(max_batch=256, seed=CHAIN_SEED)
    geo = cm.create_model(None, w.stations, w.signals, cm.make_params(P, k_per_phase=K_PER_PHASE, dtype=cm.F32))
    net.train(geo, 4000, 256, 3e-4)
    tab, centre = net.birth_table(geo, *cm.grid_tiles(10, 100.0), 80, 80, 360, hop_s=12.8, magnitudes=True)
    net.destroy()
    geo.destroy()

    def chain(learned, seed, burn, n):
        m = cm.create_model(None, w.stations, w.signals,
                            cm.make_params(P, k_per_phase=K_PER_PHASE, seed=seed, dtype=cm.F32))
        m.partition_and_color(P.L)
        if learned:
            m.set_birth_table(tab, 0.5)
            m.set_birth_magnitude(centre, MAG_HALF_WIDTH)
        m.run_sweeps(burn)
        rows = []
        for _ in range((n - burn) // 100):
            m.run_sweeps(100)
            ev, _, lp, _ = m.read_state()
            sc = metrics.scores(w.events, ev, P.L, P.tau, w.stations, P.R_max)
            rows.append((sc["f1"], sc["precision"], sc["recall"], sc["loc_err"],
                         float(metrics.detectable(ev, w.stations, P.R_max).sum()), lp))
        m.destroy()
        return np.array(rows).mean(axis=0)

    keys = ["f1", "precision", "recall", "loc_err_km", "detectable_events", "log_density"]
    runs = {"plain_2000_4000": (False, 2000, 4000), "plain_14000_16000": (False, 14000, 16000),
            "learned_2000_4000": (True, 2000, 4000)}
    out = {}
    for name, (learned, burn, n) in runs.items():
        per = np.array([chain(learned, CHAIN_SEED + 100 + i, burn, n) for i in range(4)])
        out[name] = {k: {"mean": float(per[:, j].mean()), "se": float(per[:, j].std(ddof=1) / 2.0),
                         "chains": [round(float(x), 4) for x in per[:, j]]} for j, k in enumerate(keys)}
    print(json.dumps({"metric": "posterior summaries, plain vs learned birth mixture", "unit": "summaries",
                      "config": {"workload": "1000x1000 km, 1 h, Lambda 500, 100 stations, f32, 4 chains per "
                                             "entry, empty start, summaries every 100 sweeps over the window"},
                      "data": "synthetic (seeded worldgen)", "results": out}))


def run_profile_case(args):
    """A named workload for a profiler: build the model, run --warmup sweeps,
    then --steps sweeps (or training steps), print a one-line summary.

    Workloads: ``scale`` (4000 x 4000 km, 24 h, 1600 stations, float32),
    ``corner`` (1000 x 1000 km of the same density and record length, 100
    stations: 0.7 GB of signals + variance, larger than L2), ``replay``
    (1000 x 1000 km, 1 h, 100 stations, float64; with --p-pair, --sig-a,
    --p-arr), ``train`` (the learned birth network: --warmup then --steps
    training steps of 256 windows simulated from the 1000 km, 1 h,
    100-station float32 world)."""
    import paper_1612_00595_gb300 as cm
    name = args.profile_case
    if name == "train":
        w = worldgen.config_learned(seed=1000)
        m = cm.create_model(None, w.stations, w.signals, cm.make_params(w.params, k_per_phase=K_PER_PHASE, seed=7,
                                                                        dtype=cm.F32))
        net = cm.Net(max_batch=256, seed=7)
        net.train(m, args.warmup, 256, 3e-4)
        t0 = time.perf_counter()
        loss = net.train(m, args.steps, 256, 3e-4)   # returns after the stream has finished
        dt = time.perf_counter() - t0
        print("training steps %d  loss %.4f  %.3f ms per step of 256 windows" % (
            args.warmup + args.steps, loss, 1e3 * dt / max(args.steps, 1)))
        net.destroy()
        m.destroy()
        return
    if name == "scale":
        w = worldgen.config_scale(seed=SEED)
    elif name == "corner":
        w = worldgen.config_scale(seed=SEED, side_regions=10)
    elif name == "replay":
        w = worldgen.config_replay(seed=SEED, sig_a=args.sig_a)
    else:
        raise SystemExit("unknown profile case " + name)
    dtype = cm.F32 if w.signals.dtype == np.float32 else cm.F64
    m = cm.create_model(w.events, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=K_PER_PHASE, seed=7, dtype=dtype, p_pair=args.p_pair,
                                       sig_a=args.sig_a, p_arr=args.p_arr))
    if args.sig_a:
        m.set_arrival_offsets(w.offsets)
    m.partition_and_color(w.params.L, shift_mode=1)
    m.run_sweeps(args.warmup)
    m.sync()
    m.run_sweeps(args.steps)
    ev, ids, lp, st = m.read_state()
    print("events %d  proposals %d  accepted %s  pair %s  launches %d" % (
        len(ev), n_proposals(st), st["accepted"], st["pair"], st["kernel_launches"]))
    m.destroy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=["scale", "replay", "batched", "learned", "learned-posterior"])
    ap.add_argument("--likelihood", default="variance", choices=["variance", "mean"],
                    help="scale workload: arrivals add to the sample variance (default) or to its mean")
    ap.add_argument("--p-pair", type=float, default=0.0,
                    help="replay or scale workload: share of steps that propose the joint move of a pair of events")
    ap.add_argument("--sig-a", type=float, default=0.0,
                    help="replay or scale workload: latent arrival times with offsets ~ N(0, sig_a^2) seconds")
    ap.add_argument("--p-arr", type=float, default=0.0, help="replay or scale workload: share of arrival-time moves")
    ap.add_argument("--sig-da", type=float, default=1.0, help="step of the arrival-time move, seconds")
    ap.add_argument("--profile-case", default=None, choices=["scale", "corner", "replay", "train"],
                    help="run a named workload for a profiler (--warmup, then --steps sweeps) and print a summary")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if (args.sig_a or args.p_arr) and args.workload not in ("replay", "scale"):
        raise SystemExit("--sig-a and --p-arr need the replay or the scale workload")
    if (args.sig_a or args.p_arr) and args.likelihood != "variance":
        raise SystemExit("--sig-a and --p-arr need the variance reading")
    if args.p_pair and args.workload not in ("replay", "scale"):
        raise SystemExit("--p-pair needs the replay or the scale workload")
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "learned-posterior":
        run_learned_posterior(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
