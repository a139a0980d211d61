"""Benchmark: SSA events per second of the batched direct method on GB300.

Workload (one "step"): the 32-species / 64-reaction flat network, 65,536
replicas x ~1e5 events each, sampled on a 1,000-point grid (int32 states
[65536, 1000, 32] = 8.4 GB written per step), FP64 propensities and time.
A step is one cwc_simulate call over the whole batch; events = applied
reactions summed over trajectories.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank simulates its own shard of replicas
(replica_offset = rank * R, so the shards are distinct trajectories of one
larger batch; no collective on the data path) and rank 0 prints one JSON line
with the events of all ranks over the slowest rank's time ("weak" scaling).
``--impl reference`` times the CPU oracle (the reference arm) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "flat32x64"
WORKLOAD_DESC = ("flat mass-action network, 32 species, 64 reactions (8 inflow/outflow pairs, 32 conversions, "
                 "16 bimolecular), 65536 replicas x ~1e5 events, 1000-point grid, int32 states, FP64 propensities/time")
SWEEP_DESC = ("flat32x64's network under 256 rate vectors (two decades of scale, trajectory lengths ~65x apart) "
              "x 256 replicas, 1000-point grid, tail layout (the last trajectories handed to 16-lane groups)")
CWC_DESC = ("compartmentalised CWC, 3 labels below the top, 24 species, 48 rules (transport, wrap binding, create, "
            "dissolve), <=64 compartments per term, 16384 replicas x ~1e4 events, 500-point grid, 172 observables")
METRIC = "SSA events/sec"
UNIT = "events/s"
KERNEL_SOURCES = ["paper_1010_2438_gb300/csrc/flat_ssa.cu", "paper_1010_2438_gb300/csrc/ssa_device.cuh",
                  "paper_1010_2438_gb300/csrc/cwc_internal.h"]
# Nominal FP64 pipe of one GB300: 152 SMs x 2 FP64 lanes per clock x 2.07 GHz
# (the nominal 1.25 TFLOP/s dense FP64 counts an FMA as two flops).  The
# roofline's peak is measured live instead (cwc_fp64_peak: a DADD/DMUL stream
# on the same GPU in the same run).
FP64_NOMINAL_OPS = 152 * 2 * 2.07e9


CWC_KERNEL_SOURCES = ["paper_1010_2438_gb300/csrc/cwc_ssa.cu", "paper_1010_2438_gb300/csrc/ssa_device.cuh",
                      "paper_1010_2438_gb300/csrc/cwc_internal.h"]


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for p in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def capture_record(name: str, workload: str, sources):
    """The ncu counters of a kernel (profiles/<name>_traffic.txt, JSON), if
    they were captured on the current sources of that kernel, else None."""
    path = os.path.join(ROOT, "profiles", name + "_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("kernel_source_hash") != kernel_source_hash(sources) or rec.get("workload") != workload:
        return None
    return rec


def fp64_ops_per_event(model) -> float:
    """Algorithmic FP64 arithmetic operations of one event of the method
    (written specification), averaged uniformly over the rules fired:
      tau = -L / a0 (1), t + tau (1), x = u_sel * a0 (1)                 =  3
      tree descent: one subtraction per level (5) + leaf scan (B products,
      B-1 adds)
      update: one k_i * H_i per dependent, (B-1) adds per dirty leaf, one add
      per dirty internal node.
    The logarithm is integer fixed-point arithmetic and, like Philox, the
    uniforms, the counts, comparisons of doubles as bit patterns and hashing,
    is not counted."""
    from paper_1010_2438_gb300.workloads import Model  # noqa: F401
    M, S = model.n_rules, model.n_species
    B = (M + 31) // 32
    lhs = model.lhs[:, 0, :]
    delta = model.rhs[:, 0, :] - lhs
    upd = []
    for j in range(M):
        changed = set(np.nonzero(delta[j])[0].tolist())
        deps = [i for i in range(M) if changed & set(np.nonzero(lhs[i])[0].tolist())]
        leaves = sorted(set(i // B for i in deps))
        nodes = set()
        for l in leaves:
            nodes |= {l >> 1, 16 + (l >> 2), 24 + (l >> 3), 28 + (l >> 4), 30}
        upd.append(len(deps) + (B - 1) * len(leaves) + len(nodes))
    return 3 + 5 + B + (B - 1) + float(np.mean(upd))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
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
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def oracle_events_per_sec(batch, n_traj: int, threads: int, q_begin: int = 0):
    """The oracle, unchanged, as an on-demand farm of ``threads`` host threads
    (each takes the next unstarted trajectory when it finishes one)."""
    import oracle
    t0 = time.perf_counter()
    res = oracle.simulate(batch, q_begin, q_begin + n_traj, states=True, threads=threads, schedule="farm")
    dt = time.perf_counter() - t0
    ev = int(res["events"].sum())
    return ev / dt, ev, dt


def cpu_baseline(batch, threads: int, n_traj: int, n_single: int):
    rate, ev, dt = oracle_events_per_sec(batch, n_traj, threads)
    rate1, ev1, dt1 = oracle_events_per_sec(batch, n_single, 1, q_begin=n_traj)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "schedule": "on-demand farm (a thread takes the next trajectory when it finishes one)",
            "sample": "%d of %d trajectories (%d events, %.1f s wall on %d threads), full horizon and grid"
                      % (n_traj, batch.n_traj, ev, dt, threads),
            "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                            "sample": "%d further trajectories (%d events, %.1f s) on one thread"
                                      % (n_single, ev1, dt1)}}


# ---------------------------------------------------------------------------
# Other workloads of the path (one timed step each, after one warm-up)
# ---------------------------------------------------------------------------

CLOCK_LOG = {}


def _timed(fn, name=None):
    """One warm-up call, then one call timed with CUDA events; the SM clock is
    sampled during the timed call and kept in CLOCK_LOG[name]."""
    import torch
    fn()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if name else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        CLOCK_LOG[name] = sampler.stop()
    return out, e0.elapsed_time(e1) / 1e3


def measure_extras(dev):
    import torch

    from paper_1010_2438_gb300 import api, capi
    from paper_1010_2438_gb300 import workloads as W
    extras = {}
    # compartmentalised CWC: 16,384 replicas x ~1e4 events, 500-point grid, 172 observables
    b = W.cwc3x24()
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b, dev)
    lay, thr, lanes, _ = api.autotune(cm, rates, init, grid, b.R, b.seed, tune_events=500)
    keep = {}

    def run_cwc():
        keep["o"] = api.simulate(cm, rates, init, grid, b.R, b.seed, states=True, out=keep.get("o"))
        return keep["o"]

    out, sec = _timed(run_cwc, "cwc3x24")
    ev = int(out["events"].sum().item())
    # roofline of the compartment kernel: no FP64-bound step (its FP64 work
    # is the flat step's, shared by a lane group); it is latency / issue
    # bound, so the entry reports the issue-slot fraction and the DRAM bytes
    # per event against the algorithmic bytes (the int32 observables written
    # at the grid points) from the ncu capture of the same kernel sources
    alg_bytes = 4.0 * b.G * cm.n_observables * b.n_traj / ev
    cap = capture_record("cwc_ssa_kernel_cwc3x24", "cwc3x24", CWC_KERNEL_SOURCES)
    roof = {"bound": "issue", "algorithmic_bytes_per_event": alg_bytes,
            "dram_bytes_per_event": None if cap is None else cap.get("dram_bytes_per_event"),
            "issue_active_frac": None if cap is None else cap.get("issue_active_frac"),
            "warps_per_sm": None if cap is None else cap.get("warps_per_sm"),
            "source": "ncu capture of the profiling case on the same kernel sources (hash-checked); null if stale"}
    # the same with 16-bit term counts (term_bits = 16): half the slab bytes
    keep16 = {}

    def run_cwc16():
        keep16["o"] = api.simulate(cm, rates, init, grid, b.R, b.seed, states=True, out=keep16.get("o"), term_bits=16)
        return keep16["o"]

    out16, sec16 = _timed(run_cwc16, "cwc3x24_16bit")
    same16 = bool(torch.equal(out16["hash"], out["hash"]) and torch.equal(out16["states"], out["states"]))
    cap16 = capture_record("cwc_ssa_kernel16_cwc3x24", "cwc3x24", CWC_KERNEL_SOURCES)
    extras["cwc3x24"] = {"events_per_s": ev / sec, "events": ev, "seconds": sec, "layout": lay, "block_threads": thr,
                         "lanes_per_trajectory": lanes, "roofline": roof,
                         "term_bits_16": {"events_per_s": ev / sec16, "seconds": sec16, "identical": same16,
                                          "dram_bytes_per_event": None if cap16 is None
                                          else cap16.get("dram_bytes_per_event"),
                                          "issue_active_frac": None if cap16 is None
                                          else cap16.get("issue_active_frac")},
                         "workload": "3 labels below the top, 24 species, 48 rules (transport, wrap binding, create, "
                                     "dissolve), <=64 compartments, 16384 replicas, 500-point grid"}
    del out, keep, out16, keep16
    # uneven sweep: 256 rate vectors x 256 replicas of flat32x64's network, CUDA
    # graph; the autotuned queue / static layout, then the tail layout (the last
    # trajectories handed over to a warp each), which must agree bit for bit
    b = W.sweep256x256()
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b)
    lay, thr, _, _ = api.autotune(cm, rates, init, grid, b.R, b.seed, tune_events=2000)
    g = api.GraphedSimulation(cm, rates, init, grid, b.R, b.seed, states=True)
    out_q, sec_q = _timed(g.replay, "sweep256x256_queue")
    ev_q, hash_q = out_q["events"].clone(), out_q["hash"].clone()
    del g, out_q
    g = api.GraphedSimulation(cm, rates, init, grid, b.R, b.seed, states=True, layout=capi.CWC_LAYOUT_TAIL)
    out, sec = _timed(g.replay, "sweep256x256")
    same = bool(torch.equal(out["events"], ev_q) and torch.equal(out["hash"], hash_q))
    evp = out["events"].double().mean(dim=1)
    ev = int(out["events"].sum().item())
    extras["sweep256x256"] = {"events_per_s": ev / sec, "events": ev, "seconds": sec,
                              "layout": "tail (queue, then the last trajectories on a lane group each)", "graph": True,
                              "queue_layout": {"events_per_s": ev / sec_q, "seconds": sec_q, "layout": lay,
                                               "block_threads": thr},
                              "identical_to_queue_layout": same,
                              "length_spread": float((evp.max() / evp.min()).item()),
                              "workload": "256 rate vectors x 256 replicas, flat32x64 network, 1000-point grid"}
    del g, out
    # the paper's n-species Lotka-Volterra family (its single-instance table runs n = 2 ... 32)
    lv = {}
    for nsp in (2, 4, 8, 16, 32):
        b = W.lotka_volterra(nsp, R=32768, G=100, T=1.0)
        cm = api.CompiledModel(b.model)
        rates, init, grid = api.device_inputs(b, dev)
        keep = {}

        def run_lv():
            keep["o"] = api.simulate(cm, rates, init, grid, b.R, b.seed, states=True, out=keep.get("o"))
            return keep["o"]

        out, sec = _timed(run_lv, "lotka_volterra_%d" % nsp)
        ev = int(out["events"].sum().item())
        lv[str(nsp)] = {"events_per_s": ev / sec, "events": ev, "seconds": sec}
        del keep, out
    extras["lotka_volterra"] = {"by_species": lv, "workload": "n-species Lotka-Volterra chain, 32768 replicas, "
                                                            "horizon 1, 100-point grid (Gillespie 1977 constants)"}
    # Michaelis-Menten kinetics (the flat kernel's rate-law variant): a 20-stage
    # kinase cascade, 41 species, 40 reactions, beside the same network with
    # mass-action rates (another process, for the cost of the law's division)
    mm = {}
    for law in ("michaelis_menten", "mass_action"):
        b = W.mm_cascade(stages=20, R=65536, G=100, T=20.0)
        model = b.model if law == "michaelis_menten" else dataclasses.replace(b.model, rate_law=None, rate_par=None)
        rates_np = b.rates if law == "michaelis_menten" else b.rates * 0.01
        b = W.Batch(model, rates_np, b.init, b.grid, b.R, b.seed, name=b.name)
        cm = api.CompiledModel(b.model)
        rates, init, grid = api.device_inputs(b, dev)
        keep = {}

        def run_mm():
            keep["o"] = api.simulate(cm, rates, init, grid, b.R, b.seed, states=True, out=keep.get("o"))
            return keep["o"]

        out, sec = _timed(run_mm, "mm_cascade20_" + law)
        ev = int(out["events"].sum().item())
        mm[law] = {"events_per_s": ev / sec, "events": ev, "seconds": sec}
        del keep, out
    extras["mm_cascade20"] = dict(mm["michaelis_menten"], mass_action_same_network=mm["mass_action"],
                                  workload="20-stage kinase cascade with Michaelis-Menten rates (41 species, 40 "
                                           "reactions), 65536 replicas, horizon 20, 100-point grid; the mass-action "
                                           "line runs the same reactions with k / 100")
    # likelihood-ratio sensitivities: 16 species x 24 reactions, 131,072 replicas, 100-point grid
    b = W.flat16x24()
    cm = api.CompiledModel(b.model)
    rates, init, grid = api.device_inputs(b, dev)
    fwd, t_fwd = _timed(lambda: api.simulate(cm, rates, init, grid, b.R, b.seed, states=False, means=True, traj=True),
                        "flat16x24_forward")
    ev = int(fwd["events"].sum().item())
    gm = torch.ones_like(fwd["means"])
    _, t_bwd = _timed(lambda: api.sensitivity(cm, rates, init, grid, b.R, b.seed, fwd["means"], gm),
                      "flat16x24_backward")
    extras["flat16x24_sensitivity"] = {"forward_events_per_s": ev / t_fwd, "forward_s": t_fwd, "backward_s": t_bwd,
                                       "grad_over_fwd": t_bwd / t_fwd, "events": ev,
                                       "workload": "d E[X(g)]/d k for 24 rates, 131072 replicas, 100-point grid"}
    # SM clock (median MHz) and throttle reasons seen during each timed call
    extras["clocks"] = {k: {"sm_mhz": v.get("sm_mhz"), "reasons": v.get("reasons")} for k, v in CLOCK_LOG.items()}
    return extras


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1010_2438_gb300 import workloads as W
    batch = W.flat32x64()
    threads = os.cpu_count() or 1
    n_traj = max(threads, 2 * threads)
    for _ in range(args.warmup):
        oracle_events_per_sec(batch, threads, threads)
    times, evs = [], []
    for _ in range(args.steps):
        rate, ev, dt = oracle_events_per_sec(batch, n_traj, threads)
        times.append(dt)
        evs.append(ev)
    value = sum(evs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC,
                       "sample_per_step": "%d trajectories" % n_traj},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "schedule": "on-demand farm",
                             "sample": "%d of 65536 trajectories per step, full horizon and grid" % n_traj},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads of the path")
    ap.add_argument("--layout", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0, help="lanes per trajectory (compartment workload; 0 = automatic)")
    ap.add_argument("--term-bits", type=int, default=0, help="compartment workload: 16 for 16-bit term counts")
    ap.add_argument("--replicas", type=int, default=0, help="smaller case for profiling (default: 65536)")
    ap.add_argument("--horizon-scale", type=float, default=1.0, help="scale the time grid (profiling only)")
    ap.add_argument("--grid-points", type=int, default=0, help="grid points (profiling only; default 1000)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "cwc3x24", "sweep256x256"],
                    help="profiling only: run the compartment workload, or the uneven sweep in the tail "
                         "layout, as the timed step")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    from paper_1010_2438_gb300 import api, capi, shard
    from paper_1010_2438_gb300 import build as lib_build
    from paper_1010_2438_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    lib_build.build()
    layout = args.layout
    if args.workload == "cwc3x24":
        batch = W.cwc3x24(R=args.replicas or 16384, G=args.grid_points or 500)
    elif args.workload == "sweep256x256":
        batch = W.sweep256x256(R=args.replicas or 256, G=args.grid_points or 1000)
        layout = layout or capi.CWC_LAYOUT_TAIL
    else:
        batch = W.flat32x64(R=args.replicas or 65536, G=args.grid_points or 1000)
    if args.horizon_scale != 1.0:
        batch = W.Batch(batch.model, batch.rates, batch.init, batch.grid * args.horizon_scale, batch.R, batch.seed,
                        name=batch.name)
    R = batch.R
    # kernels of this library per step: the SSA kernel; for the sweep in the
    # tail layout also the queue order (estimate, rank) and the hand-over
    # (collect, rank, lane-group kernel)
    launches_per_step = 6 if args.workload == "sweep256x256" else 1
    r_off, _ = shard.weak_shard(R, rank)
    cm = api.CompiledModel(batch.model)
    rates, init, grid = api.device_inputs(batch, dev)
    stream = torch.cuda.current_stream()
    l2_flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = None

    def step(o):
        return api.simulate(cm, rates, init, grid, R, batch.seed, batch.max_events, states=True, traj=True,
                            layout=layout, block_threads=args.threads, lanes=args.lanes, replica_offset=r_off,
                            term_bits=args.term_bits,
                            out=o)

    for _ in range(args.warmup):
        out = step(out)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    barrier()
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        l2_flush.zero_()                      # write 256 MiB > L2 between timed steps
        starts[i].record(stream)
        out = step(out)
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_total = sum(step_ms) / 1e3
    events = int(out["events"].sum().item())
    statuses = torch.bincount(out["status"].reshape(-1).to(torch.int64), minlength=8).tolist()
    ev_all, t_max = shard.combine(events * args.steps, t_total, device=dev)
    value = ev_all / t_max

    # roofline of the dominant kernel (the SSA kernel is the whole step but a
    # 256-byte workspace memset)
    f_evt = fp64_ops_per_event(batch.model)
    kernel_s = t_total / args.steps
    achieved = f_evt * events / kernel_s
    traffic = None
    issue = None
    tj = capture_record("flat_ssa_kernel_flat32x64", args.workload, KERNEL_SOURCES)
    if tj is not None:
        traffic = tj.get("dram_bytes_per_launch")
        # issue-rate roofline of the same kernel (warp instructions issued per
        # scheduler cycle, of the 1 per cycle peak) and the FP64 pipe's busy
        # fraction, from the ncu capture of the profiling case
        issue = {"frac": tj.get("issue_active_frac"), "fp64_pipe_frac": tj.get("fp64_pipe_frac"),
                 "warps_per_sm": tj.get("warps_per_sm"),
                 "source": "ncu smsp__issue_active / sm__pipe_fp64_cycles_active of the profiling case, "
                           "captured on the same kernel sources (hash-checked)"}
    peak = capi.cwc_fp64_peak(stream.cuda_stream)
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GFLOP/s (FP64)",
                "frac": achieved / peak, "peak_source": "measured in this run: cwc_fp64_peak (DADD/DMUL stream, "
                                                        "32 warps per SM, best of 3)",
                "nominal_peak": FP64_NOMINAL_OPS / 1e9, "frac_of_nominal": achieved / FP64_NOMINAL_OPS,
                "traffic": traffic, "issue": issue,
                "note": "FP64 pipe (the path's only floating-point unit; the logarithm is integer): %.1f algorithmic "
                        "FP64 ops/event x %d events / %.4f s (CUDA events on the launching stream); frac is of the "
                        "measured peak; issue: ncu issue-slot fraction of the same kernel" % (f_evt, events, kernel_s)}

    # end to end through host buffers (pinned): H2D inputs, simulate, D2H states
    e2e = None
    if not args.no_e2e:
        rates_h = torch.from_numpy(np.ascontiguousarray(batch.rates)).pin_memory()
        init_h = torch.from_numpy(np.ascontiguousarray(batch.init)).pin_memory()
        grid_h = torch.from_numpy(np.ascontiguousarray(batch.grid)).pin_memory()
        host_out = torch.empty(tuple(out["states"].shape), dtype=torch.int32, pin_memory=True)
        e2e_steps = min(args.steps, 3)

        def time_host(direct):
            bufs = {"out": out}
            api.simulate_host(cm, rates_h, init_h, grid_h, R, batch.seed, batch.max_events, dev_bufs=bufs,
                              host_out=host_out, replica_offset=r_off, direct=direct)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(e2e_steps):
                api.simulate_host(cm, rates_h, init_h, grid_h, R, batch.seed, batch.max_events, dev_bufs=bufs,
                                  host_out=host_out, replica_offset=r_off, direct=direct)
            e1.record(stream)
            barrier()
            return shard.combine(float(events * e2e_steps), e0.elapsed_time(e1) / 1e3, device=dev)

        ev_c, te_c = time_host(False)
        ev_e, te = time_host(True)
        h2d = rates_h.numel() * 8 + init_h.numel() * 4 + grid_h.numel() * 8
        e2e = {"value": ev_e / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": host_out.numel() * 4, "steps": e2e_steps,
               "d2h": "the kernel stores the grid states into page-locked host memory while it runs (NVLink-C2C); "
                      "inputs copied host to device each step",
               "copy_after": {"value": ev_c / te_c, "unit": UNIT,
                              "d2h": "states to device memory, then one copy to page-locked host memory"}}

    extras = None
    if world == 1 and not args.no_extras:
        extras = measure_extras(dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cpu = cpu_baseline(batch, threads, min(batch.n_traj, 6 * threads), 8)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if not (args.replicas or args.grid_points or args.horizon_scale != 1.0
                                                    or args.workload != WORKLOAD)
                       else "%s (profiling case: R=%d, G=%d, horizon x%g)" % (args.workload, R, batch.G,
                                                                               args.horizon_scale),
                       "description": {WORKLOAD: WORKLOAD_DESC, "cwc3x24": CWC_DESC}.get(args.workload, SWEEP_DESC),
                           "P": batch.P, "R": R,
                           "G": batch.G, "S": batch.model.n_species, "M": batch.model.n_rules,
                           "events_per_step_per_gpu": events, "statuses": statuses,
                           "layout": ["auto(queue)", "static", "queue", "tail"][layout],
                           "l2": "256 MiB buffer written between timed steps; outputs 8.4 GB per step",
                           "parallelism": "replica shards, %d GPU(s)" % world},
                "gpu_launches": args.steps * launches_per_step, "clocks": clk, "roofline": roofline,
                "e2e": e2e, "cpu_baseline": cpu, "extras": extras,
                "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
