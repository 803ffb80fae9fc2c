#!/usr/bin/env python3
"""Benchmark: output transitions/s of timing-aware 4-value re-simulation of a
1M-gate synthetic netlist on one GB300 (the paper's hot path, Sec. 4).

One step = one whole simulation of the netlist under its stimulus: every
level of the DAG evaluated on the device (Algorithm 2 + Eq. 1 per gate), all
output waveforms written to the device waveform store.

Default line (own arm):
  value    gate-output transitions / device time per step, stimulus already
           resident in HBM (CUDA events on the launching stream);
  e2e      the same metric through the public API from host buffers: each
           step copies the stimulus in (pinned host -> device), simulates and
           copies every waveform out (device -> pinned host);
  roofline level kernel's algorithmic bytes / its event-timed duration
           against the measured HBM copy bandwidth;
  cpu_baseline  the CPU oracle (event-driven, one thread) on a bounded sample
           of the same workload (the same netlist, a shorter time window).
--impl reference times that CPU oracle alone and prints its own line.
Multi-GPU (torchrun): replicas only -- every rank simulates its own copy of
the workload, no collective on the data path; value = all ranks' transitions
/ the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "output transitions/s and sim time, 1M gates, 1 GB300; served p50/p99 vs plain run"
UNIT = "transitions/s"
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--mode", default="plain", choices=["plain", "batch", "serve", "sliced", "cells"],
                    help="plain: one 1M-gate run (the headline); batch: 64 stimulus sets + 16 netlists "
                         "in batched launches vs one at a time; serve: 200 req/s over resident netlists, "
                         "continuous batching vs plain; sliced: time slices and a 2.97e9 ps stimulus; "
                         "cells: 1M general cells vs built-in cells")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--batch-sets", type=int, default=64)
    ap.add_argument("--batch-netlists", type=int, default=16)
    ap.add_argument("--workload", default="ind1m")
    ap.add_argument("--slice-ps", type=int, default=1_000_000, help="sliced mode: slice length on the 1M-gate run")
    ap.add_argument("--long-window", type=int, default=2_970_000_000,
                    help="sliced mode: duration of the long (64-bit time) stimulus, ps")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-frac", type=float, default=0.012,
                    help="time-window fraction of the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--gates", type=int, default=0, help="override the recipe's gate count (profiling cases)")
    ap.add_argument("--pis", type=int, default=0, help="override the recipe's primary-input count")
    ap.add_argument("--arena-words", type=int, default=0, help="event arena size (0: size from a first run)")
    ap.add_argument("--schedule", default="dependency", choices=["dependency", "levels"])
    ap.add_argument("--order", default="planned", choices=["planned", "level"],
                    help="dependency schedule: critical-path-first order planned from a calibration run "
                         "(an independent stimulus over 5%% of the window), or plain level order")
    ap.add_argument("--warps-per-cta", type=int, default=0)
    ap.add_argument("--kernel", default="wide", choices=["windowed", "wide", "segmented"])
    ap.add_argument("--segment", type=int, default=0, help="segmented kernel: transitions per lane segment")
    return ap.parse_args()


def overrides(a):
    ov = {}
    if a.gates:
        ov["net_n_gates"] = a.gates
    if a.pis:
        ov["net_n_pi"] = a.pis
    return ov


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_reduce(x: float, op: str, device: str) -> float:
    """MAX or SUM of x over the replica ranks (x itself on a single rank):
    the slowest rank's time, the transitions of all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def describe(name, w):
    r = w.recipe
    nl, st = w.netlist, w.stimulus
    return {
        "workload": f"{name}: {nl.n_gates} gates / {nl.n_pi} PIs / depth {r['net']['depth']}, "
                    f"{st.n_events} stimulus transitions over {r['stim']['window']} ps",
        "gates": nl.n_gates, "primary_inputs": nl.n_pi, "depth": r["net"]["depth"],
        "stimulus_transitions": st.n_events, "window_ps": r["stim"]["window"],
        "wcv": round(st.wcv(), 4), "seed": r["seed"],
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 25 ms (a timed
    region of ten 1M-gate runs lasts about 180 ms)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.m = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()   # let the sampler start before the timed region
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 3.0:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def mark(self):
        """Start of the timed region: summary() uses the samples after it."""
        self.m = len(self.lines)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.m:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("gls_eval.cu", "gls_internal.h"):
        with open(os.path.join(ROOT, "paper_2304_13398_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, cfg: dict):
    """DRAM bytes per run of the gate kernel from a committed ncu summary,
    valid only for the configuration it was taken on (sizes, seed, schedule,
    kernel variant) and while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "gate_kernel_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_source_sha") != kernel_source_sha():
        return None
    if any(cfg.get(k) != v for k, v in e.get("applies_to", {}).items()):
        return None
    return e.get("dram_bytes_per_run")


def algorithmic_bytes(nl, off):
    """Per run: every fanin arc reads its net's waveform once (4 B per
    transition), every gate writes its output (4 B per transition), plus the
    gate record (48 B), the fanin net descriptors (12 B each) and the output
    descriptor (12 B)."""
    lens = np.diff(off)
    fanin = 4 * int(lens[nl.fanin_net].sum())
    out = 4 * int(lens[nl.n_pi:].sum())
    meta = 48 * nl.n_gates + 12 * len(nl.fanin_net) + 12 * nl.n_gates
    return fanin + out + meta


def cpu_baseline(name, seed, frac):
    import oracle
    import synth
    r = synth.RECIPES[name]["stim"]
    ov = dict(stim_window=max(1, int(r["window"] * frac)), stim_mean=r["mean"] * frac)
    if r.get("clock_trans"):
        ov["stim_clock_trans"] = max(1, int(r["clock_trans"] * frac))
    w = synth.make_workload(name, seed=seed, **ov)
    t0 = time.perf_counter()
    res = oracle.sim_event(w.netlist, w.stimulus)
    dt = time.perf_counter() - t0
    e_out = int(res.off[-1] - res.off[w.netlist.n_pi])
    return {"value": e_out / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"event-driven oracle, 1 thread, same {w.netlist.n_gates}-gate netlist, first {frac:g} of the "
                      f"time window ({w.stimulus.n_events} stimulus / {e_out} output transitions, {dt:.1f} s)",
            "seconds": round(dt, 2), "output_transitions": e_out}


def cpu_levelized(name, seed, frac):
    """The oracle's second evaluator (levelized, OpenMP over the gates of a
    level) on every host core, same bounded sample as cpu_baseline."""
    import oracle
    import synth
    r = synth.RECIPES[name]["stim"]
    ov = dict(stim_window=max(1, int(r["window"] * frac)), stim_mean=r["mean"] * frac)
    if r.get("clock_trans"):
        ov["stim_clock_trans"] = max(1, int(r["clock_trans"] * frac))
    w = synth.make_workload(name, seed=seed, **ov)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = oracle.sim_levelized(w.netlist, w.stimulus, nthreads=cores)
    dt = time.perf_counter() - t0
    e_out = int(res.off[-1] - res.off[w.netlist.n_pi])
    return {"value": e_out / dt, "unit": UNIT, "cores": cores, "kind": "oracle (levelized, OpenMP)",
            "sample": f"same sample as cpu_baseline ({dt:.1f} s)", "seconds": round(dt, 2)}


# Arm "CPU part" numbers of the Neoverse cores found in Grace-class hosts
ARM_PARTS = {"0xd40": "Neoverse-V1", "0xd4f": "Neoverse-V2", "0xd84": "Neoverse-V3", "0xd0c": "Neoverse-N1",
             "0xd49": "Neoverse-N2"}


def cpu_model():
    """Host CPU model: the x86 model name, or the Arm core by part number."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key, _, val = ln.partition(":")
                key, val = key.strip().lower(), val.strip()
                if key == "model name":
                    return val
                if key == "cpu part":
                    return f"{ARM_PARTS.get(val.lower(), 'Arm core')} (CPU part {val}, {os.uname().machine})"
    except OSError:
        pass
    return os.uname().machine


REF_RUN_SECONDS = 120.0   # oracle time of all timed steps of the reference arm together


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    w = synth.make_workload(a.workload, seed=a.seed, **overrides(a))
    cfg = describe(a.workload, w)
    # the untimed warm-up samples (a quarter of the default size) also give
    # the oracle's pace, from which every timed step's sample is sized so
    # that all K of them take about REF_RUN_SECONDS together
    fw = a.cpu_frac / 4
    pace = 0.0
    for _ in range(max(a.warmup, 1)):
        pace = cpu_baseline(a.workload, a.seed, fw)["seconds"] / fw
    frac = min(a.cpu_frac, REF_RUN_SECONDS / max(1, a.steps) / max(pace, 1e-9))
    vals, secs = [], []
    for _ in range(a.steps):
        b = cpu_baseline(a.workload, a.seed, frac)
        vals.append(b["value"])
        secs.append(b["seconds"])
    v = statistics.median(vals)
    cb = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": b["sample"], "cpu": cpu_model()}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * statistics.median(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": cfg,
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


def run_own(a):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2304_13398_gb300 as gls
    import synth
    w = synth.make_workload(a.workload, seed=a.seed, **overrides(a))
    nl, st = w.netlist, w.stimulus
    ctx = gls.Context(local)
    ctx.set_schedule(a.schedule)
    ctx.set_kernel(a.kernel)
    if a.segment:
        ctx.set_option(gls.gls.GLS_OPT_SEGMENT, a.segment)
    if a.warps_per_cta:
        ctx.set_option(gls.gls.GLS_OPT_WARPS_PER_CTA, a.warps_per_cta)
    stream = torch.cuda.Stream()
    nid = ctx.load_netlist(nl)
    order = "level"
    if a.schedule == "dependency" and a.order == "planned":
        order = plan_from_calibration(ctx, nid, nl, w.recipe["stim"], a.seed, stream)
    sid = ctx.load_stimulus(st)
    # size the event arena from a first run's demand (Eq. 2 bounds summed)
    arena = a.arena_words
    rid = ctx.simulate(nid, sid, arena_events=arena, stream=stream)
    rc, demand, _ = ctx.run_stats_raw(rid)
    while rc == gls.gls.GLS_EOVERFLOW:      # the reported demand is a lower bound
        ctx.release(rid)
        arena = int(demand * 1.25) + 1024
        rid = ctx.simulate(nid, sid, arena_events=arena, stream=stream)
        rc, demand, _ = ctx.run_stats_raw(rid)
    if rc != 0:
        raise gls.GlsError(rc, "first run failed")
    stats = ctx.run_stats(rid)
    off, packed = ctx.read_all(rid)
    e_out = stats.total_events
    alg_bytes = algorithmic_bytes(nl, off)
    del packed

    for _ in range(max(a.warmup, 3)):
        ctx.rerun(rid, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    with ClockSampler(local) as clk:
        clk.mark()
        start.record(stream)
        for _ in range(a.steps):
            ctx.rerun(rid, stream)
        stop.record(stream)
        stop.synchronize()
        # level-kernel time of the last step (events around the level sequence)
        kernel_ms.append(ctx.run_stats(rid).kernel_ms)
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop) / a.steps
    for _ in range(2):   # a few more level-sequence timings for the roofline
        ctx.rerun(rid, stream)
        kernel_ms.append(ctx.run_stats(rid).kernel_ms)
    k_ms = statistics.median(kernel_ms)
    ms = replica_reduce(ms, "max", "cuda")
    all_out = replica_reduce(e_out, "sum", "cuda")   # every replica's transitions
    value = all_out / (ms / 1000.0)

    e2e = None
    if not a.no_e2e:
        N = nl.n_pi + nl.n_gates
        off_h = torch.from_numpy(st.off).pin_memory()
        t_h = torch.from_numpy(st.t).pin_memory()
        v_h = torch.from_numpy(st.v).pin_memory()
        total = int(off[-1])
        h2d = 8 * (nl.n_pi + 1) + 5 * st.n_events
        # results straight into pinned host memory: a second run of the same
        # workload whose kernels mirror every output store to the host
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 1)
        demand = ctx.run_info(rid)[0]
        mrid = ctx.simulate(nid, sid, arena_events=int(demand * 1.02) + (1 << 20), stream=stream)
        ctx.run_stats(mrid)
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 0)
        G = nl.n_gates
        goff = torch.empty(G, dtype=torch.int64).pin_memory()
        glen = torch.empty(G, dtype=torch.int32).pin_memory()
        d2h = 4 * (total - int(off[nl.n_pi])) + 12 * G   # the mirrored gate transitions + descriptors

        def e2e_step():
            ctx.update_stimulus(sid, off_h, t_h, v_h)
            ctx.rerun(mrid, stream)
            ctx.read_host(mrid, 0, goff, glen)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1000 / a.e2e_steps
        e_ms = replica_reduce(e_ms, "max", "cuda")
        e2e = {"value": all_out / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
               "timing": "host wall clock over the public calls, pinned host buffers",
               "result_path": "gls_read_host: the kernels store every output transition into a pinned host "
                              "mirror as they go; the step ends when all waveforms and their descriptors are "
                              "in host memory (primary inputs are the caller's stimulus)"}

    # `config` names the workload only (the reference arm prints the same
    # dict); how this arm ran it goes under `run`
    cfg = describe(a.workload, w)
    run_cfg = {"output_transitions_per_step": e_out, "arena_words": int(arena) if arena else "default",
               "l2_policy": "inputs larger than L2 (stimulus and intermediate waveforms >> 129 MB)",
               "parallelism": f"replicas{world}" if world > 1 else "single", "schedule": a.schedule,
               "kernel": a.kernel, "gate_order": order,
               "event_format": "packed u32 transitions (t << 2) | v: 30-bit time, 2-bit value 0/1/X/Z"}
    peak, peak_kind = measured_peak_gbs()
    achieved = alg_bytes / (k_ms / 1000.0) / 1e9
    traffic = ncu_traffic(a.workload, dict(cfg, **run_cfg))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind,
            "kernel": (f"dependency_kernel<{a.kernel}> (one launch per run)" if a.schedule == "dependency"
                       else f"level_kernel<{a.kernel}> (all levels of one run)"),
            "algorithmic_bytes_per_run": alg_bytes, "kernel_ms_per_run": k_ms}
    cb = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cb = cpu_baseline(a.workload, a.seed, a.cpu_frac)
        cb["cpu"] = cpu_model()
        cb["all_cores"] = cpu_levelized(a.workload, a.seed, a.cpu_frac)
    launches_per_step = 1 + (1 if a.schedule == "dependency" else int(w.recipe["net"]["depth"]))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": max(a.warmup, 3), "ms_per_step": ms, "sim_time_ms": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": cfg, "run": run_cfg, "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": launches_per_step * a.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def calibration_stimulus(n_pi: int, stim: dict, seed: int, frac: float = 0.05):
    """An independent stimulus of the same recipe over the first `frac` of the
    window at the same transition density (for planning the gate order)."""
    import synth
    sp = dict(stim)
    sp["window"] = max(1, int(sp["window"] * frac))
    sp["mean"] = sp["mean"] * frac
    if sp.get("clock_trans"):
        sp["clock_trans"] = max(1, int(sp["clock_trans"] * frac))
    return synth.make_stimulus(n_pi, seed=seed + 7919 + 1000003, **sp)


def plan_from_calibration(ctx, nid, nl, stim: dict, seed: int, stream=None):
    """Plan nid's dependency order from a calibration run; returns a config note."""
    cal = calibration_stimulus(nl.n_pi, stim, seed)
    cid = ctx.load_stimulus(cal)
    rid = ctx.simulate(nid, cid, stream=stream)
    ctx.run_stats(rid)
    ctx.plan_order(nid, rid)
    ctx.release(rid)
    ctx.release(cid)
    return (f"critical-path-first, planned from an independent stimulus (seed {seed + 7919}) "
            f"over 5% of the window ({len(cal.t)} PI transitions)")


def scaled_recipe(gates: int, seed: int):
    """A netlist of the 1M-gate recipe's distributions at another size:
    PIs = gates / 50, depth 20 log10(gates) - 60 clamped to [8, 60]."""
    import synth
    r = synth.RECIPES["ind1m"]
    depth = int(min(60, max(8, round(20 * np.log10(gates) - 60))))
    net = dict(r["net"], n_gates=int(gates), n_pi=max(16, int(gates) // 50), depth=depth)
    return net, dict(r["stim"]), seed


def make_scaled(gates: int, seed: int):
    import synth
    net, stim, seed = scaled_recipe(gates, seed)
    nl = synth.make_netlist(seed=seed, **net)
    st = synth.make_stimulus(net["n_pi"], seed=seed + 1000003, **stim)
    return nl, st, net, stim


def run_batch(a):
    """Batched form: 64 seeded stimulus sets on the 1M-gate netlist plus 16
    netlists of log-uniform size (10k-2M gates) with their own stimuli.
    Items run in batched launches (waves sized to fit HBM; the kernel
    configuration chosen by the autotuner) and, for comparison, one at a time."""
    import torch
    import paper_2304_13398_gb300 as gls
    import synth
    from paper_2304_13398_gb300.autotune import autotune
    torch.cuda.set_device(0)
    ctx = gls.Context(0)
    r = synth.RECIPES["ind1m"]
    nl = synth.make_netlist(seed=a.seed, **r["net"])
    nid = ctx.load_netlist(nl)
    order = plan_from_calibration(ctx, nid, nl, r["stim"], a.seed) if a.order == "planned" else "level"
    sids, pi_events = [], []
    for s in range(1, a.batch_sets + 1):
        st = synth.make_stimulus(nl.n_pi, seed=s, **r["stim"])
        sids.append(ctx.load_stimulus(st))
        pi_events.append(st.n_events)
    rng = np.random.default_rng(a.seed + 77)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), a.batch_netlists)).astype(int)
    mixed = []
    for i, G in enumerate(sizes):
        mnl, mst, _, _ = make_scaled(int(G), 5000 + i)
        mixed.append((ctx.load_netlist(mnl), ctx.load_stimulus(mst), int(G), mst.n_events))
    # per-replica arena demand, from one plain run
    rid = ctx.simulate(nid, sids[0])
    ctx.run_stats(rid)
    demand = ctx.run_info(rid)[0]
    ctx.release(rid)
    free, _ = torch.cuda.mem_get_info()
    per = int(demand * 1.05) + (1 << 20)
    wave = max(1, min(a.batch_sets, int(0.8 * free / (4 * per + 16 * (nl.n_pi + nl.n_gates)))))
    # autotune on one wave of replicas
    tune = autotune(ctx, lambda: ctx.simulate_batch([nid] * wave, sids[:wave], arena_events=per * wave))
    waves, b_ms, b_tr, b_wall = [], 0.0, 0, 0.0
    totals = {}
    for w0 in range(0, a.batch_sets, wave):
        ids = sids[w0:w0 + wave]
        t0 = time.perf_counter()
        rid = ctx.simulate_batch([nid] * len(ids), ids, arena_events=per * len(ids))
        st = ctx.run_stats(rid)
        b_wall += time.perf_counter() - t0
        b_ms += st.kernel_ms
        b_tr += st.total_events
        waves.append({"items": len(ids), "kernel_ms": st.kernel_ms, "transitions": st.total_events})
        ctx.release(rid)
    # the 16 distinct netlists together (one launch, records interleaved by level)
    mids = [m[0] for m in mixed]
    msids = [m[1] for m in mixed]
    rid = ctx.simulate_batch(mids, msids)
    rc, tot, ms = ctx.run_stats_raw(rid)
    while rc == gls.gls.GLS_EOVERFLOW:
        ctx.release(rid)
        rid = ctx.simulate_batch(mids, msids, arena_events=int(tot * 1.25) + (1 << 20))
        rc, tot, ms = ctx.run_stats_raw(rid)
    ctx.release(rid)
    b_ms += ms
    b_tr += tot
    waves.append({"items": len(mids), "kernel_ms": ms, "transitions": tot, "netlists": [int(x) for x in sizes]})
    # plain: every item alone, same configuration
    p_ms, p_tr = 0.0, 0
    rid = ctx.simulate(nid, sids[0], arena_events=per)
    ctx.run_stats(rid)
    ctx.release(rid)
    for sid in sids:
        rid = ctx.simulate(nid, sid, arena_events=per)
        st = ctx.run_stats(rid)
        p_ms += st.kernel_ms
        p_tr += st.total_events
        ctx.release(rid)
    for m_nid, m_sid, _, _ in mixed:
        rid = ctx.simulate(m_nid, m_sid)
        rc, tot, ms = ctx.run_stats_raw(rid)
        while rc == gls.gls.GLS_EOVERFLOW:
            ctx.release(rid)
            rid = ctx.simulate(m_nid, m_sid, arena_events=int(tot * 1.25) + (1 << 20))
            rc, tot, ms = ctx.run_stats_raw(rid)
        p_ms += ms
        p_tr += tot
        ctx.release(rid)
    ctx.close()
    line = {"metric": "batched output transitions/s (64 stimulus sets x 1M gates + 16 netlists 10k-2M gates)",
            "value": b_tr / (b_ms / 1000.0), "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "mode": "batch", "transitions": b_tr, "device_ms": b_ms, "wall_s": b_wall,
            "plain": {"value": p_tr / (p_ms / 1000.0), "unit": UNIT, "device_ms": p_ms, "transitions": p_tr},
            "speedup_vs_plain": (b_tr / b_ms) / (p_tr / p_ms), "items_match_plain": b_tr == p_tr,
            "gate_order_1m": order, "wave_size": wave, "waves": waves, "autotune": {"best": tune.best,
                                                             "trials": [[c, m] for c, m in tune.timings_ms]},
            "data": "synthetic", "dtype": "u32"}
    print(json.dumps(line))
    return 0


def run_sliced(a):
    """Task division over time.  (1) The 1M-gate workload in slices of
    --slice-ps against the same workload unsliced (same kernel, same order):
    the cost of cutting.  (2) The 1M-gate netlist under a stimulus of
    --long-window ps (64-bit times; the paper's longest re-simulation runs
    2.97e9 ps) with the recipe's 2000 transitions per PI, in 2^29 ps slices.
    Device time = the slices' gate kernels; wall = the whole call, including
    each slice's copy of its waveforms to host memory."""
    import torch
    import paper_2304_13398_gb300 as gls
    import synth
    torch.cuda.set_device(0)
    w = synth.make_workload(a.workload, seed=a.seed)
    nl, st = w.netlist, w.stimulus
    ctx = gls.Context(0)
    ctx.set_kernel(a.kernel)
    nid = ctx.load_netlist(nl)
    order = plan_from_calibration(ctx, nid, nl, w.recipe["stim"], a.seed)
    sid = ctx.load_stimulus(st)
    rid = ctx.simulate(nid, sid)
    rc, demand, _ = ctx.run_stats_raw(rid)
    arena = 0
    while rc == gls.gls.GLS_EOVERFLOW:
        ctx.release(rid)
        arena = int(demand * 1.25) + 1024
        rid = ctx.simulate(nid, sid, arena_events=arena)
        rc, demand, _ = ctx.run_stats_raw(rid)
    for _ in range(3):
        ctx.rerun(rid)
    ctx.rerun(rid)
    plain = ctx.run_stats(rid)
    ctx.release(rid)
    out = {}
    for label, stim_id, slice_ps in [("sliced_1m", sid, a.slice_ps)]:
        rid = ctx.simulate_sliced(nid, stim_id, slice_ps)
        ctx.release(rid)
        t0 = time.perf_counter()
        rid = ctx.simulate_sliced(nid, stim_id, slice_ps)
        wall = time.perf_counter() - t0
        stt = ctx.run_stats(rid)
        out[label] = {"slice_ps": slice_ps, "slices": ctx.run_slices(rid), "transitions": stt.total_events,
                      "device_ms": stt.kernel_ms, "value": stt.total_events / (stt.kernel_ms / 1000.0),
                      "wall_s": wall, "wall_value": stt.total_events / wall,
                      "equal_transitions_to_unsliced": stt.total_events == plain.total_events}
        ctx.release(rid)
    ctx.release(sid)
    sp = dict(w.recipe["stim"])
    sp["window"] = int(a.long_window)
    lst = synth.make_stimulus(nl.n_pi, seed=a.seed + 1000003, **sp)   # 64-bit times past 2^31 ps
    lid = ctx.load_stimulus64(lst)
    rid = ctx.simulate_sliced(nid, lid, 1 << 29)
    stt = ctx.run_stats(rid)
    ctx.release(rid)
    t0 = time.perf_counter()
    rid = ctx.simulate_sliced(nid, lid, 1 << 29)
    wall = time.perf_counter() - t0
    stt = ctx.run_stats(rid)
    out["long_64bit"] = {"window_ps": int(a.long_window), "slice_ps": 1 << 29, "slices": ctx.run_slices(rid),
                         "stimulus_transitions": int(lst.n_events), "transitions": stt.total_events,
                         "device_ms": stt.kernel_ms, "value": stt.total_events / (stt.kernel_ms / 1000.0),
                         "wall_s": wall, "wall_value": stt.total_events / wall}
    ctx.release(rid)
    ctx.close()
    line = {"metric": "sliced output transitions/s (task division over time, 1M gates)", "unit": UNIT,
            "mode": "sliced", "n_gpus": 1, "higher_is_better": True, "kernel": a.kernel, "gate_order": order,
            "unsliced": {"transitions": plain.total_events, "device_ms": plain.kernel_ms,
                         "value": plain.total_events / (plain.kernel_ms / 1000.0)},
            **out, "data": "synthetic", "dtype": "u32"}
    print(json.dumps(line))
    return 0


def run_cells(a):
    """General cells at the benchmark's size (the full delay matrix with its
    input-edge dimension, multi-output cells and user tables, Sec. 3): the
    workload's netlist structure with every cell a user cell drawn from a
    shared library (64 prototype tables per input count and output), 30%
    two-output cells, edge-dependent delays on half the outputs and 10% of
    the (pin, output) pairs without an arc, under the workload's stimulus.
    Gate-kernel device time (CUDA events, median of --steps reruns after 3
    warm-ups) against the built-in-cell netlist of the same structure in the
    same context, both in level order."""
    import torch
    import paper_2304_13398_gb300 as gls
    import synth
    torch.cuda.set_device(0)
    w = synth.make_workload(a.workload, seed=a.seed)
    net = w.recipe["net"]
    cn = synth.make_cell_netlist(net["n_pi"], net["n_gates"], net["depth"], seed=a.seed, fanout=net["fanout"],
                                 d_min=net["d_min"], d_max=net["d_max"], multi_frac=0.3, edge_frac=0.5,
                                 noarc_frac=0.1, x_frac=0.6, library=64)
    ctx = gls.Context(0)
    ctx.set_kernel(a.kernel)

    def timed(nid, sid):
        rid = ctx.simulate(nid, sid)
        rc, demand, _ = ctx.run_stats_raw(rid)
        while rc == gls.gls.GLS_EOVERFLOW:
            ctx.release(rid)
            rid = ctx.simulate(nid, sid, arena_events=int(demand * 1.25) + 1024)
            rc, demand, _ = ctx.run_stats_raw(rid)
        if rc != 0:
            raise gls.GlsError(rc, "cells run failed")
        for _ in range(3):
            ctx.rerun(rid)
        ms = []
        for _ in range(a.steps):
            ctx.rerun(rid)
            ms.append(ctx.run_stats(rid).kernel_ms)
        total = ctx.run_stats(rid).total_events
        ctx.release(rid)
        k_ms = statistics.median(ms)
        return {"transitions": total, "device_ms": k_ms, "value": total / (k_ms / 1000.0)}

    sid = ctx.load_stimulus(w.stimulus)
    cid = ctx.load_cell_netlist_shared(cn)
    cells = timed(cid, sid)
    ctx.release(cid)
    bid = ctx.load_netlist(w.netlist)
    builtin = timed(bid, sid)
    ctx.close()
    k = np.diff(cn.fanin_off)
    line = {"metric": "general-cell output transitions/s (1M cells: shared user tables, edge-dependent delays, "
                      "two-output cells, pins without arcs)", "unit": UNIT, "mode": "cells", "n_gpus": 1,
            "higher_is_better": True, "kernel": a.kernel, "schedule": "dependency", "gate_order": "level",
            "steps": a.steps, "warmup": 3,
            "cells": dict(cells, cells=int(cn.n_cells), output_records=int(cn.n_out.sum()),
                          two_output_cells=int((cn.n_out == 2).sum()),
                          edge_dependent_outputs="about half", no_arc_pairs="about 10% of multi-input pairs",
                          library_tables=64, mean_inputs=float(k.mean())),
            "builtin": dict(builtin, gates=int(w.netlist.n_gates)),
            "device_time_ratio": cells["device_ms"] / builtin["device_ms"],
            "config": describe(a.workload, w), "data": "synthetic", "dtype": "u32"}
    print(json.dumps(line))
    return 0


def run_serve(a):
    """Served form: a seeded Poisson request stream (200 req/s, 30 s) over 8
    resident netlists of log-uniform size (5k-5M gates), stimulus windows
    log-uniform in [1e4, 1e7] ps, 150 GB admission budget; continuous
    batching against the plain one-request-at-a-time form on the same trace."""
    import copy
    import torch
    import paper_2304_13398_gb300 as gls
    from paper_2304_13398_gb300.serve import Server, poisson_trace
    torch.cuda.set_device(0)
    ctx = gls.Context(0)
    free, _ = torch.cuda.mem_get_info()
    ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, int(min(free * 0.85, 200e9)))
    budget = int(150e9)
    rng = np.random.default_rng(a.seed + 99)
    sizes = np.exp(rng.uniform(np.log(5e3), np.log(5e6), 8)).astype(int)
    res = []
    for i, G in enumerate(sizes):
        nl, st, _, stim = make_scaled(int(G), 7000 + i)
        res.append((f"n{i}", nl, st, stim["window"]))
    out = {}
    for mode, kw in (("served", dict(batching=True, streams=4, max_batch=16, policy="sjf")),
                     ("served_fifo", dict(batching=True, streams=4, max_batch=16, policy="fifo")),
                     ("plain", dict(batching=False, streams=1, policy="fifo"))):
        srv = Server(ctx, budget_bytes=budget, **kw)
        for key, nl, st, window in res:
            srv.add_resident(key, nl, st, window)
        srv.calibrate()
        trace = poisson_trace(a.serve_seconds, a.serve_rate, [x[0] for x in res], 10_000, 10_000_000, a.seed)
        t0 = time.perf_counter()
        stt = srv.serve(trace)
        out[mode] = {"requests": stt.requests, "p50_ms": stt.p50_ms, "p99_ms": stt.p99_ms, "mean_ms": stt.mean_ms,
                     "transitions": stt.transitions, "transitions_per_s": stt.transitions_per_s,
                     "launches": stt.launches, "mean_batch": stt.mean_batch, "readmitted": stt.readmitted,
                     "wall_s": time.perf_counter() - t0}
        for key, *_ in res:
            ctx.release(srv.res[key].sid)
            ctx.release(srv.res[key].nid)
    ctx.close()
    line = {"metric": "served output transitions/s and p50/p99 latency (200 req/s, 8 resident netlists 5k-5M gates)",
            "value": out["served"]["transitions_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "mode": "serve", "served": out["served"], "served_fifo": out["served_fifo"], "plain": out["plain"],
            "netlists": [int(x) for x in sizes], "budget_bytes": budget,
            "latency": "request arrival -> its waveforms resident on the device",
            "data": "synthetic", "dtype": "u32"}
    print(json.dumps(line))
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.mode == "batch":
        return run_batch(a)
    if a.mode == "serve":
        return run_serve(a)
    if a.mode == "sliced":
        return run_sliced(a)
    if a.mode == "cells":
        return run_cells(a)
    return run_own(a)


if __name__ == "__main__":
    sys.exit(main())
