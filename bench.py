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
    ap.add_argument("--no-forms", action="store_true",
                    help="plain mode: leave out the batched and served blocks of the line")
    ap.add_argument("--forms-sets", type=int, default=8, help="batched block: stimulus sets on the 1M-gate netlist")
    ap.add_argument("--forms-netlists", type=int, default=4, help="batched block: distinct netlists")
    ap.add_argument("--forms-serve-seconds", type=float, default=10.0,
                    help="served block: length of the sustainable trace (the overload trace is half)")
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


def link_peaks(nbytes: int = 4 << 30, reps: int = 3):
    """Host<->device copy bandwidth of this machine: the best of `reps` pinned
    cudaMemcpyAsync transfers of nbytes each way (CUDA events on the copy's
    stream), GB/s.  The bound the end-to-end number is judged against."""
    import torch
    n = nbytes // 4
    h = torch.empty(n, dtype=torch.int32).pin_memory()
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = 0.0
        with torch.cuda.stream(s):
            for _ in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                dst.copy_(src, non_blocking=True)
                e1.record(s)
                e1.synchronize()
                best = max(best, nbytes / (e0.elapsed_time(e1) / 1000.0) / 1e9)
        out[name] = best
    del h, d
    out["bytes"] = nbytes
    out["how"] = f"pinned cudaMemcpyAsync of {nbytes >> 30} GiB, best of {reps} after one warm-up, CUDA events"
    return out


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
        mrid = ctx.simulate(nid, sid, arena_events=int(demand * 1.10) + (1 << 20), stream=stream)
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
        link = link_peaks()
        # lower bound of one step from the link: the stimulus in, then the
        # longer of the simulation and the results out (the kernels write the
        # results to host memory while they run)
        bound_ms = 1000.0 * (h2d / (link["h2d_gbs"] * 1e9)) + max(ms, 1000.0 * d2h / (link["d2h_gbs"] * 1e9))
        link["step_bound_ms"] = bound_ms
        link["frac"] = bound_ms / e_ms
        e2e = {"value": all_out / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "link": link,
               "timing": "host wall clock over the public calls, pinned host buffers",
               "result_path": "gls_read_host: the kernels copy every gate waveform into a pinned host "
                              "mirror as each gate finishes; the step ends when all waveforms and their descriptors are "
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
    ctx.close()
    if rank == 0 and world == 1 and not a.no_forms:
        # the batched and served forms beside the plain run (compact sizes;
        # --mode batch / --mode serve run them at full size)
        try:
            line["batched"] = batched_forms(a.forms_sets, a.forms_netlists, a.seed)
            line["batched"]["vs_plain_run"] = line["batched"]["value"] / value
        except Exception as ex:   # the headline stands without this block
            line["batched"] = {"error": f"{type(ex).__name__}: {ex}"}
        try:
            line["served"] = serve_forms(a.forms_serve_seconds, a.forms_serve_seconds / 2, a.serve_rate, a.seed)
            for tr in ("sustainable", "overload"):
                srv_b = line["served"][tr]["served"]
                srv_b["vs_plain_run"] = srv_b["transitions_per_s"] / value
        except Exception as ex:
            line["served"] = {"error": f"{type(ex).__name__}: {ex}"}
    if rank == 0:
        print(json.dumps(line))
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


def batched_forms(n_sets: int, n_netlists: int, seed: int, order: str = "planned", tune: bool = True):
    """Batched form: n_sets seeded stimulus sets (the 1M-gate recipe's
    distributions) on the 1M-gate netlist plus n_netlists netlists of
    log-uniform size (10k-2M gates) with their own stimuli, all items in one
    graph launch when they fit the device (else in waves of replicas, each one
    launch), the kernel configuration chosen by the autotuner on that launch;
    against every item simulated alone in the same configuration.  Device
    time = the gate kernels (CUDA events); returns the block for the line."""
    import torch
    import paper_2304_13398_gb300 as gls
    import synth
    from paper_2304_13398_gb300.autotune import autotune
    ctx = gls.Context(0)
    r = synth.RECIPES["ind1m"]
    nl = synth.make_netlist(seed=seed, **r["net"])
    nid = ctx.load_netlist(nl)
    note = plan_from_calibration(ctx, nid, nl, r["stim"], seed) if order == "planned" else "level"
    sids = [ctx.load_stimulus(synth.make_stimulus(nl.n_pi, seed=k, **r["stim"])) for k in range(1, n_sets + 1)]
    rng = np.random.default_rng(seed + 77)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), n_netlists)).astype(int)
    mixed = []
    for i, G in enumerate(sizes):
        mnl, mst, _, _ = make_scaled(int(G), 5000 + i)
        mixed.append((ctx.load_netlist(mnl), ctx.load_stimulus(mst)))

    def alone(nid_, sid_, arena=0):
        rid = ctx.simulate(nid_, sid_, arena_events=arena)
        rc, tot, ms = ctx.run_stats_raw(rid)
        while rc == gls.gls.GLS_EOVERFLOW:
            ctx.release(rid)
            rid = ctx.simulate(nid_, sid_, arena_events=int(tot * 1.25) + (1 << 20))
            rc, tot, ms = ctx.run_stats_raw(rid)
        if rc != 0:
            raise gls.GlsError(rc, "plain item failed")
        demand = ctx.run_info(rid)[0]
        ctx.rerun(rid)                          # timed on a warm run
        rc, tot, ms = ctx.run_stats_raw(rid)
        ctx.release(rid)
        return tot, ms, demand

    # plain: every item alone (also measures each item's arena demand)
    plain = [alone(nid, sid) for sid in sids] + [alone(m, s_) for m, s_ in mixed]
    p_tr, p_ms = sum(x[0] for x in plain), sum(x[1] for x in plain)
    per = int(max(x[2] for x in plain[:n_sets]) * 1.05) + (1 << 20)
    mixed_words = int(sum(x[2] for x in plain[n_sets:]) * 1.05) + (1 << 20)
    free, _ = torch.cuda.mem_get_info()
    fit = int((0.8 * free - 4 * mixed_words) / (4 * per + 16 * (nl.n_pi + nl.n_gates)))
    wave = max(1, min(n_sets, fit))
    launches = []
    for w0 in range(0, n_sets, wave):
        ids = sids[w0:w0 + wave]
        nets, stims, words = [nid] * len(ids), list(ids), per * len(ids)
        if w0 + wave >= n_sets:   # the distinct netlists ride with the last wave
            nets += [m for m, _ in mixed]
            stims += [s_ for _, s_ in mixed]
            words += mixed_words
        launches.append((nets, stims, words))
    tuned = None
    if tune:
        nets, stims, words = launches[-1]
        tuned = autotune(ctx, lambda: ctx.simulate_batch(nets, stims, arena_events=words))
        # the plain items again in the tuned configuration
        plain = [alone(nid, sid, per) for sid in sids] + [alone(m, s_) for m, s_ in mixed]
        p_tr, p_ms = sum(x[0] for x in plain), sum(x[1] for x in plain)
    b_tr, b_ms, waves = 0, 0.0, []
    for nets, stims, words in launches:
        rid = ctx.simulate_batch(nets, stims, arena_events=words)
        rc, tot, ms = ctx.run_stats_raw(rid)
        if rc != 0:
            raise gls.GlsError(rc, "batched launch failed")
        ctx.rerun(rid)
        rc, tot, ms = ctx.run_stats_raw(rid)
        ctx.release(rid)
        b_tr += tot
        b_ms += ms
        waves.append({"items": len(nets), "kernel_ms": ms, "transitions": tot})
    ctx.close()
    return {"items": n_sets + n_netlists, "stimulus_sets_on_1m": n_sets,
            "netlists": [int(x) for x in sizes], "launches": len(launches), "waves": waves,
            "value": b_tr / (b_ms / 1000.0), "unit": UNIT, "device_ms": b_ms, "transitions": b_tr,
            "plain": {"value": p_tr / (p_ms / 1000.0), "unit": UNIT, "device_ms": p_ms, "transitions": p_tr},
            "speedup_vs_plain": (b_tr / b_ms) / (p_tr / p_ms), "items_match_plain": b_tr == p_tr,
            "arena_words_per_1m_replica": per, "gate_order_1m": note,
            "autotune": None if tuned is None else {"best": tuned.best,
                                                    "trials": [[c, m] for c, m in tuned.timings_ms]}}


def run_batch(a):
    """Batched form at its full size (--batch-sets stimulus sets on the 1M-gate
    netlist + --batch-netlists netlists)."""
    import torch
    torch.cuda.set_device(0)
    out = batched_forms(a.batch_sets, a.batch_netlists, a.seed, a.order)
    line = {"metric": f"batched output transitions/s ({a.batch_sets} stimulus sets x 1M gates + "
                      f"{a.batch_netlists} netlists 10k-2M gates)", "value": out["value"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "mode": "batch", **out, "data": "synthetic", "dtype": "u32"}
    print(json.dumps(line))
    return 0


def run_sliced(a):
    """Task division over time.  (1) The 1M-gate workload in slices of
    --slice-ps against the same workload unsliced (same kernel, same order):
    the cost of cutting.  (2) The 1M-gate netlist under a stimulus of
    --long-window ps (64-bit times; the paper's longest re-simulation runs
    2.97e9 ps) with the recipe's 2000 transitions per PI, in 2^29 ps slices.
    Device time = the slices' gate kernels; wall = the whole call, including
    each slice's copy of its waveforms to host memory (into a pinned host
    pool sized for the larger run, pinned once before the timed calls)."""
    import torch
    import paper_2304_13398_gb300 as gls
    import synth
    torch.cuda.set_device(0)
    w = synth.make_workload(a.workload, seed=a.seed, **overrides(a))
    nl, st = w.netlist, w.stimulus
    arena = int(a.arena_words)   # 0: the library's default (profiling cases set it)
    ctx = gls.Context(0)
    ctx.set_kernel(a.kernel)
    host_pool = int(min(0.45 * mem_available_bytes(), 16 << 30))
    ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, host_pool)
    nid = ctx.load_netlist(nl)
    order = plan_from_calibration(ctx, nid, nl, w.recipe["stim"], a.seed)
    sid = ctx.load_stimulus(st)
    rid = ctx.simulate(nid, sid, arena_events=arena)
    rc, demand, _ = ctx.run_stats_raw(rid)
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
        rid = ctx.simulate_sliced(nid, stim_id, slice_ps, arena_events=arena)
        ctx.release(rid)
        t0 = time.perf_counter()
        rid = ctx.simulate_sliced(nid, stim_id, slice_ps, arena_events=arena)
        wall = time.perf_counter() - t0
        stt = ctx.run_stats(rid)
        t0 = time.perf_counter()
        off64, t64, v64 = ctx.read_all64(rid)   # every waveform, 64-bit times, in caller net order
        read_s = time.perf_counter() - t0
        del off64, t64, v64
        out[label] = {"slice_ps": slice_ps, "slices": ctx.run_slices(rid), "transitions": stt.total_events,
                      "device_ms": stt.kernel_ms, "value": stt.total_events / (stt.kernel_ms / 1000.0),
                      "wall_s": wall, "wall_value": stt.total_events / wall, "read_all64_s": read_s,
                      "equal_transitions_to_unsliced": stt.total_events == plain.total_events}
        ctx.release(rid)
    ctx.release(sid)
    if a.long_window > 0:   # 0: the workload in slices only (profiling cases)
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
            "host_pool_bytes": host_pool, "config": describe(a.workload, w),
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


SERVE_NOTE = ("latency = request arrival -> its waveforms in host memory (the kernels store every output "
              "transition into a pinned host mirror while they run; a request is done when its run has finished "
              "and its per-gate descriptors are in host memory)")


def serve_forms(seconds_sus: float, seconds_over: float, rate_over: float, seed: int, max_wait_s: float = 1.0):
    """Served form on one GPU: 8 resident netlists of log-uniform size
    (5k-5M gates, the 1M-gate recipe's distributions), requests naming one of
    them with a stimulus window log-uniform in [1e4, 1e7] ps, a 150 GB
    admission budget.  Two seeded Poisson traces: one at a rate the GPU
    sustains (half of the capacity measured by the plain form on a probe
    trace) and one at `rate_over` req/s, which overloads it.  Each trace is
    served with continuous batching (shortest job first), with shortest job
    first plus an aging bound, and in the plain form (one request per launch,
    one at a time, arrival order).  Returns the block for the JSON line."""
    import torch
    import paper_2304_13398_gb300 as gls
    from paper_2304_13398_gb300.serve import Server, poisson_trace
    ctx = gls.Context(0)
    free, _ = torch.cuda.mem_get_info()
    ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, int(min(free * 0.85, 200e9)))
    budget = int(150e9)
    rng = np.random.default_rng(seed + 99)
    sizes = np.exp(rng.uniform(np.log(5e3), np.log(5e6), 8)).astype(int)
    res = []
    for i, G in enumerate(sizes):
        nl, st, _, stim = make_scaled(int(G), 7000 + i)
        res.append((f"n{i}", nl, st, stim["window"]))
    keys = [x[0] for x in res]
    forms = {"served": dict(batching=True, streams=4, max_batch=16, policy="sjf"),
             "served_aging": dict(batching=True, streams=4, max_batch=16, policy="sjf", max_wait_s=max_wait_s),
             "plain": dict(batching=False, streams=1, policy="fifo")}
    servers = {}
    for name, kw in forms.items():   # one dispatcher per form over the same resident netlists
        srv = Server(ctx, budget_bytes=budget, **kw)
        if not servers:
            for key, nl, st, window in res:
                srv.add_resident(key, nl, st, window)
            srv.calibrate(frac=1.0)
        else:
            srv.res = next(iter(servers.values())).res
        servers[name] = srv
    del res
    # pinned host memory for the results: room for the two largest requests
    # (the mirrors of the launches in flight are admitted against it)
    big = max(Server._host_bytes(servers["served"].estimate_words(k, 10_000_000)) for k in keys)
    host_pool = int(min(0.45 * mem_available_bytes(), max(2 * big, 16 << 30)))
    t_pin = time.perf_counter()
    ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, host_pool)
    t_pin = time.perf_counter() - t_pin
    for srv in servers.values():
        srv.host_budget = host_pool

    def run(name, trace):
        t0 = time.perf_counter()
        stt = servers[name].serve(trace)
        return {"requests": stt.requests, "p50_ms": stt.p50_ms, "p99_ms": stt.p99_ms, "mean_ms": stt.mean_ms,
                "transitions": stt.transitions, "transitions_per_s": stt.transitions_per_s,
                "launches": stt.launches, "mean_batch": stt.mean_batch, "readmitted": stt.readmitted,
                "trace_s": max(q.arrival for q in trace), "wall_s": time.perf_counter() - t0}

    # capacity of the plain form (transitions/s with the results in host memory) from a short probe
    srv = servers["plain"]
    probe = poisson_trace(1.0, 20.0, keys, 10_000, 10_000_000, seed + 5)
    for q in probe:
        q.arrival = 0.0
    cap = run("plain", probe)["transitions_per_s"]
    mean_tr = float(np.mean([srv.expected_transitions(k, w) for k in keys
                             for w in np.exp(np.linspace(np.log(1e4), np.log(1e7), 64))]))
    rate_sus = max(1.0, 0.5 * cap / max(mean_tr, 1.0))
    out = {"netlists": [int(x) for x in sizes], "budget_bytes": budget, "latency": SERVE_NOTE,
           "host_pool_bytes": host_pool, "host_pool_pin_s": round(t_pin, 2),
           "plain_capacity_transitions_per_s": cap, "expected_transitions_per_request": mean_tr}
    sus = poisson_trace(seconds_sus, rate_sus, keys, 10_000, 10_000_000, seed)
    out["sustainable"] = {"rate_req_s": rate_sus, "seconds": seconds_sus,
                          "rate_rule": "half the plain form's measured capacity / expected transitions per request",
                          "served": run("served", copy_trace(sus)), "plain": run("plain", copy_trace(sus))}
    over = poisson_trace(seconds_over, rate_over, keys, 10_000, 10_000_000, seed + 1)
    out["overload"] = {"rate_req_s": rate_over, "seconds": seconds_over,
                       "served": run("served", copy_trace(over)),
                       "served_aging": dict(run("served_aging", copy_trace(over)), max_wait_s=max_wait_s),
                       "plain": run("plain", copy_trace(over))}
    for r in servers["served"].res.values():
        ctx.release(r.sid)
        ctx.release(r.nid)
    ctx.close()
    return out


def mem_available_bytes() -> int:
    """Host memory available to new allocations (/proc/meminfo)."""
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 64 << 30


def copy_trace(trace):
    from paper_2304_13398_gb300.serve import Request
    return [Request(q.rid, q.netlist, q.t_limit, q.arrival) for q in trace]


def run_serve(a):
    """Served form at the full trace length (--serve-seconds at --serve-rate
    for the overload trace; the sustainable trace runs as long)."""
    import torch
    torch.cuda.set_device(0)
    out = serve_forms(a.serve_seconds, a.serve_seconds, a.serve_rate, a.seed)
    line = {"metric": "served output transitions/s and p50/p99 latency (8 resident netlists 5k-5M gates)",
            "value": out["overload"]["served"]["transitions_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "mode": "serve", **out, "data": "synthetic", "dtype": "u32"}
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
