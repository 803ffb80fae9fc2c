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
    ap.add_argument("--workload", default="ind1m")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-frac", type=float, default=0.005,
                    help="time-window fraction of the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--gates", type=int, default=0, help="override the recipe's gate count (profiling cases)")
    ap.add_argument("--pis", type=int, default=0, help="override the recipe's primary-input count")
    ap.add_argument("--arena-words", type=int, default=0, help="event arena size (0: size from a first run)")
    ap.add_argument("--schedule", default="dependency", choices=["dependency", "levels"])
    ap.add_argument("--warps-per-cta", type=int, default=0)
    ap.add_argument("--kernel", default="windowed", choices=["windowed", "wide", "segmented"])
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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

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
        for ln in self.lines:
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


def ncu_traffic(workload: str):
    """DRAM bytes per run of the level kernel from a committed ncu summary,
    valid only while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "gate_kernel_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_source_sha") != kernel_source_sha():
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


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    w = synth.make_workload(a.workload, seed=a.seed, **overrides(a))
    cfg = describe(a.workload, w)
    for _ in range(a.warmup):
        cpu_baseline(a.workload, a.seed, a.cpu_frac / 4)
    vals, secs = [], []
    for _ in range(a.steps):
        b = cpu_baseline(a.workload, a.seed, a.cpu_frac)
        vals.append(b["value"])
        secs.append(b["seconds"])
    v = statistics.median(vals)
    cb = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": b["sample"], "cpu": cpu_model()}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * statistics.median(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
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
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * e_out / (ms / 1000.0)

    e2e = None
    if not a.no_e2e:
        N = nl.n_pi + nl.n_gates
        off_h = torch.from_numpy(st.off).pin_memory()
        t_h = torch.from_numpy(st.t).pin_memory()
        v_h = torch.from_numpy(st.v).pin_memory()
        total = int(off[-1])
        roff = torch.empty(N + 1, dtype=torch.int64).pin_memory()
        rpk = torch.empty(total, dtype=torch.int32).pin_memory()
        h2d = 8 * (nl.n_pi + 1) + 5 * st.n_events
        d2h = 8 * (N + 1) + 4 * total
        def e2e_step():
            ctx.update_stimulus(sid, off_h, t_h, v_h)
            ctx.rerun(rid, stream)
            ctx.run_stats(rid)
            ctx.read_all(rid, roff, rpk)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1000 / a.e2e_steps
        if world > 1:
            t = torch.tensor([e_ms], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": world * e_out / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
               "timing": "host wall clock over the public calls, pinned host buffers"}

    peak, peak_kind = measured_peak_gbs()
    achieved = alg_bytes / (k_ms / 1000.0) / 1e9
    traffic = ncu_traffic(a.workload)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind,
            "kernel": (f"dependency_kernel<{a.kernel}> (one launch per run)" if a.schedule == "dependency"
                       else f"level_kernel<{a.kernel}> (all levels of one run)"),
            "algorithmic_bytes_per_run": alg_bytes, "kernel_ms_per_run": k_ms}
    cb = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cb = cpu_baseline(a.workload, a.seed, a.cpu_frac)
        cb["cpu"] = cpu_model()
    cfg = describe(a.workload, w)
    cfg.update({"output_transitions_per_step": e_out, "arena_words": int(arena) if arena else "default",
                "l2_policy": "inputs larger than L2 (stimulus and intermediate waveforms >> 129 MB)",
                "parallelism": f"replicas{world}" if world > 1 else "single", "schedule": a.schedule, "kernel": a.kernel})
    launches_per_step = 1 + (1 if a.schedule == "dependency" else int(w.recipe["net"]["depth"]))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": max(a.warmup, 3), "ms_per_step": ms, "sim_time_ms": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 packed events (int32 time, 2-bit value)",
            "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": launches_per_step * a.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_own(a)


if __name__ == "__main__":
    sys.exit(main())
