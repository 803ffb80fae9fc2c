"""Serving: continuous batching of simulation requests over resident netlists.

A request names a resident netlist and a stimulus window t_limit (ps): it asks
for the waveforms of that netlist under the first t_limit ps of the netlist's
resident stimulus.  The dispatcher:
  - admits waiting requests as soon as a stream slot and enough of the HBM
    budget are free, estimating each request's footprint from a per-netlist
    calibration (event-arena words per stimulus transition, measured on one
    full-window run);
  - batches waiting requests of the same netlist into one launch
    (gls_simulate_batch with per-item time limits; the netlist's gate records
    are shared, not copied) -- requests that arrive while others run are
    admitted into new launches on other streams, so their work overlaps;
  - retires finished launches with a non-blocking query, records each
    request's latency and re-admits a launch whose arena was too small with
    the measured demand.
Latency is request arrival -> its waveforms in host memory (results="host",
the default): the launches are created with the context's host mirror, so
the kernels store every output transition into pinned host memory while they
run, and a request is done once its run has finished and its per-gate
(offset, length) descriptors have been copied to the host (gls_read_host);
results="device" stops the clock when the waveforms are resident on the
device.  Device buffers come from the context's pool and host mirrors from
its pinned host pool (GLS_OPT_POOL_BYTES, GLS_OPT_HOST_POOL_BYTES), so
admitting and retiring never synchronises the device.  policy="sjf" admits the waiting request with the
least estimated work first (shortest job first: small windows do not queue
behind large ones); "fifo" admits in arrival order.  With max_wait_s, a
request that has waited longer than that is admitted before any shorter one
(oldest first), which bounds how long shortest-first can hold a large
request back.  batching=False,
streams=1, policy="fifo" gives the plain form: one request per launch, one
launch at a time, in arrival order.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import gls as _g
from .gls import Context, GlsError


@dataclass
class Request:
    rid: int
    netlist: str       # key of a resident netlist
    t_limit: int       # window: stimulus transitions before this time (ps)
    arrival: float     # seconds after the start of the trace
    t_done: float = -1.0
    out_transitions: int = 0
    attempts: int = 0
    boost: float = 1.0            # growth of its footprint estimate after arena overflows
    result: tuple | None = None   # (off, packed) when the server keeps results
    host_gates: object = None     # with results="host" and kept results: the gates' words from the mirror


@dataclass
class Resident:
    key: str
    nid: int
    sid: int
    n_nets: int
    pi_events: int
    window: int
    words_per_event: float = 0.0  # arena words per stimulus transition of the window (slope)
    words_fixed: float = 0.0      # arena words of any window (intercept: per-gate slot padding, block ends)
    out_per_event: float = 0.0    # gate-output transitions per stimulus transition (calibration run)


@dataclass
class ServeStats:
    requests: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    transitions: int
    transitions_per_s: float
    launches: int
    mean_batch: float
    readmitted: int
    latencies_ms: list = field(default_factory=list)


class Server:
    def __init__(self, ctx: Context, budget_bytes: int, max_batch: int = 16, streams: int = 4,
                 batching: bool = True, safety: float = 1.3, keep_results: bool = False, policy: str = "sjf",
                 stream_factory=None, max_wait_s: float | None = None, results: str = "host",
                 host_budget_bytes: int | None = None):
        """stream_factory() makes one launch stream (default: a new CUDA
        stream); the dispatcher only hands the streams to the context.
        results: "host" (latency ends with the waveforms in host memory) or
        "device" (resident on the device).  host_budget_bytes: with results
        "host", the pinned host memory the launches in flight may hold for
        their mirrors (the context's host pool; None: not checked)."""
        if results not in ("host", "device"):
            raise ValueError(results)
        self.results = results
        self.host_budget = host_budget_bytes
        if stream_factory is None:
            import torch
            stream_factory = torch.cuda.Stream
        self.ctx = ctx
        self.budget = int(budget_bytes)
        self.max_batch = max_batch if batching else 1
        self.safety = safety
        self.keep = keep_results
        if policy not in ("sjf", "fifo"):
            raise ValueError(policy)
        self.policy = policy
        self.max_wait_s = max_wait_s
        self.streams = [stream_factory() for _ in range(max(1, streams))]
        self.res: dict[str, Resident] = {}

    # ---- resident netlists ----
    def add_resident(self, key: str, netlist, stimulus, window: int):
        nid = self.ctx.load_netlist(netlist)
        sid = self.ctx.load_stimulus(stimulus, n_pi=netlist.n_pi)
        self.res[key] = Resident(key, nid, sid, int(netlist.n_pi + netlist.n_gates), int(stimulus.n_events),
                                 int(window))

    def calibrate(self, frac: float = 1.0, plan: bool = True, short_frac: float = 1e-3):
        """Footprint model of admission for each resident netlist: arena
        words = fixed + per_event x (stimulus transitions in the window),
        fitted to two runs, over the first short_frac and the first frac of
        the netlist's window (transitions are spread evenly over it).  The
        fixed part is the per-gate slot padding and the block ends that any
        window pays; the whole window is the default for the long run
        because nets start at X, so the first part of a window carries fewer
        output transitions per input transition than the rest.  With plan,
        the long run also plans the netlist's critical-path-first gate order
        for the dependency schedule (gls_plan_order)."""
        for r in self.res.values():
            pts = []
            for f in ((short_frac, frac) if short_frac < frac else (frac,)):
                t_limit = max(1, int(r.window * f))
                arena = 0
                while True:
                    rid = self.ctx.simulate_batch([r.nid], [r.sid], t_limits=[t_limit], arena_events=arena)
                    rc, total, _ = self.ctx.run_stats_raw(rid)
                    if rc == 0:
                        demand = self.ctx.run_info(rid)[0]
                        if f == frac:
                            r.out_per_event = total / max(1.0, r.pi_events * f)
                            if plan:
                                self.ctx.plan_order(r.nid, rid)
                    self.ctx.release(rid)
                    if rc == 0:
                        break
                    if rc != _g.GLS_EOVERFLOW:
                        raise GlsError(rc, "calibration run failed")
                    arena = int(total * 1.5) + 4096
                pts.append((r.pi_events * f, float(demand)))
            if len(pts) == 2 and pts[1][0] > pts[0][0]:
                (e1, d1), (e2, d2) = pts
                r.words_per_event = max(0.0, (d2 - d1) / (e2 - e1))
                r.words_fixed = max(0.0, d1 - r.words_per_event * e1)
            else:
                e2, d2 = pts[-1]
                r.words_per_event = max(1.0, d2 / max(1.0, e2))
                r.words_fixed = 0.0

    def estimate_words(self, key: str, t_limit: int) -> int:
        r = self.res[key]
        frac = min(1.0, max(t_limit, 1) / r.window)
        return int((r.words_fixed + r.words_per_event * r.pi_events * frac) * self.safety) + 4096

    def expected_transitions(self, key: str, t_limit: int) -> float:
        """Gate-output transitions a request is expected to produce (the
        calibration run's output per stimulus transition x the window's
        stimulus transitions)."""
        r = self.res[key]
        return r.out_per_event * r.pi_events * min(1.0, max(t_limit, 1) / r.window)

    def _footprint(self, words: int, n_items: int, n_nets: int) -> int:
        return 4 * words + n_items * n_nets * 16 + (1 << 20)

    @staticmethod
    def _host_bytes(words: int) -> int:
        """Pinned host mirror of an arena of `words` (its padding, rounded up)."""
        return ((4 * (words + 64)) + 255) & ~255

    # ---- serving ----
    def serve(self, requests: list[Request]) -> ServeStats:
        ctx = self.ctx
        host = self.results == "host"
        if host:
            ctx.set_option(_g.GLS_OPT_HOST_MIRROR, 1)
            gmax = max(r.n_nets for r in self.res.values())
            goff_buf, glen_buf = _pinned(gmax, np.int64), _pinned(gmax, np.uint32)
        try:
            return self._serve(requests, host, goff_buf if host else None, glen_buf if host else None)
        finally:
            if host:
                ctx.set_option(_g.GLS_OPT_HOST_MIRROR, 0)

    def _serve(self, requests: list[Request], host: bool, goff_buf, glen_buf) -> ServeStats:
        ctx = self.ctx
        pending: deque[Request] = deque()
        lock = threading.Lock()
        t0 = time.perf_counter() + 0.05
        done_arriving = threading.Event()

        def arrivals():
            for q in sorted(requests, key=lambda x: x.arrival):
                dt = t0 + q.arrival - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                with lock:
                    pending.append(q)
            done_arriving.set()

        th = threading.Thread(target=arrivals, daemon=True)
        th.start()
        inflight = []            # (run_id, reqs, stream index, device bytes, words, host bytes)
        free_streams = list(range(len(self.streams)))
        used = used_host = 0
        launches, items, readmitted = 0, 0, 0
        while True:
            progressed = False
            # retire finished launches
            for entry in list(inflight):
                rid, reqs, si, nbytes, words, hbytes = entry
                if not ctx.run_done(rid):
                    continue
                rc, total, _ = ctx.run_stats_raw(rid)
                now = time.perf_counter()
                if rc == _g.GLS_EOVERFLOW:
                    # the estimate was too small for these requests: grow theirs and re-admit
                    grow = max(2.0, 1.2 * total / max(1, words))
                    with lock:
                        for q in reversed(reqs):
                            q.attempts += 1
                            q.boost *= grow
                            pending.appendleft(q)
                    readmitted += len(reqs)
                elif rc != 0:
                    raise GlsError(rc, ctx.lib.gls_last_error(ctx.h).decode())
                else:
                    # the launch's gate transitions, shared among its requests
                    share, rem = divmod(total, len(reqs))
                    for i, q in enumerate(reqs):
                        if host:   # descriptors to host memory: the waveforms are already there
                            arena, goff, glen = ctx.read_host(rid, i, goff_buf, glen_buf)
                            now = time.perf_counter()
                            if self.keep:
                                q.host_gates = np.concatenate(
                                    [arena[o:o + n] for o, n in zip(goff.tolist(), glen.tolist())] or
                                    [np.zeros(0, np.uint32)])
                        q.t_done = now - t0
                        q.out_transitions = share + (rem if i == 0 else 0)
                        if self.keep:
                            q.result = ctx.read_item(rid, i)
                ctx.release(rid)
                inflight.remove(entry)
                free_streams.append(si)
                used -= nbytes
                used_host -= hbytes
                progressed = True
            # admit waiting requests
            while free_streams:
                with lock:
                    if not pending:
                        break
                    now_s = time.perf_counter() - t0
                    overdue = [] if self.max_wait_s is None else \
                        [q for q in pending if now_s - q.arrival > self.max_wait_s]
                    if overdue:
                        head = min(overdue, key=lambda q: q.arrival)
                    elif self.policy == "sjf":
                        head = min(pending, key=lambda q: self.estimate_words(q.netlist, q.t_limit))
                    else:
                        head = pending[0]
                    group = [head]
                    if self.max_batch > 1:
                        for q in list(pending):
                            if len(group) >= self.max_batch:
                                break
                            if q is not head and q.netlist == head.netlist:
                                group.append(q)
                r = self.res[head.netlist]
                words = [int(self.estimate_words(q.netlist, q.t_limit) * q.boost) for q in group]
                hb = self.host_budget if host and self.host_budget is not None else None
                while len(group) > 1 and (used + self._footprint(sum(words), len(group), r.n_nets) > self.budget or
                                          (hb is not None and used_host + self._host_bytes(sum(words)) > hb)):
                    group.pop()
                    words.pop()
                need = self._footprint(sum(words), len(group), r.n_nets)
                need_host = self._host_bytes(sum(words)) if host else 0
                if hb is not None and need_host > hb:
                    raise GlsError(_g.GLS_ENOMEM, f"request {head.rid} needs a {need_host}-byte host mirror, "
                                                  f"beyond the {hb}-byte host budget")
                if (used + need > self.budget or (hb is not None and used_host + need_host > hb)) and inflight:
                    break       # wait for memory
                si = free_streams.pop()
                with lock:
                    for q in group:
                        pending.remove(q)
                try:
                    rid = ctx.simulate_batch([r.nid] * len(group), [r.sid] * len(group),
                                             t_limits=[q.t_limit for q in group], arena_events=sum(words),
                                             stream=self.streams[si])
                except GlsError:
                    free_streams.append(si)
                    with lock:
                        for q in reversed(group):
                            pending.appendleft(q)
                    if not inflight:
                        raise
                    break
                inflight.append((rid, group, si, need, sum(words), need_host))
                used += need
                used_host += need_host
                launches += 1
                items += len(group)
                progressed = True
            with lock:
                idle = not pending
            if done_arriving.is_set() and idle and not inflight:
                break
            if not progressed:
                time.sleep(50e-6)
        th.join()
        lat = np.array([(q.t_done - q.arrival) * 1000.0 for q in requests])
        wall = max(q.t_done for q in requests) - min(q.arrival for q in requests)
        tr = int(sum(q.out_transitions for q in requests))
        return ServeStats(len(requests), wall, float(np.percentile(lat, 50)), float(np.percentile(lat, 99)),
                          float(lat.mean()), tr, tr / max(wall, 1e-9), launches, items / max(1, launches),
                          readmitted, lat.tolist())


def _pinned(n: int, dtype):
    """A page-locked host array of n elements (for the descriptor copies)."""
    try:
        import torch
        if torch.cuda.is_available():
            t = torch.empty(max(n, 1) * np.dtype(dtype).itemsize, dtype=torch.uint8).pin_memory()
            return t.numpy().view(dtype)
    except ImportError:
        pass
    return np.zeros(max(n, 1), dtype)


def poisson_trace(n_seconds: float, rate: float, keys: list[str], wmin: int, wmax: int, seed: int) -> list[Request]:
    """Seeded request stream: Poisson arrivals, a uniformly chosen resident
    netlist, a window log-uniform in [wmin, wmax] ps."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= n_seconds:
            break
        w = int(np.exp(rng.uniform(np.log(wmin), np.log(wmax))))
        out.append(Request(len(out), keys[int(rng.integers(0, len(keys)))], w, t))
    return out
