"""Host logic of the serving dispatcher and the autotuner, on the CPU.

A fake context stands in for the library: launches complete after a set
number of polls, and an item's arena demand is a fixed number of words per
picosecond of its window, so admission, batching, the shortest-job-first
policy, the HBM budget and re-admission after an arena overflow can be
checked without a GPU (the served form on the GPU, with results compared to
the oracle, is in test_gpu_serve.py).
"""
import itertools

import numpy as np

from paper_2304_13398_gb300 import autotune
from paper_2304_13398_gb300 import gls as G
from paper_2304_13398_gb300.serve import Request, Server


class FakeCtx:
    def __init__(self, words_per_ps, polls=3, demand_scale=1.0):
        self.wpp = dict(words_per_ps)     # netlist id -> arena words per ps of window
        self.polls = polls
        self.scale = demand_scale          # demand at serve time / demand at calibration
        self.calibrating = True
        self.ids = itertools.count(1)
        self.runs = {}
        self.launches = []                 # (netlist ids, t_limits, arena words) in launch order
        self.planned = []
        self.options = {}
        self.mirror_set = []               # GLS_OPT_HOST_MIRROR values in the order set
        self.host_reads = []               # (run id, item) of every gls_read_host

    def demand(self, items):
        sc = 1.0 if self.calibrating else self.scale
        return int(sum(self.wpp[n] * t for n, t in items) * sc)

    def load_netlist(self, nl):
        return nl.nid

    def load_stimulus(self, st, n_pi=None):
        return next(self.ids)

    def simulate_batch(self, nids, sids, t_limits=None, arena_events=0, stream=None):
        rid = next(self.ids)
        items = list(zip(nids, t_limits))
        self.runs[rid] = {"items": items, "arena": arena_events, "polls": self.polls,
                          "demand": self.demand(items)}
        if not self.calibrating:
            self.launches.append(([n for n, _ in items], [t for _, t in items], arena_events))
        return rid

    def run_done(self, rid):
        r = self.runs[rid]
        r["polls"] -= 1
        return r["polls"] <= 0

    def run_stats_raw(self, rid):
        r = self.runs[rid]
        if r["arena"] and r["arena"] < r["demand"]:
            return G.GLS_EOVERFLOW, r["demand"], 0.0
        return G.GLS_OK, r["demand"], 0.0

    def run_info(self, rid):
        r = self.runs[rid]
        return r["demand"], r["arena"]

    def plan_order(self, nid, rid=-1, item=0):
        self.planned.append(nid)

    def set_option(self, option, value):
        self.options[option] = value
        if option == G.GLS_OPT_HOST_MIRROR:
            self.mirror_set.append(value)

    def read_host(self, rid, item=0, gate_off=None, gate_len=None):
        assert self.options.get(G.GLS_OPT_HOST_MIRROR) == 1, "results read from a run without a host mirror"
        self.host_reads.append((rid, item))
        return np.zeros(1, np.uint32), np.zeros(0, np.int64), np.zeros(0, np.uint32)

    def release(self, rid):
        self.runs.pop(rid, None)


class Net:
    def __init__(self, nid, n_pi=4, n_gates=100):
        self.nid, self.n_pi, self.n_gates = nid, n_pi, n_gates


class Stim:
    n_events = 1000


def make_server(ctx, nets, window=10_000, **kw):
    srv = Server(ctx, stream_factory=object, **kw)
    for n in nets:
        srv.add_resident(f"n{n}", Net(n), Stim(), window)
    srv.calibrate()
    ctx.calibrating = False
    return srv


def test_calibration_fits_the_footprint_model_and_plans_orders():
    ctx = FakeCtx({1: 2.0, 2: 0.5})
    srv = make_server(ctx, [1, 2], budget_bytes=1 << 40)
    assert sorted(ctx.planned) == [1, 2]
    # the fake's demand is proportional to the window: the two-point fit finds
    # no fixed part, and the estimate is the demand with the safety factor
    for nid, wpp in ((1, 2.0), (2, 0.5)):
        assert abs(srv.res[f"n{nid}"].words_fixed) < 1e-6
        est = srv.estimate_words(f"n{nid}", 10_000)
        assert abs(est - (int(wpp * 10_000 * srv.safety) + 4096)) <= 1


def test_plain_form_is_fifo_one_request_per_launch():
    ctx = FakeCtx({1: 1.0})
    srv = make_server(ctx, [1], budget_bytes=1 << 40, batching=False, streams=1, policy="fifo")
    reqs = [Request(i, "n1", w, 0.0005 * i) for i, w in enumerate([900, 100, 500, 300, 700])]
    st = srv.serve(reqs)
    assert st.launches == 5 and st.mean_batch == 1.0
    assert [l[1] for l in ctx.launches] == [[900], [100], [500], [300], [700]]
    assert all(q.t_done >= q.arrival for q in reqs)
    # latency ends with the results in host memory: one descriptor read per
    # request, from runs created with the host mirror, which is off again after
    assert len(ctx.host_reads) == 5 and ctx.mirror_set == [1, 0]


def test_device_results_skip_the_host_read():
    ctx = FakeCtx({1: 1.0})
    srv = make_server(ctx, [1], budget_bytes=1 << 40, batching=False, streams=1, policy="fifo", results="device")
    st = srv.serve([Request(i, "n1", 500, 0.0005 * i) for i in range(3)])
    assert st.requests == 3 and ctx.host_reads == [] and ctx.mirror_set == []


def test_shortest_job_first():
    # the first launch keeps the single stream busy while the rest arrive
    ctx = FakeCtx({1: 1.0}, polls=400)
    srv = make_server(ctx, [1], budget_bytes=1 << 40, batching=False, streams=1, policy="sjf")
    windows = [5000, 9000, 100, 3000, 700, 6000]
    reqs = [Request(0, "n1", windows[0], 0.0)] + [Request(i, "n1", w, 0.001) for i, w in enumerate(windows) if i]
    srv.serve(reqs)
    order = [l[1][0] for l in ctx.launches]
    # in arrival order the rest would start with 9000; shortest first sorts them
    # (all six sorted if the dispatcher first looked after every arrival)
    assert order[1:] == sorted(windows[1:]) if order[0] == 5000 else order == sorted(windows)


def test_aging_bounds_how_long_shortest_first_holds_a_large_request():
    def order(max_wait_s):
        ctx = FakeCtx({1: 1.0}, polls=2000)  # each launch holds the one stream for >= 100 ms
        srv = make_server(ctx, [1], budget_bytes=1 << 40, batching=False, streams=1, policy="sjf",
                          max_wait_s=max_wait_s)
        reqs = [Request(0, "n1", 5000, 0.0), Request(1, "n1", 9000, 0.001)]
        reqs += [Request(2 + i, "n1", 100 + i, 0.0015 + 0.0001 * i) for i in range(4)]
        srv.serve(reqs)
        return [l[1][0] for l in ctx.launches]

    assert order(None)[-1] == 9000            # pure shortest-first: the large request goes last
    aged = order(0.005)                       # waited past 5 ms: oldest first
    assert aged[:2] == [5000, 9000] and aged[2:] == [100, 101, 102, 103]


def test_batches_hold_one_netlist_and_respect_max_batch():
    ctx = FakeCtx({1: 1.0, 2: 1.0}, polls=50)
    srv = make_server(ctx, [1, 2], budget_bytes=1 << 40, max_batch=3, streams=2)
    reqs = [Request(i, f"n{1 + i % 2}", 100 + 10 * i, 0.0) for i in range(14)]
    st = srv.serve(reqs)
    assert sum(len(l[0]) for l in ctx.launches) == 14
    for nids, _, _ in ctx.launches:
        assert len(set(nids)) == 1 and 1 <= len(nids) <= 3
    assert st.mean_batch > 1.0
    assert all(q.t_done > 0 for q in reqs)


def test_admission_stays_within_the_budget():
    ctx = FakeCtx({1: 400.0}, polls=20)   # ~10 MB of arena per request: the arena dominates
    srv = make_server(ctx, [1], budget_bytes=0, max_batch=4, streams=4)
    one = srv._footprint(srv.estimate_words("n1", 5000), 1, 104)
    srv.budget = int(2.5 * one)        # room for two requests at a time, in one launch or two
    peak, peak_items = [0], [0]
    real_simulate = ctx.simulate_batch

    def simulate(nids, sids, t_limits=None, arena_events=0, stream=None):
        rid = real_simulate(nids, sids, t_limits, arena_events, stream)
        live = [r for r in ctx.runs.values() if r["polls"] > 0]
        peak[0] = max(peak[0], sum(srv._footprint(r["arena"], len(r["items"]), 104) for r in live))
        peak_items[0] = max(peak_items[0], sum(len(r["items"]) for r in live))
        return rid

    ctx.simulate_batch = simulate
    reqs = [Request(i, "n1", 5000, 0.0) for i in range(8)]
    st = srv.serve(reqs)
    assert st.requests == 8 and all(q.t_done > 0 for q in reqs)
    assert peak[0] <= srv.budget
    assert peak_items[0] == 2


def test_overflow_is_readmitted_with_a_larger_estimate():
    ctx = FakeCtx({1: 10.0}, polls=2, demand_scale=5.0)   # serve-time demand 5x the calibrated one
    srv = make_server(ctx, [1], budget_bytes=1 << 40, max_batch=1, streams=1)
    reqs = [Request(i, "n1", 2000, 0.0) for i in range(3)]
    st = srv.serve(reqs)
    assert st.readmitted >= 1
    assert all(q.t_done > 0 and q.out_transitions > 0 for q in reqs)
    # the last launch had room for the real demand
    assert ctx.launches[0][2] < ctx.demand([(1, 2000)]) <= ctx.launches[-1][2]
    assert any(q.attempts > 0 for q in reqs)


class TuneCtx:
    """Times by configuration; records what is applied."""
    def __init__(self, ms):
        self.ms = ms
        self.kernel, self.opts = None, {}
        self.ids = itertools.count(1)

    def set_kernel(self, k):
        self.kernel = k

    def set_option(self, opt, v):
        self.opts[opt] = v

    def key(self):
        return (self.kernel, self.opts.get(G.GLS_OPT_WARPS_PER_CTA), self.opts.get(G.GLS_OPT_SEGMENT))

    def rerun(self, rid):
        pass

    def run_stats(self, rid):
        return G.RunStats(1, self.ms.get(self.key(), 99.0))

    def release(self, rid):
        pass


def test_autotune_leaves_the_fastest_candidate_applied():
    ms = {("wide", 4, None): 3.0, ("wide", 2, None): 2.5, ("windowed", 4, None): 4.0,
          ("windowed", 2, None): 4.5, ("segmented", 4, 32): 9.0, ("segmented", 4, 128): 8.0}
    ctx = TuneCtx(ms)
    built = []
    res = autotune.autotune(ctx, lambda: built.append(1) or len(built))
    assert res.best == {"kernel": "wide", "warps_per_cta": 2}
    assert ctx.key()[:2] == ("wide", 2)
    assert len(built) == len(autotune.DEFAULT_CANDIDATES) == len(res.timings_ms)


def test_host_mirror_budget_limits_launches_in_flight():
    # each request's mirror takes about 4 * (1000 * 1.3 + 4096) bytes; a host
    # budget for one and a half of them keeps one launch in flight at a time
    ctx = FakeCtx({1: 0.1}, polls=50)
    one = Server._host_bytes(int(0.1 * 10_000 * 1.3) + 4096)
    srv = make_server(ctx, [1], budget_bytes=1 << 40, batching=False, streams=4, policy="fifo",
                      host_budget_bytes=int(1.5 * one))
    seen = []
    orig = ctx.simulate_batch

    def counting(*a, **k):
        seen.append(sum(1 for r in ctx.runs.values() if r["polls"] > 0))
        return orig(*a, **k)
    ctx.simulate_batch = counting
    st = srv.serve([Request(i, "n1", 10_000, 0.0) for i in range(4)])
    assert st.launches == 4 and max(seen) == 0, "a second mirror was admitted beyond the host budget"
    # a request whose mirror alone exceeds the budget is refused with a clear error
    srv.host_budget = one // 2
    import pytest
    with pytest.raises(G.GlsError) as ei:
        srv.serve([Request(0, "n1", 10_000, 0.0)])
    assert ei.value.code == G.GLS_ENOMEM


def test_footprint_model_has_a_fixed_part():
    # demand = 50,000 words of any window (slot padding, block ends) + 2 words per ps
    class FixedCtx(FakeCtx):
        def demand(self, items):
            sc = 1.0 if self.calibrating else self.scale
            return int(sum(50_000 + self.wpp[n] * t for n, t in items) * sc)
    ctx = FixedCtx({1: 2.0})
    srv = make_server(ctx, [1], budget_bytes=1 << 40)
    r = srv.res["n1"]
    assert abs(r.words_fixed - 50_000) <= 2 and abs(r.words_per_event - 20.0) < 0.01
    # a short window is estimated above its demand (a purely proportional
    # model would give it about 2% of it), a long one too
    for t in (10, 1_000, 10_000):
        assert srv.estimate_words("n1", t) >= ctx.demand([(1, t)])
    # served without overflow
    st = srv.serve([Request(i, "n1", t, 0.0) for i, t in enumerate((10, 100, 5_000, 10_000))])
    assert st.readmitted == 0 and st.requests == 4
