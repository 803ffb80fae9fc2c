"""GPU parity of task division over time (sliced runs): the concatenated
slices equal the CPU oracle's unsliced waveforms transition by transition --
for slices shorter than a gate delay, around the delays, and longer than the
whole stimulus; on 64-bit times past 2^32 ps; with an arena too small for a
slice (re-evaluated with a larger one); and after a rerun; in a planned
gate order; and at 20,000 gates of the benchmark recipe's shape."""
import os

import numpy as np
import pytest

import bench
import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def case(seed=31, n_gates=1500, depth=12):
    nl = synth.make_netlist(16, n_gates, depth, fanout="pareto", d_min=5, d_max=200, seed=seed, shuffle=True)
    st = synth.make_stimulus(16, mean=90, window=40_000, seed=seed + 1)
    return nl, st


def shifted(st, D):
    return synth.Stimulus(st.off.copy(), st.t.astype(np.int64) + D, st.v.copy())


@pytest.mark.parametrize("kernel,schedule", [("windowed", "dependency"), ("windowed", "levels"),
                                             ("wide", "dependency")])
@pytest.mark.parametrize("slice_ps", [61, 700, 9_000, 10**6])
def test_sliced_equals_oracle(kernel, schedule, slice_ps):
    nl, st = case()
    ref = oracle.sim_event(nl, st)
    with gls.Context(0) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_schedule(schedule)
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate_sliced(nid, sid, slice_ps)
        assert ctx.run_slices(rid) == int(st.t.max()) // slice_ps + 1
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, f"slice {slice_ps}")
        assert ctx.run_stats(rid).total_events == int(ref.off[-1] - ref.off[nl.n_pi])
        tw, vw = ctx.read_waveform64(rid, nl.n_pi + 7)
        a, b = ref.off[nl.n_pi + 7], ref.off[nl.n_pi + 8]
        np.testing.assert_array_equal(tw, ref.t[a:b])
        np.testing.assert_array_equal(vw, ref.v[a:b])


def test_64bit_times_and_rerun():
    nl, st = case(seed=41)
    D = 3 * (1 << 31) + 12345
    st64 = shifted(st, D)
    ref = oracle.sim_event(nl, st64)
    assert ref.t.max() > (1 << 32)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus64(st64)
        rid = ctx.simulate_sliced(nid, sid, 1 << 28)
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, "64-bit times")
        ctx.rerun(rid)
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, "64-bit rerun")
        with pytest.raises(gls.GlsError):
            ctx.simulate(nid, sid)          # 64-bit stimulus: sliced runs only
        with pytest.raises(gls.GlsError):
            ctx.read_all(rid)               # sliced run: 64-bit reads only


def test_bursts_spread_over_seconds_of_simulated_time():
    """Activity in bursts billions of ps apart: most slices are empty, gate
    state crosses long idle stretches."""
    nl, _ = case(seed=51, n_gates=800, depth=10)
    parts = [synth.make_stimulus(16, mean=25, window=6_000, seed=60 + k) for k in range(4)]
    starts = [0, 1_500_000_000, 2_900_000_000, 5_000_000_123]
    off = np.zeros(17, np.int64)
    ts, vs = [], []
    for i in range(16):
        ti, vi = [], []
        last = None
        for p, T in zip(parts, starts):
            a, b = p.off[i], p.off[i + 1]
            for tt, vv in zip(p.t[a:b], p.v[a:b]):
                if last is not None and vv == last:
                    continue
                ti.append(int(tt) + T)
                vi.append(int(vv))
                last = vv
        ts += ti
        vs += vi
        off[i + 1] = off[i] + len(ti)
    st = synth.Stimulus(off, np.array(ts, np.int64), np.array(vs, np.uint8))
    ref = oracle.sim_event(nl, st)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus64(st)
        rid = ctx.simulate_sliced(nid, sid, 1 << 29)
        off2, t, v = ctx.read_all64(rid)
        assert_same(ref, off2, t, v, "bursts")


def test_small_arena_is_grown_per_slice():
    nl, st = case(seed=71)
    ref = oracle.sim_event(nl, st)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate_sliced(nid, sid, 5_000, arena_events=2_000)
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, "grown arena")
        demand, cap = ctx.run_info(rid)
        assert cap >= demand > 2_000


def test_sliced_rejections():
    nl, st = case(seed=81, n_gates=200, depth=6)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        ctx.set_kernel("segmented")
        with pytest.raises(gls.GlsError):
            ctx.simulate_sliced(nid, sid, 1000)
        ctx.set_kernel("windowed")
        with pytest.raises(gls.GlsError):
            ctx.simulate_sliced(nid, sid, (1 << 30) - 10)   # slice + longest path reaches 2^30
        with pytest.raises(gls.GlsError):
            ctx.simulate_sliced(nid, sid, 0)


@pytest.mark.parametrize("slice_ps", [61, 2_000])
def test_sliced_planned_order_equals_oracle(slice_ps):
    """The slices of a launch in a planned (critical-path-first) gate order,
    as the benchmark runs them; then a rerun of the same run."""
    nl, st = case(seed=91)
    ref = oracle.sim_event(nl, st)
    with gls.Context(0) as ctx:
        ctx.set_kernel("wide")
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate(nid, sid)
        ctx.run_stats(rid)
        ctx.plan_order(nid, rid)
        ctx.release(rid)
        rid = ctx.simulate_sliced(nid, sid, slice_ps)
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, f"planned, slice {slice_ps}")
        ctx.rerun(rid)
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, f"planned rerun, slice {slice_ps}")


def test_sliced_mid_size_industrial_shape():
    """20,000 gates of the 1M-gate recipe's distributions (depth 26, 400 PIs
    at 2,000 transitions each over 1e7 ps) in ten 1e6 ps slices, all in one
    launch, planned order: every waveform against the levelized oracle."""
    nl, st, net, stim = bench.make_scaled(20_000, 5)
    ref = oracle.sim_levelized(nl, st, nthreads=os.cpu_count() or 1)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        bench.plan_from_calibration(ctx, nid, nl, stim, 5)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate_sliced(nid, sid, 1_000_000)
        assert ctx.run_slices(rid) == int(st.t.max()) // 1_000_000 + 1
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, "20k gates, 1e6 ps slices")
        assert ctx.run_stats(rid).total_events == int(ref.off[-1] - ref.off[nl.n_pi])


@pytest.mark.parametrize("group", [1, 2, 3, 5, 64])
def test_slice_groups_equal_oracle(group):
    """Launches of 1, 2, 3, 5 and up to 64 slices each: 700 ps slices of the
    40,000 ps stimulus make 58 slices, so groups of 3 and 5 end with a
    ragged launch, and odd and even group sizes hand the state buffers on
    differently."""
    nl, st = case(seed=101)
    ref = oracle.sim_event(nl, st)
    with gls.Context(0) as ctx:
        ctx.set_option(gls.gls.GLS_OPT_SLICE_GROUP, group)
        ctx.set_kernel("wide")
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate_sliced(nid, sid, 700)
        assert ctx.run_slices(rid) == int(st.t.max()) // 700 + 1
        off, t, v = ctx.read_all64(rid)
        assert_same(ref, off, t, v, f"groups of {group}")
        assert ctx.run_stats(rid).total_events == int(ref.off[-1] - ref.off[nl.n_pi])


def test_slice_group_option_range():
    with gls.Context(0) as ctx:
        for bad in (0, 65, -1):
            with pytest.raises(gls.GlsError):
                ctx.set_option(gls.gls.GLS_OPT_SLICE_GROUP, bad)


def test_sliced_bounded_wait_reports_timeout():
    """A gate that never signals completion in a launch over several slices:
    its readers give up after the wait limit, the call returns GLS_ETIMEOUT,
    and the context stays usable."""
    E = gls.gls
    w = synth.make_workload("tiny200", seed=3)
    nl, st = w.netlist, w.stimulus
    with gls.Context(0) as c:
        c.set_option(E.GLS_OPT_WAIT_LIMIT_MS, 50)
        c.set_option(E.GLS_OPT_TEST_WITHHOLD_GATE, 0)   # first gate of level 1 has readers
        nid = c.load_netlist(nl)
        sid = c.load_stimulus(st)
        with pytest.raises(gls.GlsError) as ei:
            c.simulate_sliced(nid, sid, 20_000)
        assert ei.value.code == E.GLS_ETIMEOUT
        c.set_option(E.GLS_OPT_TEST_WITHHOLD_GATE, -1)
        rid = c.simulate_sliced(nid, sid, 20_000)
        assert c.run_slices(rid) > 1
        off, t, v = c.read_all64(rid)
        assert_same(oracle.sim_event(nl, st), off, t, v, "sliced after timeout")


def test_sliced_results_in_the_pinned_host_pool():
    """With a pinned host pool the slices' waveforms are carved from it; the
    pool cannot be dropped while the run holds blocks, and can once the run
    is released.  A pool too small for a slice falls back to ordinary host
    memory."""
    nl, st = case(seed=121)
    ref = oracle.sim_event(nl, st)
    E = gls.gls
    with gls.Context(0) as ctx:
        ctx.set_kernel("wide")
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        for pool in (64 << 20, 4096):
            ctx.set_option(E.GLS_OPT_HOST_POOL_BYTES, pool)
            rid = ctx.simulate_sliced(nid, sid, 3_000)
            off, t, v = ctx.read_all64(rid)
            assert_same(ref, off, t, v, f"host pool of {pool} bytes")
            ctx.rerun(rid)                      # the slices' blocks are given back and taken again
            off, t, v = ctx.read_all64(rid)
            assert_same(ref, off, t, v, f"host pool of {pool} bytes, rerun")
            if pool > 4096:
                with pytest.raises(gls.GlsError):
                    ctx.set_option(E.GLS_OPT_HOST_POOL_BYTES, 0)   # blocks in use
            ctx.release(rid)
            ctx.set_option(E.GLS_OPT_HOST_POOL_BYTES, 0)
