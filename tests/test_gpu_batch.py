"""GPU parity of batched runs: every item of one batched launch equals the
CPU oracle (and the single-item run) transition by transition."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def items():
    out = []
    base = synth.make_netlist(12, 400, 10, fanout="pareto", d_min=5, d_max=200, seed=21)
    for s in range(5):   # several stimulus sets on one netlist
        out.append((base, synth.make_stimulus(12, mean=150 + 40 * s, window=50_000, seed=100 + s)))
    for s in range(4):   # distinct netlists of uneven size and depth
        nl = synth.make_netlist(4 + 3 * s, 30 + 250 * s, 3 + 4 * s, d_min=1, d_max=120, seed=40 + s,
                                shuffle=bool(s % 2))
        out.append((nl, synth.make_stimulus(nl.n_pi, mean=80, window=20_000, seed=200 + s)))
    return out


@pytest.mark.parametrize("kernel,schedule", [("windowed", "dependency"), ("windowed", "levels"),
                                             ("wide", "dependency"), ("segmented", "dependency")])
def test_batch_items_equal_oracle(kernel, schedule):
    its = items()
    refs = [oracle.sim_event(nl, st) for nl, st in its]
    with gls.Context(0) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_schedule(schedule)
        nid_of = {}
        nids, sids = [], []
        for nl, st in its:
            if id(nl) not in nid_of:
                nid_of[id(nl)] = ctx.load_netlist(nl)
            nids.append(nid_of[id(nl)])
            sids.append(ctx.load_stimulus(st, n_pi=nl.n_pi))
        rid = ctx.simulate_batch(nids, sids)
        stats = ctx.run_stats(rid)
        total = 0
        for i, ref in enumerate(refs):
            off, packed = ctx.read_item(rid, i)
            t, v = gls.unpack(packed)
            assert_same(ref, off, t, v, f"item {i}")
            total += int(ref.off[-1] - ref.off[its[i][0].n_pi])
        assert stats.total_events == total
        # a rerun of the batch gives the same waveforms
        ctx.rerun(rid)
        ctx.run_stats(rid)
        off, packed = ctx.read_item(rid, 3)
        t, v = gls.unpack(packed)
        assert_same(refs[3], off, t, v, "rerun item 3")


def test_batch_of_one_equals_simulate():
    w = synth.make_workload("tiny200", seed=9)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(w.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        a = ctx.simulate(nid, sid)
        b = ctx.simulate_batch([nid], [sid])
        ctx.run_stats(a)
        ctx.run_stats(b)
        oa, pa = ctx.read_all(a)
        ob, pb = ctx.read_item(b, 0)
        assert np.array_equal(oa, ob) and np.array_equal(pa, pb)


def test_batch_errors():
    E = gls.gls
    w = synth.make_workload("tiny200", seed=9)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(w.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        other = ctx.load_stimulus(synth.make_stimulus(5, mean=10, window=1000, seed=1))
        with pytest.raises(gls.GlsError) as ei:
            ctx.simulate_batch([nid, nid], [sid, other])      # PI count mismatch
        assert ei.value.code == E.GLS_EINVAL
        rid = ctx.simulate_batch([nid, nid], [sid, sid])
        ctx.run_stats(rid)
        with pytest.raises(gls.GlsError):
            ctx.read_item(rid, 2)
        with pytest.raises(gls.GlsError):
            ctx.release(sid)                                  # still used by the batch


def _cut(st, t_limit):
    """stimulus restricted to transitions before t_limit (oracle-side reference)"""
    keep = st.t < t_limit
    lens = np.diff(st.off)
    per = np.add.reduceat(keep.astype(np.int64), st.off[:-1]) if len(st.t) else np.zeros(len(lens), np.int64)
    per = np.where(lens > 0, per, 0)
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(per, out=off[1:])
    return synth.Stimulus(off, st.t[keep], st.v[keep])


@pytest.mark.parametrize("schedule", ["dependency", "levels"])
def test_replicas_with_time_limits(schedule):
    nl = synth.make_netlist(10, 600, 12, fanout="pareto", d_min=5, d_max=200, seed=77)
    stims = [synth.make_stimulus(10, mean=300, window=100_000, seed=300 + s) for s in range(3)]
    plan = [(0, None), (1, 40_000), (0, 1), (2, 99_999), (1, 0), (2, 7_777), (0, 55_555)]
    with gls.Context(0) as ctx:
        ctx.set_schedule(schedule)
        nid = ctx.load_netlist(nl)
        sids = [ctx.load_stimulus(st) for st in stims]
        limits = [(1 << 30) - 2 if t is None else t for _, t in plan]
        rid = ctx.simulate_batch([nid] * len(plan), [sids[k] for k, _ in plan], t_limits=limits)
        stats = ctx.run_stats(rid)
        total = 0
        for i, (k, t) in enumerate(plan):
            st = stims[k] if t is None else _cut(stims[k], t)
            ref = oracle.sim_event(nl, st)
            off, packed = ctx.read_item(rid, i)
            tt, vv = gls.unpack(packed)
            assert_same(ref, off, tt, vv, f"replica {i} (stimulus {k}, limit {t})")
            total += int(ref.off[-1] - ref.off[nl.n_pi])
        assert stats.total_events == total
