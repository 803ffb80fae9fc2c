"""GPU parity on the skewed-activity recipe (skew10m) at reduced gate count.

The recipe's shape is kept where it matters for the device path: depth 120,
1% of the primary inputs are clock-like square waves (period 1000 ps) with the
full 50,000 transitions each, the others Poisson with mean 200 transitions
over 2.5e7 ps, values 0/1/X/Z at 0.49/0.49/0.015/0.005, delays 5-200 ps, and a
heavy-tailed fanout.  That gives the recipe's load imbalance (WCV about 7,
Eq. 5): a few nets carry tens of thousands of transitions next to nets with a
few hundred, which stresses the uneven output slots (Eq. 2 bounds), the
carried transitions between chunks and the longest dependency chains.

Every waveform is compared with the oracle's levelized evaluator (independent
code, Algorithm 2 + Eq. 1 per gate on all host cores), under the schedule and
gate order bench.py times (dependency schedule, critical-path-first order
planned from a calibration run), under level order and under one launch per
level."""
import os

import numpy as np
import pytest

import bench
import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu

GATES, PIS, CLOCKS = 200_000, 2_000, 20    # 1% clocks, as in the full recipe


@pytest.fixture(scope="module")
def skew():
    w = synth.make_workload("skew10m", seed=3, net_n_gates=GATES, net_n_pi=PIS, stim_n_clock=CLOCKS)
    ref = oracle.sim_levelized(w.netlist, w.stimulus, nthreads=os.cpu_count() or 1)
    return w, ref


def _run(ctx, nid, sid):
    rid = ctx.simulate(nid, sid)
    rc, demand, _ = ctx.run_stats_raw(rid)
    while rc == gls.gls.GLS_EOVERFLOW:
        ctx.release(rid)
        rid = ctx.simulate(nid, sid, arena_events=int(demand * 1.25) + 1024)
        rc, demand, _ = ctx.run_stats_raw(rid)
    assert rc == 0, f"simulate returned {rc}"
    total = ctx.run_stats(rid).total_events
    off, packed = ctx.read_all(rid)
    ctx.release(rid)
    return total, off, packed


def test_skew_recipe_shape(skew):
    w, ref = skew
    st = w.stimulus
    lens = np.diff(st.off)
    assert int((lens >= 50_000).sum()) == CLOCKS, "clock inputs carry the full 50k transitions"
    assert st.wcv() > 5.0, "the skew of the full recipe (WCV about 7)"
    assert w.recipe["net"]["depth"] == 120
    gl = np.diff(ref.off)[w.netlist.n_pi:]
    assert gl.max() > 40 * max(1.0, gl.mean()), "gate waveforms are as uneven as their inputs"


@pytest.mark.parametrize("schedule,order", [("dependency", "planned"), ("dependency", "level"),
                                            ("levels", "level")])
def test_skew_every_gate_equals_oracle(skew, schedule, order):
    w, ref = skew
    nl, st = w.netlist, w.stimulus
    with gls.Context(0) as ctx:
        ctx.set_schedule(schedule)
        nid = ctx.load_netlist(nl)
        if order == "planned":
            bench.plan_from_calibration(ctx, nid, nl, w.recipe["stim"], 3)
        sid = ctx.load_stimulus(st)
        total, off, packed = _run(ctx, nid, sid)
    t, v = gls.unpack(packed)
    assert total == int(ref.off[-1] - ref.off[nl.n_pi])
    assert_same(ref, off, t, v, f"skew {schedule}/{order}")
