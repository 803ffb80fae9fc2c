"""GPU parity of the planned (critical-path-first) dependency order: the
order is planned from another stimulus of the same netlist, and single and
replicated runs created afterwards still equal the CPU oracle transition by
transition; run_id = -1 restores level order."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", ["windowed", "segmented"])
def test_planned_order_equals_oracle(kernel):
    nl = synth.make_netlist(24, 3000, 14, fanout="pareto", d_min=5, d_max=200, seed=77, shuffle=True)
    calib = synth.make_stimulus(nl.n_pi, mean=40, window=20_000, seed=501)
    stims = [synth.make_stimulus(nl.n_pi, mean=120 + 30 * s, window=60_000, seed=600 + s) for s in range(3)]
    refs = [oracle.sim_event(nl, st) for st in stims]
    with gls.Context(0) as ctx:
        ctx.set_kernel(kernel)
        nid = ctx.load_netlist(nl)
        cid = ctx.load_stimulus(calib)
        rc = ctx.simulate(nid, cid)
        ctx.run_stats(rc)
        ctx.plan_order(nid, rc)
        ctx.release(rc)
        ctx.release(cid)
        sids = [ctx.load_stimulus(st) for st in stims]
        # one instance
        rid = ctx.simulate(nid, sids[0])
        st0 = ctx.run_stats(rid)
        off, packed = ctx.read_all(rid)
        t, v = gls.unpack(packed)
        assert_same(refs[0], off, t, v, "planned single")
        assert st0.total_events == int(refs[0].off[-1] - refs[0].off[nl.n_pi])
        ctx.release(rid)
        # replicated instances (work index -> record, replica)
        rid = ctx.simulate_batch([nid] * 3, sids)
        ctx.run_stats(rid)
        for i in range(3):
            off, packed = ctx.read_item(rid, i)
            t, v = gls.unpack(packed)
            assert_same(refs[i], off, t, v, f"planned replica {i}")
        ctx.release(rid)
        # back to level order
        ctx.plan_order(nid, -1)
        rid = ctx.simulate(nid, sids[1])
        ctx.run_stats(rid)
        off, packed = ctx.read_all(rid)
        t, v = gls.unpack(packed)
        assert_same(refs[1], off, t, v, "level order again")


def test_plan_order_rejects_bad_ids():
    w = synth.make_workload("tiny200", seed=3)
    other = synth.make_workload("tiny200", seed=4)
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(w.netlist)
        nid2 = ctx.load_netlist(other.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        rid = ctx.simulate(nid, sid)
        ctx.run_stats(rid)
        with pytest.raises(gls.GlsError):
            ctx.plan_order(nid2, rid)        # item of another netlist
        with pytest.raises(gls.GlsError):
            ctx.plan_order(nid, rid, 1)      # no item 1
        with pytest.raises(gls.GlsError):
            ctx.plan_order(nid, 12345)       # unknown run
        ctx.plan_order(nid, rid)
