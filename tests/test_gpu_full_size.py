"""Parity at the benchmark's full size, in the configuration bench.py times
(1M gates, default kernel, dependency schedule, critical-path-first order
planned from a calibration run): the oracle re-evaluates every gate from its
fanin waveforms as the GPU produced them (Algorithm 2 + Eq. 1 per gate, on all
host cores); with the primary inputs equal to the stimulus this checks every
waveform exactly, by induction over the levels.  Every waveform also
satisfies the method's invariants: strictly increasing times, no repeated
value, gates never output Z, no gate output X first (a waveform starts from
X)."""
import os

import numpy as np
import pytest

import bench
import oracle
import paper_2304_13398_gb300 as gls
import synth

pytestmark = pytest.mark.gpu


def test_ind1m_every_gate_and_invariants():
    w = synth.make_workload("ind1m", seed=1)
    nl, st = w.netlist, w.stimulus
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        bench.plan_from_calibration(ctx, nid, nl, w.recipe["stim"], 1)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate(nid, sid)
        rc, demand, _ = ctx.run_stats_raw(rid)
        while rc == gls.gls.GLS_EOVERFLOW:
            ctx.release(rid)
            rid = ctx.simulate(nid, sid, arena_events=int(demand * 1.25) + 1024)
            rc, demand, _ = ctx.run_stats_raw(rid)
        assert rc == 0
        total = ctx.run_stats(rid).total_events
        demand, _ = ctx.run_info(rid)
        off, packed = ctx.read_all(rid)
    G, P = nl.n_gates, nl.n_pi
    assert total == int(off[-1] - off[P])
    # the warps' arena blocks keep each slot at its waveform's length: the
    # arena claimed stays well below the gates' Eq. 2 bounds (the sum of their
    # fanin lengths, in whole 128-byte lines) and above the output itself
    lens = np.diff(off)
    bounds = np.add.reduceat(lens[nl.fanin_net], nl.fanin_off[:-1]) if G else np.zeros(0, np.int64)
    bounds = np.where(np.diff(nl.fanin_off) > 0, bounds, 0)
    reserved = int(((bounds + 31) // 32 * 32).sum())
    assert total <= demand < 0.75 * reserved, (total, demand, reserved)
    # the primary inputs come back as given
    np.testing.assert_array_equal(np.diff(off[:P + 1]), np.diff(st.off))
    v = (packed & 3).astype(np.uint8)
    np.testing.assert_array_equal((packed[:off[P]] >> 2).astype(np.int64), st.t)
    np.testing.assert_array_equal(v[:off[P]], st.v)
    # invariants of every gate waveform; times strictly increase iff the
    # packed words (t << 2 | v) do
    gp, gv = packed[off[P]:], v[off[P]:]
    first = np.zeros(len(gp), bool)
    first[(off[P:-1] - off[P])[np.diff(off[P:]) > 0]] = True
    assert np.all((gp[1:] > gp[:-1]) | first[1:]), "times not strictly increasing within a waveform"
    assert np.all((gv[1:] != gv[:-1]) | first[1:]), "repeated value within a waveform"
    assert np.all(gv <= 2), "a gate output Z"
    assert np.all(gv[first] != 2), "a waveform starts with X"
    del gp, gv, first
    t = (packed >> 2).astype(np.int64)
    # every gate re-evaluated by the oracle from the GPU's own fanin waveforms,
    # in four bands of the caller's gate order
    cores = os.cpu_count() or 1
    for g0 in range(0, G, G // 4):
        g1 = min(G, g0 + G // 4)
        bad, first_bad = oracle.check_gates(nl, off, t, v, g0, g1, nthreads=cores)
        assert bad == 0, f"{bad} gates in [{g0}, {g1}) differ from the oracle; first {first_bad}"
